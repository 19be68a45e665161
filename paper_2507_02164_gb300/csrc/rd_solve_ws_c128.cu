// rd_solve_ws_c128.cu -- the warp-specialised RD_MIXED solver (rd_solve_ws.cuh)
// with the FP64 polish for complex128 coefficients.
#include "rd_solve_ws_launch.cuh"

namespace rd {

int launch_solve_ws_c128(int degree, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                         int ring_slots, cudaStream_t st)
{
    return launch_ws_degree<double2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, polish_warps, ring_slots, st);
}

}  // namespace rd
