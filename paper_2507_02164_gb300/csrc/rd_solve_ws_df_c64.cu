// rd_solve_ws_df_c64.cu -- the warp-specialised RD_MIXED solver (rd_solve_ws.cuh)
// with the FP32-pipe compensated polish (RD_POLISH_DF), complex64
// coefficients, and the dispatch of that polish by storage type.
#include "rd_solve_ws_launch.cuh"

namespace rd {

int launch_solve_ws_df_c128(int degree, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                            int ring_slots, cudaStream_t st);

int launch_solve_ws_df(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                       int ring_slots, cudaStream_t st)
{
    if (dt == RD_C64)
        return launch_ws_degree<float2, MODE_MIXED_DF>(degree, a, block, ctas_per_sm, polish_warps, ring_slots, st);
    return launch_solve_ws_df_c128(degree, a, block, ctas_per_sm, polish_warps, ring_slots, st);
}

}  // namespace rd
