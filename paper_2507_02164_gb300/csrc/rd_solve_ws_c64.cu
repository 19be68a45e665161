// rd_solve_ws_c64.cu -- the warp-specialised RD_MIXED solver (rd_solve_ws.cuh)
// with the FP64 polish for complex64 coefficients, the dispatch by storage
// type and polish mode, and the self-test of its bounded waits.
#include "rd_solve_ws_launch.cuh"

namespace rd {

int launch_solve_ws_c128(int degree, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                         int ring_slots, cudaStream_t st);
int launch_solve_ws_df(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                       int ring_slots, cudaStream_t st);

int launch_solve_ws(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                    int ring_slots, cudaStream_t st)
{
    if (a.polish_mode == RD_POLISH_DF)
        return launch_solve_ws_df(degree, dt, a, block, ctas_per_sm, polish_warps, ring_slots, st);
    if (dt == RD_C64)
        return launch_ws_degree<float2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, polish_warps, ring_slots, st);
    return launch_solve_ws_c128(degree, a, block, ctas_per_sm, polish_warps, ring_slots, st);
}

int launch_solve_ws_selftest(const SolveArgs &a, cudaStream_t st)
{
    return launch_ws_n<6, float2, MODE_MIXED_FP64>(a, 64, 1, 0, 2, st, true);
}

}  // namespace rd
