// rd_solve_mixed.cu -- RD_MIXED solver instantiations (FP32 sweeps + FP64
// polish); the double-float polish variant is in rd_solve_mixed_df.cu.
#include "rd_solve_launch.cuh"

namespace rd {
int launch_solve_mixed_df(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st);

int launch_solve_mixed(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    if (a.polish_mode == RD_POLISH_DF) return launch_solve_mixed_df(degree, dt, a, block, ctas_per_sm, st);
    if (dt == RD_C64) return launch_degree<float2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
    return launch_degree<double2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
}
}  // namespace rd
