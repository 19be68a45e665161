// rd_solve_mixed_df.cu -- RD_MIXED solver instantiations with the
// double-float polish (RD_POLISH_DF).
#include "rd_solve_launch.cuh"

namespace rd {
int launch_solve_mixed_df(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    if (dt == RD_C64) return launch_degree<float2, MODE_MIXED_DF>(degree, a, block, ctas_per_sm, st);
    return launch_degree<double2, MODE_MIXED_DF>(degree, a, block, ctas_per_sm, st);
}
}  // namespace rd
