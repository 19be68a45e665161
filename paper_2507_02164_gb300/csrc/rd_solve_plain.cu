// rd_solve_plain.cu -- RD_PLAIN_FP64 solver instantiations (FP64 sweeps).
#include "rd_solve_launch.cuh"

namespace rd {
int launch_solve_plain(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    if (dt == RD_C64) return launch_degree<float2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
    return launch_degree<double2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
}
}  // namespace rd
