// rd_solve2_mixed.cu -- the two-lane solver for degrees 2..12 with FP32 sweeps
// and the FP64 polish, both storage types.
#include "rd_solve2.cuh"

namespace rd {
int launch_solve2_mixed(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    if (dt == RD_C64) return launch_two_degree<float2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
    return launch_two_degree<double2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
}
}  // namespace rd
