// rd_solve2.cu -- the per-degree choice between one and two lanes per
// polynomial, and the two-lane solver (rd_solve2.cuh) for degrees 2..12 with
// FP64 sweeps, both storage types (FP32 sweeps: rd_solve2_mixed.cu).
#include "rd_solve2.cuh"

namespace rd {

// Lanes per polynomial: params.lanes when set, else one. Measured on GB300
// (2^20 complex-Gaussian polynomials per degree, best launch shape of each):
// two lanes take 1.14-1.43x the time of one at degrees 6..12 with FP32 sweeps
// and 1.33-1.69x with FP64 sweeps. The pair halves the registers per thread
// but not the FP64-pipe work per polynomial: both lanes form every Givens
// rotation (a warp instruction costs the pipe the same for any active mask),
// and the shuffles and selects add issue slots. The autotuner still times
// both layouts per degree.
int lanes_for(int degree, bool mixed, int polish_mode, int requested)
{
    (void)mixed;
    (void)polish_mode;
    if (degree < 2) return 1;
    return requested == 2 ? 2 : 1;
}

int launch_solve2_mixed(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st);

int launch_solve2(int degree, rd_dtype dt, bool mixed, const SolveArgs &a, int block, int ctas_per_sm,
                  cudaStream_t st)
{
    if (mixed) return launch_solve2_mixed(degree, dt, a, block, ctas_per_sm, st);
    if (dt == RD_C64) return launch_two_degree<float2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
    return launch_two_degree<double2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
}

}  // namespace rd
