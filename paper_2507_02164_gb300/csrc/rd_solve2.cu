// rd_solve2.cu -- instantiation and launch of the two-lanes-per-polynomial
// solver (rd_solve2.cuh) for degrees 2..12, both storage types, FP64 sweeps
// and FP32 sweeps with the FP64 polish; and the per-degree choice between
// one and two lanes.
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

template <int N, typename In, int MODE>
static int launch_two(const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    using T = typename std::conditional<MODE != MODE_PLAIN, float, double>::type;
    auto kern = solve2_kernel<N, T, In, MODE>;
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    int64_t warps_needed = (a.n + 15) / 16;
    int64_t ctas_needed = (warps_needed + (block / 32) - 1) / (block / 32);
    int64_t grid = (int64_t)per_sm * rd_sm_count_cached();
    if (grid > ctas_needed) grid = ctas_needed;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(a);
    return rd_check_launch("solve2_kernel");
}

template <typename In, int MODE>
static int launch_two_degree(int degree, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    switch (degree) {
    case 2: return launch_two<2, In, MODE>(a, block, ctas_per_sm, st);
    case 3: return launch_two<3, In, MODE>(a, block, ctas_per_sm, st);
    case 4: return launch_two<4, In, MODE>(a, block, ctas_per_sm, st);
    case 5: return launch_two<5, In, MODE>(a, block, ctas_per_sm, st);
    case 6: return launch_two<6, In, MODE>(a, block, ctas_per_sm, st);
    case 7: return launch_two<7, In, MODE>(a, block, ctas_per_sm, st);
    case 8: return launch_two<8, In, MODE>(a, block, ctas_per_sm, st);
    case 9: return launch_two<9, In, MODE>(a, block, ctas_per_sm, st);
    case 10: return launch_two<10, In, MODE>(a, block, ctas_per_sm, st);
    case 11: return launch_two<11, In, MODE>(a, block, ctas_per_sm, st);
    case 12: return launch_two<12, In, MODE>(a, block, ctas_per_sm, st);
    default: return rd_set_error(RD_EUNSUPPORTED, "two-lane solver built for degrees 2..12, not %d", degree);
    }
}

int launch_solve2(int degree, rd_dtype dt, bool mixed, const SolveArgs &a, int block, int ctas_per_sm,
                  cudaStream_t st)
{
    if (mixed) {
        if (dt == RD_C64) return launch_two_degree<float2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
        return launch_two_degree<double2, MODE_MIXED_FP64>(degree, a, block, ctas_per_sm, st);
    }
    if (dt == RD_C64) return launch_two_degree<float2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
    return launch_two_degree<double2, MODE_PLAIN>(degree, a, block, ctas_per_sm, st);
}

}  // namespace rd
