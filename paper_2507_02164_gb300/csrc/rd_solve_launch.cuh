// rd_solve_launch.cuh -- instantiation and launch of solve_kernel for every
// degree 1..12 and both storage types; included once per precision mode.
#pragma once

#include "rd_solve.cuh"

namespace rd {

template <int N, typename In, int MODE>
static int launch_one(const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    using T = typename std::conditional<MODE != MODE_PLAIN, float, double>::type;
    auto kern = solve_kernel<N, T, In, MODE>;
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    int64_t warps_needed = (a.n + 31) / 32;
    int64_t ctas_needed = (warps_needed + (block / 32) - 1) / (block / 32);
    int64_t grid = (int64_t)per_sm * rd_sm_count_cached();
    if (grid > ctas_needed) grid = ctas_needed;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(a);
    return rd_check_launch("solve_kernel");
}

template <typename In, int MODE>
static int launch_degree(int degree, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st)
{
    switch (degree) {
    case 1: return launch_one<1, In, MODE>(a, block, ctas_per_sm, st);
    case 2: return launch_one<2, In, MODE>(a, block, ctas_per_sm, st);
    case 3: return launch_one<3, In, MODE>(a, block, ctas_per_sm, st);
    case 4: return launch_one<4, In, MODE>(a, block, ctas_per_sm, st);
    case 5: return launch_one<5, In, MODE>(a, block, ctas_per_sm, st);
    case 6: return launch_one<6, In, MODE>(a, block, ctas_per_sm, st);
    case 7: return launch_one<7, In, MODE>(a, block, ctas_per_sm, st);
    case 8: return launch_one<8, In, MODE>(a, block, ctas_per_sm, st);
    case 9: return launch_one<9, In, MODE>(a, block, ctas_per_sm, st);
    case 10: return launch_one<10, In, MODE>(a, block, ctas_per_sm, st);
    case 11: return launch_one<11, In, MODE>(a, block, ctas_per_sm, st);
    case 12: return launch_one<12, In, MODE>(a, block, ctas_per_sm, st);
    default: return rd_set_error(RD_EUNSUPPORTED, "degree %d not built (1..12)", degree);
    }
}

}  // namespace rd
