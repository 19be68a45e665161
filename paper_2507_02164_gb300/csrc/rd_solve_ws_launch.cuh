// rd_solve_ws_launch.cuh -- host-side launch of the warp-specialised solver
// (rd_solve_ws.cuh): shape validation, the shared-memory opt-in, grid size.
#pragma once

#include <atomic>

#include "rd_solve_ws.cuh"

namespace rd {

// Dynamic shared memory above the default 48 KB needs the kernel's opt-in,
// per device; it is raised once per device to the largest size asked for
// (host calls, outside any stream order), so a graph capture that follows
// the first launch on a device makes none.
template <int N, typename In, int MAXB, int MODE>
static int ws_allow_smem(size_t bytes)
{
    static std::atomic<size_t> allowed[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return rd_check_launch("cudaGetDevice");
    if (dev < 0 || dev >= 64) return rd_set_error(RD_EUNSUPPORTED, "device %d: at most 64 devices", dev);
    if (bytes <= 48 * 1024 || bytes <= allowed[dev].load()) return RD_OK;
    if (cudaFuncSetAttribute(solve_ws_kernel<N, In, MAXB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return rd_check_launch("cudaFuncSetAttribute(solve_ws_kernel)");
    size_t cur = allowed[dev].load();
    while (cur < bytes && !allowed[dev].compare_exchange_weak(cur, bytes)) {
    }
    return RD_OK;
}

template <int N, typename In, int MAXB, int MODE>
static int launch_ws_build(const SolveArgs &a, int block, int ctas_per_sm, int polish_warps, int slots, cudaStream_t st)
{
    const size_t smem = ws_smem_bytes(N, slots);
    int rc = ws_allow_smem<N, In, MAXB, MODE>(smem);
    if (rc) return rc;
    auto kern = solve_ws_kernel<N, In, MAXB, MODE>;
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    const int64_t tasks = (a.n + 31) / 32;
    int64_t grid = (int64_t)per_sm * rd_sm_count_cached();
    if (grid > tasks) grid = tasks;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, smem, st>>>(a, polish_warps, slots);
    return rd_check_launch("solve_ws_kernel");
}

// Validate the shape and launch.
// no_sweep_warps: the self-test of the bounded waits (every warp polishes, so
// no slot is ever filled); otherwise 1 <= polish_warps < block / 32.
template <int N, typename In, int MODE>
static int launch_ws_n(const SolveArgs &a, int block, int ctas_per_sm, int polish_warps, int slots, cudaStream_t st,
                       bool no_sweep_warps = false)
{
    if (block <= 0) block = ws_max_block(N);
    if (block > ws_max_block(N) || block % 32 != 0)
        return rd_set_error(RD_EINVAL, "params.block %d: the warp-specialised solver takes a multiple of 32 up to %d "
                            "at degree %d", block, ws_max_block(N), N);
    const int warps = block / 32;
    if (no_sweep_warps) polish_warps = warps;
    else if (polish_warps < 1 || polish_warps >= warps)
        return rd_set_error(RD_EINVAL, "params.polish_warps %d must be in [1, %d] for block %d", polish_warps,
                            warps - 1, block);
    if (slots <= 0) slots = 2 * warps < WS_MAX_SLOTS ? 2 * warps : WS_MAX_SLOTS;
    if (slots < 2 || slots > WS_MAX_SLOTS)
        return rd_set_error(RD_EINVAL, "params.ring_slots must be 0 or in [2, %d]", WS_MAX_SLOTS);
    return launch_ws_build<N, In, ws_max_block(N), MODE>(a, block, ctas_per_sm, polish_warps, slots, st);
}

template <typename In, int MODE>
static int launch_ws_degree(int degree, const SolveArgs &a, int block, int cps, int pw, int slots, cudaStream_t st)
{
    switch (degree) {
    case 1: return launch_ws_n<1, In, MODE>(a, block, cps, pw, slots, st);
    case 2: return launch_ws_n<2, In, MODE>(a, block, cps, pw, slots, st);
    case 3: return launch_ws_n<3, In, MODE>(a, block, cps, pw, slots, st);
    case 4: return launch_ws_n<4, In, MODE>(a, block, cps, pw, slots, st);
    case 5: return launch_ws_n<5, In, MODE>(a, block, cps, pw, slots, st);
    case 6: return launch_ws_n<6, In, MODE>(a, block, cps, pw, slots, st);
    case 7: return launch_ws_n<7, In, MODE>(a, block, cps, pw, slots, st);
    case 8: return launch_ws_n<8, In, MODE>(a, block, cps, pw, slots, st);
    case 9: return launch_ws_n<9, In, MODE>(a, block, cps, pw, slots, st);
    case 10: return launch_ws_n<10, In, MODE>(a, block, cps, pw, slots, st);
    case 11: return launch_ws_n<11, In, MODE>(a, block, cps, pw, slots, st);
    case 12: return launch_ws_n<12, In, MODE>(a, block, cps, pw, slots, st);
    default: return rd_set_error(RD_EUNSUPPORTED, "degree %d not built (1..12)", degree);
    }
}

}  // namespace rd
