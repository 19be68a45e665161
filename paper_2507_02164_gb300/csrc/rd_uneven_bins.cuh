// rd_uneven_bins.cuh -- the persistent solve kernels of the uneven-degree
// path (one per degree, tasks pulled from the bin's atomic queue) and
// launch_uneven_bins. Included only by the rd_uneven_bins_*.cu files, each
// of which instantiates it for one storage type and precision mode.
#pragma once

#include <atomic>

#include "rd_solve2.cuh"
#include "rd_solve_ws.cuh"
#include "rd_uneven.cuh"

namespace rd {


// Persistent solver for the degree-N bin: each warp takes the next task of
// the bin's queue (task = 32 consecutive slots) until the queue is empty.
// One kernel per degree keeps each degree's own register allocation.
template <int N, typename In, int MODE>
__global__ void __launch_bounds__(256, (MODE != MODE_PLAIN && N <= 6) ? 2 : 1)
    uneven_solve_kernel(SolveArgs A, UnevenHeader *hdr, const uint32_t *perm, const char *bins, const int64_t *offsets)
{
    using T = typename std::conditional<MODE != MODE_PLAIN, float, double>::type;
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, A.stats);
    const int lane = threadIdx.x & 31;
    const int64_t cnt = hdr->count[N];
    const unsigned tasks = (unsigned)((cnt + 31) / 32);
    const PackedMap map{{}, perm + hdr->poly_base[N], offsets};
    const void *base = bins + (size_t)hdr->coef_base[N] * sizeof(In);
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&hdr->head[N], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= tasks) break;
        solve_warp<N, T, In, MODE>(A, base, cnt, (int64_t)t * 32, map, S);
    }
    stats_end(S, A.stats);
}

// The same with two lanes per polynomial (rd_solve2.cuh): tasks of 16 slots.
template <int N, typename In, int MODE>
__global__ void __maxnreg__(two_lane_regs(N, MODE))
    uneven_solve2_kernel(SolveArgs A, UnevenHeader *hdr, const uint32_t *perm, const char *bins, const int64_t *offsets)
{
    using T = typename std::conditional<MODE != MODE_PLAIN, float, double>::type;
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, A.stats);
    const int lane = threadIdx.x & 31;
    const int64_t cnt = hdr->count[N];
    const unsigned tasks = (unsigned)((cnt + 15) / 16);
    const PackedMap map{{}, perm + hdr->poly_base[N], offsets};
    const void *base = bins + (size_t)hdr->coef_base[N] * sizeof(In);
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&hdr->head[N], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= tasks) break;
        solve_warp2<N, T, In, MODE>(A, base, cnt, (int64_t)t * 16, map, S);
    }
    stats_end(S, A.stats);
}

// The warp-specialised form (rd_solve_ws.cuh) of the degree-N bin: sweep
// warps and polish warps meet at a shared-memory ring; CTA b takes the bin's
// tasks b, b + G, ... (the bin's size is read on the device). Built for the
// degrees up to UNEVEN_WS_MAX_DEG, where the split measured faster than the
// one-role kernel.
constexpr int UNEVEN_WS_MAX_DEG = 8;

template <int N, typename In, int MAXB, int MODE>
__global__ void __launch_bounds__(MAXB, 1)
    uneven_solve_ws_kernel(SolveArgs A, UnevenHeader *hdr, const uint32_t *perm, const char *bins,
                           const int64_t *offsets, int polish_warps, int slots)
{
    const int64_t cnt = hdr->count[N];
    const PackedMap map{{}, perm + hdr->poly_base[N], offsets};
    const void *base = bins + (size_t)hdr->coef_base[N] * sizeof(In);
    ws_cta<N, In, MODE>(A, base, cnt, map, polish_warps, slots);
}

// Dynamic shared memory above 48 KB needs the kernel's opt-in, per device
// (raised once per device to the largest size asked for; host calls only).
template <int N, typename In, int MAXB, int MODE>
static int uneven_ws_allow_smem(size_t bytes)
{
    static std::atomic<size_t> allowed[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return rd_check_launch("cudaGetDevice");
    if (dev < 0 || dev >= 64) return rd_set_error(RD_EUNSUPPORTED, "device %d: at most 64 devices", dev);
    if (bytes <= 48 * 1024 || bytes <= allowed[dev].load()) return RD_OK;
    if (cudaFuncSetAttribute(uneven_solve_ws_kernel<N, In, MAXB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return rd_check_launch("cudaFuncSetAttribute(uneven_solve_ws_kernel)");
    size_t cur = allowed[dev].load();
    while (cur < bytes && !allowed[dev].compare_exchange_weak(cur, bytes)) {
    }
    return RD_OK;
}

template <int N, typename In, int MODE>
static int launch_uneven_ws(const SolveArgs &a, const UnevenLayout &L, const int64_t *offsets, int block,
                            int polish_warps, cudaStream_t st)
{
    constexpr int MAXB = ws_max_block(N);
    const int warps = block / 32;
    const int slots = 2 * warps < WS_MAX_SLOTS ? 2 * warps : WS_MAX_SLOTS;
    const size_t smem = ws_smem_bytes(N, slots);
    int rc = uneven_ws_allow_smem<N, In, MAXB, MODE>(smem);
    if (rc) return rc;
    auto kern = uneven_solve_ws_kernel<N, In, MAXB, MODE>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    kern<<<per_sm * rd_sm_count_cached(), block, smem, st>>>(a, L.hdr, L.perm, L.bins, offsets, polish_warps, slots);
    return rd_check_launch("uneven_solve_ws_kernel");
}

int lanes_for(int degree, bool mixed, int polish_mode, int requested);

template <typename K>
static int launch_persistent(K kern, const SolveArgs &a, const UnevenLayout &L, const int64_t *offsets, int block,
                             int ctas_per_sm, cudaStream_t st, const char *what)
{
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    int grid = per_sm * rd_sm_count_cached();
    kern<<<grid, block, 0, st>>>(a, L.hdr, L.perm, L.bins, offsets);
    return rd_check_launch(what);
}

template <int N, typename In, int MODE>
static int launch_degree_bin(const SolveArgs &a, const UnevenLayout &L, const int64_t *offsets, int block,
                             int ctas_per_sm, int lanes, int polish_warps, cudaStream_t st)
{
    if constexpr (MODE != MODE_PLAIN && N <= UNEVEN_WS_MAX_DEG) {
        if (polish_warps > 0) return launch_uneven_ws<N, In, MODE>(a, L, offsets, block, polish_warps, st);
    }
    if constexpr (N >= 2 && MODE != MODE_MIXED_DF) {
        if (lanes_for(N, MODE != MODE_PLAIN, a.polish_mode, lanes) == 2)
            return launch_persistent(uneven_solve2_kernel<N, In, MODE>, a, L, offsets, block, ctas_per_sm, st,
                                     "uneven_solve2_kernel");
    }
    return launch_persistent(uneven_solve_kernel<N, In, MODE>, a, L, offsets, block, ctas_per_sm, st,
                             "uneven_solve_kernel");
}

// The twelve degree bins run as two chains of persistent kernels, forked from
// the caller's stream onto a helper stream and joined back (under stream
// capture: two parallel graph branches), so that one chain's kernels take
// over the SMs the other chain's kernel leaves while its queue drains
// (fork_bins = false: all on the caller's stream, no helper stream). Work
// per bin grows about as d^2.5; the chains hold about equal shares, each
// largest first: 12, 9, 8, 5, 2, 1 on the caller's stream and 11, 10, 7, 6, 4,
// 3 on the helper.
template <typename In, int MODE>
int launch_uneven_bins(const SolveArgs &a, const UnevenLayout &L, const int64_t *offsets, const int *block,
                       const int *cps, const int *lanes, const int *pw, bool fork_bins, cudaStream_t st)
{
    cudaStream_t side = st;
    cudaEvent_t fork = nullptr, join = nullptr;
    int rc = fork_bins ? uneven_fork(st, &side, &fork, &join) : RD_OK;
    if (rc) return rc;
#define RD_BIN(D, S) \
    if (!rc) rc = launch_degree_bin<D, In, MODE>(a, L, offsets, block[D], cps[D], lanes[D], pw[D], S);
    RD_BIN(11, side) RD_BIN(12, st) RD_BIN(10, side) RD_BIN(9, st) RD_BIN(7, side) RD_BIN(8, st)
    RD_BIN(6, side) RD_BIN(5, st) RD_BIN(4, side) RD_BIN(2, st) RD_BIN(3, side) RD_BIN(1, st)
#undef RD_BIN
    const int rj = fork_bins ? uneven_join(st, side, join) : RD_OK;
    return rc ? rc : rj;
}

}  // namespace rd

#define RD_UNEVEN_BINS(IN, MODE)                                                                          \
    namespace rd {                                                                                      \
    template int launch_uneven_bins<IN, MODE>(const SolveArgs &, const UnevenLayout &, const int64_t *, \
                                              const int *, const int *, const int *, const int *, bool, \
                                              cudaStream_t);                                            \
    }
