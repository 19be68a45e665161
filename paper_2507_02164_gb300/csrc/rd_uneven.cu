// rd_uneven.cu -- polynomials of uneven degree (1..12) in one pass: bin the
// batch by degree, then solve every bin with persistent kernels that pull
// 32-polynomial tasks from atomic queues.
//
// The paper solves one degree at a time (n <= 6, Sec. II-A, Table III). A
// batch of mixed degrees would otherwise run every polynomial at the largest
// degree's cost, or diverge inside warps; binning gives each warp one
// compile-time degree, so the Hessenberg matrix stays in registers.
//
// Workspace (caller-allocated, contents overwritten, 256-byte aligned):
//   [header 512 B][perm: uint32 per polynomial][bins: the coefficients again,
//   coefficient-major within each degree bin]
// Launch sequence on the caller's stream (graph-capturable, no allocation,
// no synchronisation): clear header -> count -> scan -> pack -> one
// persistent solve kernel per degree, largest degree first, each with its
// own register allocation and its own task queue.
#include "rd_uneven.cuh"

namespace rd {

int launch_clear(uint32_t *p, int64_t words, cudaStream_t st);


struct UnevenArgs {
    const uint8_t *degrees;
    const int64_t *offsets;
    int64_t n;
    int64_t n_coeffs;
};

// A polynomial is solvable when its offsets hold exactly degree + 1
// coefficients, its degree is 1..12, and its roots fit the packed root array
// of n_coeffs - n elements: o0 >= i keeps root 0 (at o0 - i) at or above 0,
// o1 <= n_coeffs - (n - 1 - i) keeps its last root (at o1 - i - 2) below
// n_coeffs - n. The comparisons are ordered so that no difference overflows.
// These bounds hold for each polynomial alone; polynomials whose ranges
// overlap (offsets that are not monotone) are caught by the total the scan
// kernel checks.
__device__ __forceinline__ int checked_degree(const UnevenArgs &U, int64_t i, bool &consistent)
{
    int d = __ldg(U.degrees + i);
    int64_t o0 = __ldg(U.offsets + i), o1 = __ldg(U.offsets + i + 1);
    consistent = (o0 >= i) && (o1 >= o0) && (o1 <= U.n_coeffs - (U.n - 1 - i)) && (o1 - o0 == (int64_t)d + 1);
    return (consistent && d >= 1 && d <= UNEVEN_MAX_DEG) ? d : -1;
}

// NaN roots of polynomial i (its offsets passed checked_degree's bounds).
__device__ __forceinline__ void nan_roots(const UnevenArgs &U, int64_t i, double *roots)
{
    if (!roots) return;
    const int dd = __ldg(U.degrees + i);
    const int64_t r0 = __ldg(U.offsets + i) - i;
    const double q = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = 0; j < dd; ++j) reinterpret_cast<double2 *>(roots)[r0 + j] = make_double2(q, q);
}

// Count polynomials per degree; mark the unsolvable ones DEGENERATE (NaN
// roots where the offsets are consistent, nothing written where they are not).
__global__ void __launch_bounds__(256) uneven_count_kernel(UnevenArgs U, UnevenHeader *hdr, double *roots,
                                                           uint8_t *status, rd_stats *stats)
{
    __shared__ unsigned cnt[16];
    __shared__ unsigned long long acc[ST_WORDS];
    if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
    const CtaStats S = stats_begin(acc, stats);  // synchronises the CTA
    __syncthreads();
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    unsigned bad = 0, invalid = 0;
    for (int64_t base = warp_id * 32; base < U.n; base += warps_total * 32) {
        int64_t i = base + lane;
        if (i < U.n) {
            bool consistent;
            int d = checked_degree(U, i, consistent);
            if (d > 0) {
                atomicAdd(&cnt[d], 1u);
            } else {
                invalid += 1;
                bad += consistent ? 0u : 1u;
                if (status) status[i] = RD_STATUS_DEGENERATE;
                if (consistent) nan_roots(U, i, roots);
            }
        }
    }
    S.add(ST_POLYS, invalid);
    S.add(ST_STATUS0 + RD_STATUS_DEGENERATE, invalid);
    unsigned wb = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0 && wb) atomicAdd(&hdr->bad, wb);
    __syncthreads();
    if (threadIdx.x < 16 && cnt[threadIdx.x]) atomicAdd(&hdr->count[threadIdx.x], cnt[threadIdx.x]);
    stats_end(S, stats);
}

// Bin bases: poly_base[d] = sum of count[d'] for d' < d, coef_base[d] = sum
// of count[d'] (d' + 1). One warp. When the solvable polynomials need more
// than n_coeffs coefficients in all, their ranges overlap (offsets that are
// not monotone) and the bins would not fit the workspace: the batch is then
// not packed or solved (overflow = 1, every count 0), and the pack kernel
// marks its solvable polynomials DEGENERATE instead.
__global__ void uneven_scan_kernel(UnevenHeader *hdr, int64_t n_coeffs)
{
    const int lane = threadIdx.x;
    unsigned c = lane < 16 ? hdr->count[lane] : 0u;
    int64_t e = lane < 16 ? (int64_t)c * (lane + 1) : 0;
    unsigned pc = c;
    int64_t pe = e;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned oc = __shfl_up_sync(0xffffffffu, pc, off);
        int64_t oe = __shfl_up_sync(0xffffffffu, pe, off);
        if (lane >= off) {
            pc += oc;
            pe += oe;
        }
    }
    const int64_t total = __shfl_sync(0xffffffffu, pe, 31);
    const bool overflow = total > n_coeffs;
    if (lane < 16) {
        hdr->poly_base[lane] = pc - c;  // exclusive
        hdr->coef_base[lane] = pe - e;
        hdr->cursor[lane] = 0;
        hdr->head[lane] = 0;
        if (overflow) hdr->count[lane] = 0;
    }
    if (lane == 0) hdr->overflow = overflow ? 1u : 0u;
}

// Scatter every solvable polynomial into its degree's bin: a slot from a
// warp-aggregated cursor, perm[slot] = its index, its coefficients
// coefficient-major at bins[coef_base[d] + k * count[d] + slot].
template <typename E>
__global__ void __launch_bounds__(256) uneven_pack_kernel(UnevenArgs U, const E *__restrict__ coeffs,
                                                          UnevenHeader *hdr, uint32_t *perm, E *bins,
                                                          double *roots, uint8_t *status, rd_stats *stats)
{
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (hdr->overflow) {
        // overlapping ranges: nothing is packed; the solvable polynomials are
        // reported DEGENERATE with NaN roots (their own bounds hold)
        __shared__ unsigned long long acc[ST_WORDS];
        const CtaStats S = stats_begin(acc, stats);
        unsigned marked = 0;
        for (int64_t base = warp_id * 32; base < U.n; base += warps_total * 32) {
            int64_t i = base + lane;
            bool consistent;
            if (i < U.n && checked_degree(U, i, consistent) > 0) {
                marked += 1;
                if (status) status[i] = RD_STATUS_DEGENERATE;
                nan_roots(U, i, roots);
            }
        }
        S.add(ST_POLYS, marked);
        S.add(ST_STATUS0 + RD_STATUS_DEGENERATE, marked);
        stats_end(S, stats);
        return;
    }
    for (int64_t base = warp_id * 32; base < U.n; base += warps_total * 32) {
        int64_t i = base + lane;
        int d = -1;
        if (i < U.n) {
            bool consistent;
            d = checked_degree(U, i, consistent);
        }
        unsigned act = __ballot_sync(0xffffffffu, d > 0);
        if (d > 0) {
            unsigned peers = __match_any_sync(act, d);
            int leader = __ffs(peers) - 1;
            unsigned rank = __popc(peers & ((1u << lane) - 1u));
            unsigned b = 0;
            if (lane == leader) b = atomicAdd(&hdr->cursor[d], (unsigned)__popc(peers));
            b = __shfl_sync(peers, b, leader);
            unsigned slot = b + rank;
            unsigned cnt = hdr->count[d];
            perm[hdr->poly_base[d] + slot] = (uint32_t)i;
            const E *src = coeffs + __ldg(U.offsets + i);
            E *dst = bins + hdr->coef_base[d] + slot;
            for (int k = 0; k <= d; ++k) dst[(int64_t)k * cnt] = __ldg(src + k);
        }
    }
}

namespace {
// The helper stream and its two events, per device, owned by one host thread
// and released when that thread exits (errors ignored: at process exit the
// runtime may already be gone).
struct ForkState {
    int device = -1;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~ForkState()
    {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
    }
};
thread_local ForkState g_fork[64];
}  // namespace

int uneven_fork(cudaStream_t st, cudaStream_t *side, cudaEvent_t *fork, cudaEvent_t *join, bool retry)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rd_set_error(RD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return rd_set_error(RD_EUNSUPPORTED, "device index %d above 63", dev);
    ForkState &f = g_fork[dev];
    if (!f.side) {
        // all three or none: a partial failure releases what it made
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming)) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            if (s) cudaStreamDestroy(s);
            return rd_set_error(RD_ECUDA, "uneven helper stream: %s (the first call on a device from a host thread "
                                          "creates it; make that call outside stream capture)",
                                cudaGetErrorString(e));
        }
        f.side = s;
        f.fork = a;
        f.join = b;
        f.device = dev;
    }
    if ((e = cudaEventRecord(f.fork, st)) != cudaSuccess || (e = cudaStreamWaitEvent(f.side, f.fork, 0)) != cudaSuccess) {
        // handles made before a cudaDeviceReset are gone: forget them (they
        // cannot be destroyed any more) and make new ones, once
        if (e != cudaErrorInvalidResourceHandle || retry) return rd_set_error(RD_ECUDA, "uneven fork: %s", cudaGetErrorString(e));
        cudaGetLastError();
        f.side = nullptr;
        f.fork = f.join = nullptr;
        return uneven_fork(st, side, fork, join, true);
    }
    *side = f.side;
    *fork = f.fork;
    *join = f.join;
    return RD_OK;
}

int uneven_join(cudaStream_t st, cudaStream_t side, cudaEvent_t join)
{
    cudaError_t e;
    if ((e = cudaEventRecord(join, side)) != cudaSuccess || (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
        return rd_set_error(RD_ECUDA, "uneven join: %s", cudaGetErrorString(e));
    return RD_OK;
}

size_t uneven_workspace_bytes(int64_t n, int64_t n_coeffs, rd_dtype dt)
{
    if (!uneven_sizes_ok(n, n_coeffs)) return 0;
    return uneven_bytes(n, n_coeffs, dt == RD_C64 ? 8 : 16);
}

int launch_uneven(const SolveArgs &a, rd_dtype dt, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                  int64_t n_coeffs, bool mixed, void *ws, const int *block, const int *cps, const int *lanes,
                  const int *pw, bool fork, cudaStream_t st)
{
    UnevenLayout L = uneven_layout(ws, n);
    UnevenArgs U{degrees, offsets, n, n_coeffs};
    int rc = launch_clear(reinterpret_cast<uint32_t *>(L.hdr), UNEVEN_HEADER_BYTES / 4, st);
    if (rc) return rc;
    const int tb = 256;
    int64_t ctas = (n + tb - 1) / tb;
    int64_t cap = (int64_t)rd_sm_count_cached() * 8;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    uneven_count_kernel<<<(unsigned)ctas, tb, 0, st>>>(U, L.hdr, a.roots, a.status, a.stats);
    if ((rc = rd_check_launch("uneven_count_kernel"))) return rc;
    uneven_scan_kernel<<<1, 32, 0, st>>>(L.hdr, n_coeffs);
    if ((rc = rd_check_launch("uneven_scan_kernel"))) return rc;
    if (dt == RD_C64)
        uneven_pack_kernel<float2><<<(unsigned)ctas, tb, 0, st>>>(U, reinterpret_cast<const float2 *>(a.coeffs), L.hdr,
                                                                  L.perm, reinterpret_cast<float2 *>(L.bins), a.roots,
                                                                  a.status, a.stats);
    else
        uneven_pack_kernel<double2><<<(unsigned)ctas, tb, 0, st>>>(U, reinterpret_cast<const double2 *>(a.coeffs),
                                                                   L.hdr, L.perm, reinterpret_cast<double2 *>(L.bins),
                                                                   a.roots, a.status, a.stats);
    if ((rc = rd_check_launch("uneven_pack_kernel"))) return rc;
    const int mode = !mixed ? MODE_PLAIN : (a.polish_mode == RD_POLISH_DF ? MODE_MIXED_DF : MODE_MIXED_FP64);
    if (dt == RD_C64) {
        if (mode == MODE_PLAIN) return launch_uneven_bins<float2, MODE_PLAIN>(a, L, offsets, block, cps, lanes, pw, fork, st);
        if (mode == MODE_MIXED_DF) return launch_uneven_bins<float2, MODE_MIXED_DF>(a, L, offsets, block, cps, lanes, pw, fork, st);
        return launch_uneven_bins<float2, MODE_MIXED_FP64>(a, L, offsets, block, cps, lanes, pw, fork, st);
    }
    if (mode == MODE_PLAIN) return launch_uneven_bins<double2, MODE_PLAIN>(a, L, offsets, block, cps, lanes, pw, fork, st);
    if (mode == MODE_MIXED_DF) return launch_uneven_bins<double2, MODE_MIXED_DF>(a, L, offsets, block, cps, lanes, pw, fork, st);
    return launch_uneven_bins<double2, MODE_MIXED_FP64>(a, L, offsets, block, cps, lanes, pw, fork, st);
}

}  // namespace rd
