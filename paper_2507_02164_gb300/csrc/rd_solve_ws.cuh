// rd_solve_ws.cuh -- warp-specialised RD_MIXED solver (FP32 sweeps, FP64
// polish) for a uniform batch.
//
// In the one-role kernel (solve_kernel) every warp sweeps 32 polynomials on
// the FP32 pipe and then polishes them on the FP64 pipe, which GB300 runs 64x
// slower. The FP64 pipe idles whenever all warps of an SM sub-partition
// happen to be sweeping: on the degree-6 Littlewood batch the sweeps alone
// take a third of the one-role kernel's time and the FP64 pipe is busy 80 %
// of it. Here each CTA splits its warps into two roles:
//
//   sweep warps   load, normalise and sweep 32 polynomials (sweep_lane), put
//                 the FP32 eigenvalues and the flags into a ring slot;
//   polish warps  take the slot, polish, check, write status and roots, and
//                 bin them (finish_lane: the same code as the one-role kernel,
//                 so the roots are the same bit for bit).
//
// Hand-off: the CTA's tasks (32 polynomials each; CTA b takes tasks b, b + G,
// b + 2G, ... of the grid's G CTAs) are numbered by two tickets in shared
// memory, one for each role. Sweep ticket k fills slot k mod S in round
// k / S; polish ticket k empties it. A slot's state word counts its
// hand-offs: 2r = empty for round r, 2r + 1 = full in round r. A sweep warp
// waits only for the polish warp of ticket k - S, which waits only for the
// sweep warp of ticket k - S, and so on down to the first S tickets, which
// wait for nothing: the protocol cannot deadlock. Every wait is still bounded
// (%globaltimer): a wait that runs out sets the CTA's abort flag, after which
// no warp waits again, sweep warps stop, and polish warps mark each task they
// could not take REJECTED and count it in rd_stats.wait_timeouts.
#pragma once

#include "rd_solve.cuh"

namespace rd {

constexpr int WS_MAX_SLOTS = 64;
constexpr unsigned long long WS_WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr unsigned WS_MAX_POLLS = 1u << 26;               // and at most this many polls

// One ring slot: the FP32 eigenvalues of a task, lane-major per eigenvalue
// (a warp's 32 stores or loads of eigenvalue j are 256 contiguous bytes),
// and the task's per-lane flags as warp ballots.
template <int N>
struct WsSlot {
    float2 d[N][32];
    unsigned degenerate;
    unsigned not_conv;
    unsigned pad[2];
};

struct WsCtl {
    unsigned sweep_ticket;
    unsigned polish_ticket;
    unsigned abort;
    unsigned pad;
    unsigned state[WS_MAX_SLOTS];
};

__host__ __device__ constexpr size_t ws_smem_bytes(int n, int slots)
{
    return sizeof(WsCtl) + (size_t)slots * ((size_t)n * 32 * sizeof(float2) + 16);
}

// Threads per CTA: up to 16 warps at 116 registers for degrees <= 6, up to 8
// warps at 255 registers above (the larger Hessenberg matrices). (A 20-warp
// build for degree 6 needs 96 registers and spills; measured slower.)
__host__ __device__ constexpr int ws_max_block(int n) { return n <= 6 ? 512 : 256; }

__device__ __forceinline__ unsigned long long ws_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *state == want (all 32 lanes call it; the result is
// warp-uniform). false: the CTA is aborting, or this wait ran out of time
// and started the abort.
__device__ __forceinline__ bool ws_wait(const volatile unsigned *state, unsigned want, volatile unsigned *abort_flag)
{
    bool ok = *state == want;
    if (!__all_sync(0xffffffffu, ok)) {
        const unsigned long long t0 = ws_clock_ns();
        bool gave_up = false;
        for (unsigned it = 0; !ok && !gave_up; ++it) {
            if (*abort_flag) {
                gave_up = true;
                break;
            }
            __nanosleep(2048);
            ok = *state == want;
            if (!ok && ((it & 63u) == 63u || it >= WS_MAX_POLLS) &&
                (it >= WS_MAX_POLLS || ws_clock_ns() - t0 > WS_WAIT_NS)) {
                *abort_flag = 1u;
                gave_up = true;
            }
        }
        ok = __all_sync(0xffffffffu, ok && !gave_up);
        if (!ok) *abort_flag = 1u;
    }
    __threadfence_block();  // what the other role wrote before moving the state is visible after it
    return ok;
}

// Publish a slot's new state once all 32 lanes' shared-memory accesses of it are done.
__device__ __forceinline__ void ws_publish(volatile unsigned *state, unsigned value)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();
        *state = value;
    }
}

// Put swept task k (its FP32 eigenvalues d and per-lane flags) into ring
// slot k mod slots once the slot is empty for round k / slots; all 32 lanes
// call it together. false: the CTA is aborting.
template <int N>
__device__ __forceinline__ bool ws_put(WsCtl *ctl, WsSlot<N> *ring, int slots, unsigned k, const cx<float> (&d)[N],
                                       bool degenerate, bool not_conv, volatile unsigned *abort_flag)
{
    const int lane = threadIdx.x & 31;
    const unsigned slot = k % (unsigned)slots, round = k / (unsigned)slots;
    if (!ws_wait(&ctl->state[slot], 2u * round, abort_flag)) return false;
    WsSlot<N> &w = ring[slot];
#pragma unroll
    for (int j = 0; j < N; ++j) w.d[j][lane] = make_float2(d[j].re, d[j].im);
    const unsigned dm = __ballot_sync(0xffffffffu, degenerate);
    const unsigned nm = __ballot_sync(0xffffffffu, not_conv);
    if (lane == 0) {
        w.degenerate = dm;
        w.not_conv = nm;
    }
    ws_publish(&ctl->state[slot], 2u * round + 1u);
    return true;
}

// The polish role of a warp-specialised CTA: take polish tickets until the
// CTA's my_tasks tasks are done; each task's slot is emptied and its 32
// polynomials finished (finish_lane). A task whose slot never fills (the CTA
// aborted) is reported REJECTED and counted as a wait timeout.
template <int N, typename In, int MODE, class Map>
__device__ __forceinline__ void ws_polish_role(const SolveArgs &A, const void *coeffs, int64_t n, const Map &map,
                                               const CtaStats &S, WsCtl *ctl, const WsSlot<N> *ring, int slots,
                                               unsigned my_tasks, volatile unsigned *abort_flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x, b = blockIdx.x;
    for (;;) {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(&ctl->polish_ticket, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= my_tasks) break;
        const int64_t i = (b + (int64_t)k * G) * 32 + lane;
        const unsigned slot = k % (unsigned)slots, round = k / (unsigned)slots;
        if (!ws_wait(&ctl->state[slot], 2u * round + 1u, abort_flag)) {
            // abandoned: its polynomials are reported, not solved
            const bool valid = i < n;
            if (valid && A.status) A.status[map.poly(i)] = RD_STATUS_REJECTED;
            S.add(ST_POLYS, valid ? 1u : 0u);
            S.add(ST_STATUS0 + RD_STATUS_REJECTED, valid ? 1u : 0u);
            S.add(ST_TIMEOUT, valid ? 1u : 0u);
            continue;
        }
        const WsSlot<N> &w = ring[slot];
        cx<float> d[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 v = w.d[j][lane];
            d[j] = {v.x, v.y};
        }
        const bool degenerate = (w.degenerate >> lane) & 1u;
        const bool not_conv = (w.not_conv >> lane) & 1u;
        ws_publish(&ctl->state[slot], 2u * round + 2u);
        finish_lane<N, float, In, MODE>(A, coeffs, n, i, map, S, d, degenerate, not_conv);
    }
}

// One warp-specialised CTA over a coefficient-major batch `coeffs` of n
// polynomials of degree N whose results go where `map` says (a uniform batch,
// or one degree bin of a packed batch): blockDim.x / 32 warps, the first
// polish_warps of them (1 .. blockDim.x / 32 - 1) polishing; `slots`
// (2 .. WS_MAX_SLOTS) ring slots in the dynamic shared memory
// (ws_smem_bytes(N, slots)). CTA b of the grid's G takes the tasks
// (32 polynomials each) b, b + G, b + 2G, ...
template <int N, typename In, int MODE, class Map>
__device__ __forceinline__ void ws_cta(const SolveArgs &A, const void *coeffs, int64_t n, const Map &map,
                                       int polish_warps, int slots)
{
    static_assert(MODE == MODE_MIXED_FP64 || MODE == MODE_MIXED_DF, "the warp-specialised solver is mixed-mode");
    extern __shared__ __align__(16) unsigned char ws_smem[];
    WsCtl *ctl = reinterpret_cast<WsCtl *>(ws_smem);
    WsSlot<N> *ring = reinterpret_cast<WsSlot<N> *>(ws_smem + sizeof(WsCtl));
    __shared__ unsigned long long acc[ST_WORDS];
    if (threadIdx.x == 0) {
        ctl->sweep_ticket = 0;
        ctl->polish_ticket = 0;
        ctl->abort = 0;
    }
    if (threadIdx.x < WS_MAX_SLOTS) ctl->state[threadIdx.x] = 0;
    __syncthreads();
    const CtaStats S = stats_begin(acc, A.stats);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tasks = (n + 31) / 32;
    const int64_t G = gridDim.x, b = blockIdx.x;
    const unsigned my_tasks = b < tasks ? (unsigned)((tasks - b + G - 1) / G) : 0u;
    volatile unsigned *abort_flag = &ctl->abort;

    if (warp >= polish_warps) {
        for (;;) {
            unsigned k = 0;
            if (lane == 0) k = atomicAdd(&ctl->sweep_ticket, 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
            // a warp vote: the sweep below needs all 32 lanes, whatever each read of abort saw
            if (__any_sync(0xffffffffu, k >= my_tasks || *abort_flag)) break;
            const int64_t i = (b + (int64_t)k * G) * 32 + lane;
            cx<float> d[N];
            bool degenerate, not_conv;
            sweep_lane<N, float, In, MODE>(A, coeffs, n, i, S, d, degenerate, not_conv);
            if (!ws_put<N>(ctl, ring, slots, k, d, degenerate, not_conv, abort_flag)) break;
        }
    } else {
        ws_polish_role<N, In, MODE>(A, coeffs, n, map, S, ctl, ring, slots, my_tasks, abort_flag);
    }
    stats_end(S, A.stats);
}

// Uniform batch of A.n polynomials of degree N, at most MAXB = ws_max_block(N)
// threads per CTA.
template <int N, typename In, int MAXB, int MODE>
__global__ void __launch_bounds__(MAXB, 1) solve_ws_kernel(SolveArgs A, int polish_warps, int slots)
{
    ws_cta<N, In, MODE>(A, A.coeffs, A.n, UniformMap{{}, A.n}, polish_warps, slots);
}

}  // namespace rd
