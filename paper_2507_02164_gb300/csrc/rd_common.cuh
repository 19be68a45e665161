// rd_common.cuh -- complex arithmetic, Givens rotations and host plumbing
// shared by the libroots kernels (sm_103a).
//
// Paper: Tang & Quan, arXiv 2507.02164. Sec. II-C defines the complex Givens
// rotation G = [[c, s], [-conj(s), conj(c)]] with G (a, b)^T = (r, 0)^T and the
// in-place update A <- (Q_{n-1}..Q_1) A (Q_1^H..Q_{n-1}^H): each left rotation
// touches two rows, each right rotation two columns.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rootdensity.h"

namespace rd {

template <typename T>
struct cx {
    T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T re, T im) { return cx<T>{re, im}; }

template <typename T>
__device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }

template <typename T>
__device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }

template <typename T>
__device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}

// a * b + c
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c)
{
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}

template <typename T>
__device__ __forceinline__ cx<T> scale(T s, cx<T> a) { return {s * a.re, s * a.im}; }

template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return fma(a.re, a.re, a.im * a.im); }

template <typename T>
__device__ __forceinline__ T abs1(cx<T> a) { return fabs(a.re) + fabs(a.im); }

template <typename T>
__device__ __forceinline__ cx<T> sel(bool p, cx<T> a, cx<T> b) { return {p ? a.re : b.re, p ? a.im : b.im}; }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// a / b
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b)
{
    // scale by the larger component of b so that |b|^2 cannot overflow
    T s = fmax(fabs(b.re), fabs(b.im));
    T inv_s = T(1) / s;
    cx<T> bs = scale(inv_s, b);
    T inv = T(1) / norm2(bs);
    cx<T> num = {fma(a.re, bs.re, a.im * bs.im), fma(a.im, bs.re, -a.re * bs.im)};
    return scale(inv * inv_s, num);
}

// principal square root
template <typename T>
__device__ __forceinline__ cx<T> csqrt(cx<T> w)
{
    T m = sqrt(fma(w.re, w.re, w.im * w.im));
    T t = sqrt(T(0.5) * (m + fabs(w.re)));
    if (t == T(0)) return {T(0), T(0)};
    T u = T(0.5) * w.im / t;
    if (w.re >= T(0)) return {t, u};
    return {fabs(u), copysign(t, w.im)};
}

// Givens pair for (a, b) with a real cosine (Sec. II-C, up to a unit phase):
//   c = |a| / r,  s = (a/|a|) conj(b) / r,  r = sqrt(|a|^2 + |b|^2),
// so that [[c, s], [-conj(s), c]] (a, b)^T = ((a/|a|) r, 0)^T. `top` receives
// (a/|a|) r, the new diagonal entry. a = 0 takes phase 1; a = b = 0 gives the
// identity.
template <typename T>
__device__ __forceinline__ void givens(cx<T> a, cx<T> b, T &c, cx<T> &s, cx<T> &top)
{
    T na2 = norm2(a), nb2 = norm2(b);
    T r2 = na2 + nb2;
    T rinv = rsq(r2);
    T ainv = rsq(na2);
    bool a0 = !(na2 > T(0));
    cx<T> ph = a0 ? cx<T>{T(1), T(0)} : scale(ainv, a);
    c = a0 ? T(0) : na2 * ainv * rinv;
    cx<T> bc = {b.re, -b.im};
    s = scale(rinv, mul(ph, bc));
    top = scale(r2 * rinv, ph);
    if (!(r2 > T(0))) {
        c = T(1);
        s = {T(0), T(0)};
        top = a;
    }
}

// rows (x, y) <- (c x + s y, -conj(s) x + c y)
template <typename T>
__device__ __forceinline__ void rot_rows(T c, cx<T> s, cx<T> &x, cx<T> &y)
{
    cx<T> nx = {fma(c, x.re, fma(s.re, y.re, -s.im * y.im)), fma(c, x.im, fma(s.re, y.im, s.im * y.re))};
    cx<T> ny = {fma(c, y.re, fma(-s.re, x.re, -s.im * x.im)), fma(c, y.im, fma(-s.re, x.im, s.im * x.re))};
    x = nx;
    y = ny;
}

// columns (x, y) <- (conj(c) x + conj(s) y, -s x + c y) with c real
template <typename T>
__device__ __forceinline__ void rot_cols(T c, cx<T> s, cx<T> &x, cx<T> &y)
{
    cx<T> nx = {fma(c, x.re, fma(s.re, y.re, s.im * y.im)), fma(c, x.im, fma(s.re, y.im, -s.im * y.re))};
    cx<T> ny = {fma(c, y.re, fma(-s.re, x.re, s.im * x.im)), fma(c, y.im, fma(-s.re, x.im, -s.im * x.re))};
    x = nx;
    y = ny;
}

// ---- warp helpers --------------------------------------------------------

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
    return __reduce_add_sync(0xffffffffu, v);
}

// ---- pixel binning (Sec. III, Roots to Pixels) ---------------------------

struct Binner {
    double xmin, ymax, sx, sy;  // sx = W / (xmax - xmin), sy = H / (ymax - ymin)
    int W, H;
};

// Pixel index of z, or -1 when outside the window or NaN. FP64 throughout, no
// contraction: fx = (x - xmin) * sx, fy = (ymax - y) * sy.
__device__ __forceinline__ int pixel_of(const Binner &b, double x, double y)
{
    double fx = __dmul_rn(__dsub_rn(x, b.xmin), b.sx);
    double fy = __dmul_rn(__dsub_rn(b.ymax, y), b.sy);
    bool in = (fx >= 0.0) && (fx < (double)b.W) && (fy >= 0.0) && (fy < (double)b.H);
    if (!in) return -1;
    int ix = (int)fx;  // fx >= 0, so truncation is floor
    int iy = (int)fy;
    return iy * b.W + ix;
}

// Warp-aggregated histogram increment: lanes holding the same pixel elect one
// leader that adds the group size. Lanes with pix < 0 take no part.
__device__ __forceinline__ void hist_add(uint32_t *hist, int pix)
{
    unsigned act = __ballot_sync(0xffffffffu, pix >= 0);
    if (pix >= 0) {
        unsigned peers = __match_any_sync(act, pix);
        int leader = __ffs(peers) - 1;
        if ((int)(threadIdx.x & 31) == leader) atomicAdd(hist + pix, (unsigned)__popc(peers));
    }
}

// ---- per-call counters ---------------------------------------------------

struct LaneStats {
    unsigned polys = 0, st[4] = {0, 0, 0, 0}, sweeps = 0, pairs = 0, rots = 0, newton = 0,
             binned = 0, oow = 0, clipped = 0;
};

// Sum the lane counters of the whole CTA and add them to *out (one atomic per
// counter per CTA). Every thread of the CTA must call it.
__device__ inline void flush_stats(const LaneStats &s, rd_stats *out)
{
    __shared__ unsigned long long acc[13];
    if (threadIdx.x < 13) acc[threadIdx.x] = 0;
    __syncthreads();
    unsigned v[13] = {s.polys, s.st[0], s.st[1], s.st[2], s.st[3], s.sweeps, s.pairs,
                      s.rots, s.newton, s.binned, s.oow, s.clipped, 0};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        unsigned w = warp_sum_u32(v[k]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&acc[k], (unsigned long long)w);
    }
    __syncthreads();
    if (out && threadIdx.x < 12 && acc[threadIdx.x]) {
        unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
        // rd_stats field order: polys, status[4], sweeps, pair_updates, rotations,
        // newton_steps, binned, out_of_window, clipped
        atomicAdd(o + threadIdx.x, acc[threadIdx.x]);
    }
}

}  // namespace rd

// ---- host-side error reporting (rd_abi.cu) -------------------------------
int rd_set_error(int code, const char *fmt, ...);
int rd_check_launch(const char *what);
int rd_sm_count_cached();
