// rd_common.cuh -- complex arithmetic, Givens rotations and host plumbing
// shared by the libroots kernels (sm_103a).
//
// Paper: Tang & Quan, arXiv 2507.02164. Sec. II-C defines the complex Givens
// rotation G = [[c, s], [-conj(s), conj(c)]] with G (a, b)^T = (r, 0)^T and the
// in-place update A <- (Q_{n-1}..Q_1) A (Q_1^H..Q_{n-1}^H): each left rotation
// touches two rows, each right rotation two columns.
#pragma once

#include <cstdint>
#include <type_traits>
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

// a / b, b scaled first so that |b|^2 cannot overflow. FP32: by its larger
// component (two reciprocals, each a single MUFU instruction). FP64: by the
// power of two of its larger component, read from the exponent bits (exact,
// one FP64 reciprocal instead of two; 7 % faster FP64 sweeps at degree 6).
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b)
{
    if constexpr (std::is_same<T, double>::value) {
        const unsigned er = ((unsigned)__double2hiint(b.re) >> 20) & 0x7ffu;
        const unsigned ei = ((unsigned)__double2hiint(b.im) >> 20) & 0x7ffu;
        int e = (int)max(er, ei) - 1023;
        e = e > 1000 ? 1000 : (e < -1000 ? -1000 : e);
        const double f = __longlong_as_double((long long)(1023 - e) << 52);  // 2^-e
        const cx<double> bs = scale(f, b);
        const double inv = 1.0 / norm2(bs);
        const cx<double> num = {fma(a.re, bs.re, a.im * bs.im), fma(a.im, bs.re, -a.re * bs.im)};
        return scale(inv * f, num);
    } else {
        T s = fmax(fabs(b.re), fabs(b.im));
        T inv_s = T(1) / s;
        cx<T> bs = scale(inv_s, b);
        T inv = T(1) / norm2(bs);
        cx<T> num = {fma(a.re, bs.re, a.im * bs.im), fma(a.im, bs.re, -a.re * bs.im)};
        return scale(inv * inv_s, num);
    }
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
    if constexpr (std::is_same<T, double>::value) {
        // FP64: one reciprocal square root, t = 1 / (|a| r), gives c = |a|^2 t,
        // s = t a conj(b) and top = (r^2 t) a (an FP64 rsqrt is a multi-
        // instruction sequence); a = 0 and products outside [1e-300, 1e300]
        // take the two-rsqrt form below
        const double p = na2 * r2;
        if (p >= 1e-300 && p <= 1e300) {
            const double t = rsq(p);
            c = na2 * t;
            s = scale(t, mul(a, cx<double>{b.re, -b.im}));
            top = scale(r2 * t, a);
            return;
        }
    }
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

// ---- FP32 <-> FP64 without the FP64 pipe ---------------------------------
// On GB300 the FP64 pipe runs 2 lane-ops per SM per clock and conversions
// between float and double issue to it. These helpers build the result from
// the IEEE-754 bit layouts with integer instructions instead.

// Exact float -> double (normal, subnormal, zero, inf and NaN inputs).
__device__ __forceinline__ double f2d(float f)
{
    unsigned u = __float_as_uint(f);
    unsigned sign = u & 0x80000000u;
    unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);  // exponent bias 127 -> 1023
    unsigned lo = m << 29;
    if (e == 0u) {
        // zero, or subnormal m * 2^-149: shift the leading one to bit 23
        int sh = __clz((int)m) - 8;
        unsigned mm = (m << (sh & 31)) & 0x7fffffu;
        hi = m ? (sign | ((unsigned)(897 - sh) << 20) | (mm >> 3)) : sign;
        lo = m ? (mm << 29) : 0u;
    }
    if (e == 255u) hi = sign | 0x7ff00000u | (m >> 3);  // inf / NaN (payload kept)
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float rounded to nearest (ties away from zero). Magnitudes below
// the normal FP32 range become signed zero and above it +-FLT_MAX; inf and
// NaN are kept. Used for Newton step sizes, residual magnitudes and pixel
// screening, which need a correctly scaled FP32 value, not the last bit.
__device__ __forceinline__ float d2f(double d)
{
    unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    unsigned sign = hi & 0x80000000u;
    unsigned ed = (hi >> 20) & 0x7ffu;
    int e = (int)ed - 1023 + 127;
    unsigned bits = sign | ((unsigned)(e & 0xff) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    bits += (lo >> 28) & 1u;  // round on the first dropped bit (may carry into the exponent)
    bits = e <= 0 ? sign : bits;
    bits = e >= 255 ? (sign | 0x7f7fffffu) : bits;
    if (ed == 0x7ffu) bits = sign | 0x7f800000u | ((((hi & 0xfffffu) | lo) != 0u) ? 0x400000u : 0u);
    return __uint_as_float(bits);
}

// isfinite for a double, on its exponent bits
__device__ __forceinline__ bool finite_bits(double d)
{
    return ((((unsigned)__double2hiint(d)) >> 20) & 0x7ffu) != 0x7ffu;
}

__device__ __forceinline__ cx<double> f2d(cx<float> a) { return {f2d(a.re), f2d(a.im)}; }
__device__ __forceinline__ cx<float> d2f(cx<double> a) { return {d2f(a.re), d2f(a.im)}; }

// ---- double-float arithmetic on the FP32 pipe ----------------------------
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 48 significant bits. TwoSum (Knuth) and the FMA-based exact product
// make the elementary steps error-free; every operation below uses explicit
// round-to-nearest intrinsics so that no contraction changes them.
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = two_sum(a.hi, b.hi);
    dfl t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Error-free product: a b = p + e exactly (p = fl(a b), e from one FMA).
__device__ __forceinline__ dfl two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Compensated Horner scheme (Graillat, Langlois, Louvet, "Compensated Horner
// scheme", 2005; the complex form: Graillat and Menissier-Morain, 2012) at the
// FP32 point x for coefficients a_k = hi_k + lo_k (lo only when LO). Each
// Horner step's product acc * x and sum with hi_k are split error-free into
// a float and its rounding error (four TwoProducts, four TwoSums); the errors
// run through a second Horner recurrence. On return p + err equals p(x) as
// if evaluated in twice the working precision, and d1 = p'(x), d2 = p''(x)/2
// in FP32 (plain Horner on the FP32 iterates). TwoProduct and TwoSum are
// error-free, so their outputs do not depend on how the real operations are
// grouped; the plain sums of the errors keep the scalar order per part. The
// same bits as the scalar form, about 35 instead of 50 issue slots per
// coefficient (one-role compensated polish on the degree-6 Littlewood batch
// 16 % faster).
template <int N, bool LO>
__device__ __forceinline__ void comp_horner(const cx<float> (&hi)[N + 1], const cx<float> (&lo)[LO ? N + 1 : 1],
                                            cx<float> x, cx<float> &p, cx<float> &err, cx<float> &d1,
                                            cx<float> &d2)
{
    // On (real, imaginary) pairs as packed FP32 instructions, each half the
    // scalar scheme's operation on that part (a product with -x_im is the
    // negated product exactly), in one issue slot for both:
    //   a z = (a_re x_re - a_im x_im, a_re x_im + a_im x_re)
    //       = bcast(a_re) (x_re, x_im) + bcast(a_im) (-x_im, x_re)
    const float2 X = make_float2(x.re, x.im), Xr = make_float2(-x.im, x.re);
    auto bc = [](float v) { return make_float2(v, v); };
    auto neg2 = [](float2 v) { return make_float2(-v.x, -v.y); };
    // a z + c, as cfma
    auto cfma2 = [&](float2 a, float2 c) { return __ffma2_rn(bc(a.x), X, __ffma2_rn(bc(a.y), Xr, c)); };
    float2 P = make_float2(hi[N].re, hi[N].im);
    float2 E = LO ? make_float2(lo[LO ? N : 0].re, lo[LO ? N : 0].im) : make_float2(0.0f, 0.0f);
    float2 D1 = make_float2(0.0f, 0.0f), D2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
        D2 = cfma2(D2, D1);
        D1 = cfma2(D1, P);
        // (t1, t3) = p_re (x_re, x_im), (-t2, t4) = p_im (-x_im, x_re), each with its exact error
        const float2 Ah = __fmul2_rn(bc(P.x), X), Bh = __fmul2_rn(bc(P.y), Xr);
        const float2 Al = __ffma2_rn(bc(P.x), X, neg2(Ah)), Bl = __ffma2_rn(bc(P.y), Xr, neg2(Bh));
        // two_sum(Ah, Bh), then two_sum(that, hi_k)
        const float2 S = __fadd2_rn(Ah, Bh);
        const float2 Sb = __fadd2_rn(S, neg2(Ah));
        const float2 Se = __fadd2_rn(__fadd2_rn(Ah, neg2(__fadd2_rn(S, neg2(Sb)))), __fadd2_rn(Bh, neg2(Sb)));
        const float2 H = make_float2(hi[k].re, hi[k].im);
        const float2 U = __fadd2_rn(S, H);
        const float2 Ub = __fadd2_rn(U, neg2(S));
        const float2 Ue = __fadd2_rn(__fadd2_rn(S, neg2(__fadd2_rn(U, neg2(Ub)))), __fadd2_rn(H, neg2(Ub)));
        P = U;
        float2 Er = __fadd2_rn(__fadd2_rn(__fadd2_rn(Al, Bl), Se), Ue);
        if constexpr (LO) Er = __fadd2_rn(Er, make_float2(lo[k].re, lo[k].im));
        E = cfma2(E, Er);
    }
    p = {P.x, P.y};
    err = {E.x, E.y};
    d1 = {D1.x, D1.y};
    d2 = {D2.x, D2.y};
}

// Split d * 2^-shift into hi + lo floats (|d * 2^-shift| <= 2): hi = d's
// significand rounded to 24 bits, lo = the rest rounded to 24 bits (relative
// error 2^-48). Magnitudes below the FP32 normal range become zero.
__device__ __forceinline__ dfl split_scaled(double d, int shift)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    int E = (int)((b >> 52) & 0x7ff);
    unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);  // 53-bit significand
    unsigned long long H = (M + (1ull << 28)) >> 29;                 // rounded to 24 bits (may be 2^24)
    long long r = (long long)M - (long long)(H << 29);               // |r| <= 2^28, exact remainder
    int e = E - 1023 - shift;                                         // unbiased exponent after scaling
    // hi = H * 2^(e - 23): float bits, the carry of H = 2^24 moves into the exponent
    unsigned hib = sign | (unsigned)((e + 127) << 23) + (unsigned)(H - (1ull << 23));
    float hi = (e + 127 > 0 && E != 0) ? __uint_as_float(hib) : 0.0f;
    // lo = r * 2^(e - 52)
    float lo = __int2float_rn((int)r);
    int le = e - 52 + 127;
    lo = (le > 0 && E != 0) ? lo * __uint_as_float((unsigned)le << 23) : 0.0f;
    lo = sign ? -lo : lo;
    if (E == 0x7ff) return {__int_as_float(0x7fc00000), 0.0f};  // inf or NaN sample: NaN coefficients
    return {hi, lo};
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

// Pixel index of z, or -1 when outside the window or NaN. FP64, no
// contraction: fx = (x - xmin) * sx, fy = (ymax - y) * sy, then
// ix = floor(fx), iy = floor(fy). The window test 0 <= fx < W is done on the
// floored integers (equivalent, as W is an integer; the conversion saturates
// for huge values) so that no FP64 comparison is issued; NaN is caught on
// the exponent bits.
__device__ __forceinline__ int pixel_of(const Binner &b, double x, double y)
{
    double fx = __dmul_rn(__dsub_rn(x, b.xmin), b.sx);
    double fy = __dmul_rn(__dsub_rn(b.ymax, y), b.sy);
    int ix = __double2int_rd(fx);
    int iy = __double2int_rd(fy);
    bool in = finite_bits(x) && finite_bits(y) && ix >= 0 && ix < b.W && iy >= 0 && iy < b.H;
    return in ? iy * b.W + ix : -1;
}

// Arguments of the standalone binning kernel (rd_density.cu).
struct DensityArgs {
    Binner bin;
    const uint8_t *status;  // [n_polys] or null
    int64_t n_polys;        // 0: ungrouped (no status, no clip)
    int clip_on;
    const double *centres;  // rd_c128 [n_polys]
    double radius;
    const int64_t *tile_index;  // [n_polys] or null (= polynomial index)
    Binner tiles;
};

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
// rd_stats word indices
enum : int { ST_POLYS = 0, ST_STATUS0 = 1, ST_SWEEPS = 5, ST_PAIRS = 6, ST_ROTS = 7, ST_NEWTON = 8,
             ST_BINNED = 9, ST_OOW = 10, ST_CLIPPED = 11, ST_F32 = 12, ST_F64 = 13, ST_TIMEOUT = 14,
             ST_WORDS = 15 };

// Counters are summed over the warp as soon as they are produced and kept
// per CTA in shared memory, so no thread carries them in registers through
// the solve. Every member function must be reached by all 32 lanes together.
struct CtaStats {
    unsigned long long *acc;  // ST_WORDS entries in shared memory, or null
    __device__ void add(int k, unsigned v) const
    {
        if (!acc) return;
        unsigned w = __reduce_add_sync(0xffffffffu, v);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(acc + k, (unsigned long long)w);
    }
};

// Zero the CTA's counters (all threads of the CTA call this).
__device__ inline CtaStats stats_begin(unsigned long long *smem, rd_stats *out)
{
    if (!out) return CtaStats{nullptr};
    if (threadIdx.x < ST_WORDS) smem[threadIdx.x] = 0;
    __syncthreads();
    return CtaStats{smem};
}

// Add the CTA's counters to *out, one atomic per non-zero word (all threads call this).
__device__ inline void stats_end(const CtaStats &cs, rd_stats *out)
{
    if (!out) return;
    __syncthreads();
    unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
    if (threadIdx.x < ST_WORDS && cs.acc[threadIdx.x]) atomicAdd(o + threadIdx.x, cs.acc[threadIdx.x]);
}

}  // namespace rd

// ---- host-side error reporting (rd_abi.cu) -------------------------------
int rd_set_error(int code, const char *fmt, ...);
int rd_check_launch(const char *what);
int rd_sm_count_cached();
