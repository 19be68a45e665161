// rd_solve.cuh -- batched roots of uniform-degree complex polynomials by
// single-shift QR on the companion matrix, held in registers (sm_103a).
//
// Paper: Tang & Quan, arXiv 2507.02164.
//   Sec. II-B  roots of the monic P = eigenvalues of its Frobenius companion
//              matrix; Alg. 1 (QR iteration with single shift, deflation of
//              the bottom eigenvalue, the active block shrinks by one).
//   Sec. II-C  the matrix stays upper Hessenberg (Appendix A), so a sweep is
//              m-1 Givens row rotations followed by m-1 column rotations.
//   Alg. 2     the CPU/GPU restatement the sweep order follows.
//
// GPU design (one thread = one polynomial):
//   * the Hessenberg matrix h[N][N] lives in registers; every index is a
//     compile-time constant (N is a template parameter, all loops unrolled),
//     entries below the subdiagonal are never touched, so the compiler keeps
//     only the N(N+1)/2 + N-1 live entries;
//   * each lane has its own active size m; a warp runs a sweep of size
//     M = max over its lanes of m, and a lane whose m < M applies identity
//     rotations for r >= m (no divergent code paths, no dynamic register
//     indexing); the frozen part of a finished lane is not changed;
//   * deflation |h[m-1][m-2]| <= tol (|h[m-1][m-1]| + |h[m-2][m-2]|) with
//     1-norms of (re, im), at most max_iters sweeps per eigenvalue;
//   * RD_MIXED: sweeps in FP32, then FP64 Newton polish of every root on the
//     original coefficients (FP64 p(z), FP32 p'(z)), an FP64 residual check
//     |p(z)| <= residual_tol sum |a_k||z|^k, up to polish_extra more Newton
//     steps in full FP64 for a root that fails it, and a root-separation
//     check; float <-> double conversions use integer bit operations (on
//     GB300 the conversion instructions take the FP64 pipe, the bottleneck);
//   * optional fused binning with warp-aggregated atomics.
#pragma once

#include <type_traits>

#include "rd_common.cuh"

namespace rd {

// Kernel variants: plain FP64 sweeps; FP32 sweeps with the FP64 Newton
// polish; FP32 sweeps with the double-float Newton polish.
enum : int { MODE_PLAIN = 0, MODE_MIXED_FP64 = 1, MODE_MIXED_DF = 2 };

struct SolveArgs {
    const void *coeffs;  // [N+1][n]
    int64_t n;
    double tol;
    int max_iters;
    int shift;       // rd_shift
    int exc_period;
    int polish_steps;
    int polish_extra;
    int fixed_sweeps;  // > 0: exactly this many sweeps per eigenvalue, no deflation test
    int polish_mode;   // rd_polish (selects the kernel variant at launch)
    double residual_tol;
    double collapse_tol;
    double *roots;    // [N][n] c128 or null
    uint8_t *status;  // [n] or null
    uint32_t *hist;   // or null
    Binner bin;
    // tile clip (full pipeline): clip_on => z = centre + radius * w and keep
    // only roots whose tile (nx x ny over the tile window) is the polynomial's
    int clip_on;
    const double *centres;
    double radius;
    const int64_t *tile_index;
    Binner tiles;
    rd_stats *stats;
};

template <typename In>
struct InLoad;
template <>
struct InLoad<float2> {
    __device__ static cx<double> ld(const void *p, int64_t idx)
    {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p) + idx);
        return {(double)v.x, (double)v.y};
    }
    __device__ static cx<float> ldf(const void *p, int64_t idx)
    {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p) + idx);
        return {v.x, v.y};
    }
};
template <>
struct InLoad<double2> {
    __device__ static cx<double> ld(const void *p, int64_t idx)
    {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p) + idx);
        return {v.x, v.y};
    }
    __device__ static cx<float> ldf(const void *p, int64_t idx)
    {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p) + idx);
        return {(float)v.x, (float)v.y};
    }
};

// Complex128 coefficients staged in shared memory by the kernel itself
// (plain loads: the read-only path does not serve shared memory).
struct SharedC128 {};
template <>
struct InLoad<SharedC128> {
    __device__ static cx<double> ld(const void *p, int64_t idx)
    {
        double2 v = reinterpret_cast<const double2 *>(p)[idx];
        return {v.x, v.y};
    }
    __device__ static cx<float> ldf(const void *p, int64_t idx)
    {
        double2 v = reinterpret_cast<const double2 *>(p)[idx];
        return {(float)v.x, (float)v.y};
    }
};

template <typename T>
__device__ __forceinline__ bool finite_c(cx<T> z) { return isfinite(z.re) && isfinite(z.im); }

// Multiply complex128 coefficients by the power of two that brings the
// largest exponent among them to 0 (clamped to 2^+-1000): exact, and it
// changes neither the roots, nor the Newton iterates, nor the relative
// residual test, but keeps the FP32 copies used for p'(z) and the residual
// bound finite when coefficients lie beyond the FP32 range (an L2 fit of
// sin(z^3) reaches 1e41). The exponents are read from the bits (integer ops).
template <int K>
__device__ __forceinline__ void scale_pow2(cx<double> (&a)[K])
{
    unsigned emax = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const unsigned er = ((unsigned)__double2hiint(a[k].re) >> 20) & 0x7ffu;
        const unsigned ei = ((unsigned)__double2hiint(a[k].im) >> 20) & 0x7ffu;
        emax = max(emax, max(er, ei));
    }
    int sh = (int)emax - 1023;
    sh = sh > 1000 ? 1000 : (sh < -1000 ? -1000 : sh);
    const double f = __longlong_as_double((long long)(1023 - sh) << 52);  // 2^-sh
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = {a[k].re * f, a[k].im * f};
}

// Degrees from which qr_sweep leaves its unrolled loops by an early exit
// at the warp-uniform size M instead of nesting every step in `if (< M)`:
// the same operations on the same values, but a chain of forward jumps in
// place of nested blocks that each reconverge. Measured on 2^19 complex-
// Gaussian polynomials per degree (one-role, FP64 polish): degree 9 3 %,
// 10 and 11 6 %, 12 11 % faster, warp-specialised degrees 7 and 8 up to
// 16 %; at degrees 4..6 the nested form measured 0..2.5 % faster.
constexpr int SWEEP_EARLY_EXIT_MIN = 7;

// One shifted QR sweep of size M (warp-uniform, 2 <= M <= N) on h; this
// lane's rotations r >= m are the identity and its diagonal is shifted only
// for i < m.
template <int N, typename T>
__device__ __forceinline__ void qr_sweep(cx<T> (&h)[N][N], int m, int M, cx<T> shift)
{
    if constexpr (N >= SWEEP_EARLY_EXIT_MIN) {
        __builtin_assume(M >= 2 && M <= N);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i >= M) break;
            bool a = i < m;
            h[i][i].re -= a ? shift.re : T(0);
            h[i][i].im -= a ? shift.im : T(0);
        }
        T c[N];
        cx<T> s[N];
        // left rotations Q_r, r = 1..M-1: zero h[r][r-1], update rows r-1, r
#pragma unroll
        for (int r = 1; r < N; ++r) {
            if (r >= M) break;
            cx<T> top;
            givens(h[r - 1][r - 1], h[r][r - 1], c[r], s[r], top);
            bool act = r < m;
            c[r] = act ? c[r] : T(1);
            s[r] = sel(act, s[r], cx<T>{T(0), T(0)});
            h[r - 1][r - 1] = sel(act, top, h[r - 1][r - 1]);
            h[r][r - 1] = sel(act, cx<T>{T(0), T(0)}, h[r][r - 1]);
#pragma unroll
            for (int j = r; j < N; ++j) {
                if (j >= M) break;
                rot_rows(c[r], s[r], h[r - 1][j], h[r][j]);
            }
        }
        // right rotations Q_r^H: columns r-1, r over rows 0..r (the matrix is
        // upper triangular before them, Appendix A)
#pragma unroll
        for (int r = 1; r < N; ++r) {
            if (r >= M) break;
#pragma unroll
            for (int i = 0; i <= r; ++i) rot_cols(c[r], s[r], h[i][r - 1], h[i][r]);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i >= M) break;
            bool a = i < m;
            h[i][i].re += a ? shift.re : T(0);
            h[i][i].im += a ? shift.im : T(0);
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < M) {
                bool a = i < m;
                h[i][i].re -= a ? shift.re : T(0);
                h[i][i].im -= a ? shift.im : T(0);
            }
        T c[N];
        cx<T> s[N];
        // left rotations Q_r, r = 1..M-1: zero h[r][r-1], update rows r-1, r
#pragma unroll
        for (int r = 1; r < N; ++r) {
            if (r < M) {
                cx<T> top;
                givens(h[r - 1][r - 1], h[r][r - 1], c[r], s[r], top);
                bool act = r < m;
                c[r] = act ? c[r] : T(1);
                s[r] = sel(act, s[r], cx<T>{T(0), T(0)});
                h[r - 1][r - 1] = sel(act, top, h[r - 1][r - 1]);
                h[r][r - 1] = sel(act, cx<T>{T(0), T(0)}, h[r][r - 1]);
#pragma unroll
                for (int j = r; j < N; ++j)
                    if (j < M) rot_rows(c[r], s[r], h[r - 1][j], h[r][j]);
            }
        }
        // right rotations Q_r^H: columns r-1, r over rows 0..r
#pragma unroll
        for (int r = 1; r < N; ++r) {
            if (r < M) {
#pragma unroll
                for (int i = 0; i <= r; ++i) rot_cols(c[r], s[r], h[i][r - 1], h[i][r]);
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < M) {
                bool a = i < m;
                h[i][i].re += a ? shift.re : T(0);
                h[i][i].im += a ? shift.im : T(0);
            }
    }
}

// Trailing 2x2 of the active block [[a, b], [c, d]] for this lane's m.
template <int N, typename T>
__device__ __forceinline__ void trailing(const cx<T> (&h)[N][N], int m, cx<T> &a, cx<T> &b,
                                         cx<T> &c, cx<T> &d)
{
    a = h[0][0];
    b = h[0][1 < N ? 1 : 0];
    c = h[1 < N ? 1 : 0][0];
    d = h[1 < N ? 1 : 0][1 < N ? 1 : 0];
#pragma unroll
    for (int k = 2; k < N; ++k)
        if (m == k + 1) {
            a = h[k - 1][k - 1];
            b = h[k - 1][k];
            c = h[k][k - 1];
            d = h[k][k];
        }
}

// Eigenvalue of [[a, b], [c, d]] nearer d: with t = (a - d)/2 and
// disc = sqrt(t^2 + bc), the two are d + t +- disc; the nearer one is
// d - bc / (t + disc') with disc' the sign of disc that makes |t + disc'|
// largest (no cancellation).
template <typename T>
__device__ __forceinline__ cx<T> wilkinson(cx<T> a, cx<T> b, cx<T> c, cx<T> d)
{
    cx<T> t = scale(T(0.5), sub(a, d));
    cx<T> bc = mul(b, c);
    cx<T> disc = csqrt(cfma(t, t, bc));
    T dir = fma(t.re, disc.re, t.im * disc.im);  // Re(conj(t) disc)
    cx<T> den = dir >= T(0) ? add(t, disc) : sub(t, disc);
    if (den.re == T(0) && den.im == T(0)) return d;
    return sub(d, cdiv(bc, den));
}

// Deflation test of the trailing 2x2 [[a, b], [c, d]] of the active block.
// Adaptive: the bottom subdiagonal c is negligible against the diagonal;
// fixed schedule (Alg. 2): this eigenvalue has had its T sweeps.
template <typename T>
__device__ __forceinline__ bool deflates(const SolveArgs &A, T tol, int its, cx<T> a, cx<T> c, cx<T> d)
{
    return A.fixed_sweeps > 0 ? (its >= A.fixed_sweeps) : (abs1(c) <= tol * (abs1(a) + abs1(d)));
}

// The shift of the next sweep: Wilkinson's, or the paper's h[m-1][m-1] with
// Wilkinson's every exc_period sweeps without deflation.
template <typename T>
__device__ __forceinline__ cx<T> pick_shift(const SolveArgs &A, int its, cx<T> a, cx<T> b, cx<T> c, cx<T> d)
{
    const bool wilk = (A.shift == RD_SHIFT_WILKINSON) || (A.exc_period > 0 && its > 0 && (its % A.exc_period) == 0);
    return wilk ? wilkinson(a, b, c, d) : d;
}

// Where the results of local polynomial i of a solved batch go, and (for
// the tile clip) the centre and tile of polynomial p, read from the caller's
// arrays (A.centres, A.tile_index; no tile_index: tile p).
struct ClipFromArrays {
    __device__ static cx<double> centre(const SolveArgs &A, int64_t p)
    {
        double2 c = __ldg(reinterpret_cast<const double2 *>(A.centres) + p);
        return {c.x, c.y};
    }
    __device__ static int64_t tile(const SolveArgs &A, int64_t p) { return A.tile_index ? __ldg(A.tile_index + p) : p; }
};
// Uniform batch: polynomial i itself, root j at j*n + i (coefficient-major).
struct UniformMap : ClipFromArrays {
    int64_t n;
    __device__ int64_t poly(int64_t i) const { return i; }
    __device__ int64_t root(int64_t p, int j) const { return (int64_t)j * n + p; }
};
// Degree bin of a packed uneven batch: local slot i is polynomial perm[i];
// its roots are packed like its coefficients without the leading one.
struct PackedMap : ClipFromArrays {
    const uint32_t *perm;
    const int64_t *offsets;
    __device__ int64_t poly(int64_t i) const { return (int64_t)__ldg(perm + i); }
    __device__ int64_t root(int64_t p, int j) const { return __ldg(offsets + p) - p + j; }
};

// Load a_0..a_N of local polynomial i (< n: valid) of a coefficient-major
// batch of n polynomials of degree N (coalesced across a warp) and normalise
// it to the monic b_0..b_{N-1} in the sweep precision T. Returns true when
// the polynomial is degenerate (not valid, a coefficient not finite, or
// a_N = 0); b is then zero or not meaningful.
template <int N, typename T, typename In, int MODE>
__device__ __forceinline__ bool load_monic(const void *coeffs, int64_t n, int64_t i, cx<T> (&b)[N])
{
    constexpr bool MIXED = MODE != MODE_PLAIN;
    const bool valid = i < n;
    bool degenerate = !valid;
    if (valid) {
        if constexpr (MIXED && std::is_same<In, float2>::value) {
            // complex64 storage: FP32 normalisation is exact enough for the sweeps
            cx<float> a[N + 1];
#pragma unroll
            for (int k = 0; k <= N; ++k) a[k] = InLoad<In>::ldf(coeffs, (int64_t)k * n + i);
#pragma unroll
            for (int k = 0; k <= N; ++k) degenerate |= !finite_c(a[k]);
            degenerate |= (a[N].re == 0.0f && a[N].im == 0.0f);
            cx<float> inv = cdiv(cx<float>{1.0f, 0.0f}, degenerate ? cx<float>{1.0f, 0.0f} : a[N]);
#pragma unroll
            for (int k = 0; k < N; ++k) b[k] = mul(a[k], inv);
        } else {
            // FP64 coefficients: test and normalise in FP64 (a coefficient outside
            // the FP32 range is still a valid input), then round for FP32 sweeps
            cx<double> a[N + 1];
#pragma unroll
            for (int k = 0; k <= N; ++k) a[k] = InLoad<In>::ld(coeffs, (int64_t)k * n + i);
#pragma unroll
            for (int k = 0; k <= N; ++k) degenerate |= !finite_c(a[k]);
            degenerate |= (a[N].re == 0.0 && a[N].im == 0.0);
            cx<double> inv = cdiv(cx<double>{1.0, 0.0}, degenerate ? cx<double>{1.0, 0.0} : a[N]);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                cx<double> q = mul(a[k], inv);
                b[k] = {(T)q.re, (T)q.im};
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) b[k] = {T(0), T(0)};
    }
    return degenerate;
}

// Sweep half of one lane's solve: local polynomial i (< n: valid) of a
// coefficient-major batch `coeffs` of n polynomials of degree N is loaded,
// normalised and swept to the diagonal d (its eigenvalues in the sweep
// precision T). All 32 lanes of the warp must call it together (the sweep
// size is warp-uniform).
template <int N, typename T, typename In, int MODE>
__device__ __forceinline__ void sweep_lane(const SolveArgs &A, const void *coeffs, int64_t n, int64_t i,
                                           const CtaStats &S, cx<T> (&d)[N], bool &degenerate_out,
                                           bool &not_conv_out)
{
    constexpr bool MIXED = MODE != MODE_PLAIN;
    const T tol = (T)A.tol;
    {
        cx<T> b[N];
        const bool degenerate = load_monic<N, T, In, MODE>(coeffs, n, i, b);

        // ---- Frobenius companion matrix: subdiagonal ones, last column -b
        cx<T> h[N][N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int j = 0; j < N; ++j) h[r][j] = {T(0), T(0)};
#pragma unroll
        for (int r = 0; r + 1 < N; ++r) h[r + 1][r] = {T(1), T(0)};
#pragma unroll
        for (int r = 0; r < N; ++r) h[r][N - 1] = degenerate ? cx<T>{T(0), T(0)} : cx<T>{-b[r].re, -b[r].im};

        // ---- QR iteration with deflation (Alg. 1)
        int m = degenerate ? 0 : N;
        int its = 0;
        bool not_conv = false;
        unsigned n_sweeps = 0, n_pairs = 0, n_rots = 0;
        for (;;) {
            // deflate while the bottom subdiagonal is negligible (at most once per pass)
            if (m >= 2) {
                cx<T> ta, tb, tc, td;
                trailing<N, T>(h, m, ta, tb, tc, td);
                bool small = deflates(A, tol, its, ta, tc, td);
                if (small || its >= A.max_iters) {
                    not_conv |= !small;
                    m -= 1;
                    its = 0;
                }
            }
            int mm = m >= 2 ? m : 0;
            int M = __reduce_max_sync(0xffffffffu, mm);
            if (M < 2) break;
            cx<T> ta, tb, tc, td;
            trailing<N, T>(h, mm >= 2 ? mm : 2, ta, tb, tc, td);
            cx<T> shift = pick_shift(A, its, ta, tb, tc, td);
            qr_sweep<N, T>(h, mm, M, shift);
            if (mm >= 2) {
                its += 1;
                n_sweeps += 1;
                n_pairs += (unsigned)(mm * (mm + 1) - 2);
                n_rots += (unsigned)(mm - 1);
            }
        }
        S.add(ST_SWEEPS, n_sweeps);
        S.add(ST_PAIRS, n_pairs);
        S.add(ST_ROTS, n_rots);
        // algorithmic flops of the sweeps, in the sweep precision (rd_stats convention)
        const unsigned sweep_flops = 20u * n_pairs + 24u * n_rots + 60u * n_sweeps;
        S.add(MIXED ? ST_F32 : ST_F64, sweep_flops);
#pragma unroll
        for (int j = 0; j < N; ++j) d[j] = h[j][j];
        degenerate_out = degenerate;
        not_conv_out = not_conv;
    }
}

// Finish half: polish (RD_MIXED) and check the eigenvalues d of local
// polynomial i, write its status and roots, and bin them. All 32 lanes of
// the warp must call it together (warp votes decide the rare paths).
template <int N, typename T, typename In, int MODE, class Map>
__device__ __forceinline__ void finish_lane(const SolveArgs &A, const void *coeffs, int64_t n, int64_t i,
                                            const Map &map, const CtaStats &S, const cx<T> (&d)[N],
                                            bool degenerate, bool not_conv)
{
    constexpr bool MIXED = MODE != MODE_PLAIN;
    {
        const bool valid = i < n;
        const int64_t pid = valid ? map.poly(i) : 0;  // the polynomial's index in the caller's batch

        // ---- roots: the diagonal; MIXED polishes them in FP64
        uint8_t st = degenerate ? RD_STATUS_DEGENERATE : (not_conv ? RD_STATUS_NOT_CONVERGED : RD_STATUS_OK);
        // Loops over the roots below run with a runtime counter (one copy of
        // their body in the instruction stream) and rotate the root arrays by
        // one register per iteration, so every register index stays static.
        cx<double> z[N];
        if constexpr (!MIXED) {
#pragma unroll
            for (int j = 0; j < N; ++j) z[j] = {(double)d[j].re, (double)d[j].im};
        } else {
            cx<float> zq[N];
#pragma unroll
            for (int j = 0; j < N; ++j) zq[j] = {d[j].re, d[j].im};
            unsigned newton = 0;
            const bool polish = A.polish_steps > 0 || A.polish_extra > 0;
            if (!polish) {
                // FP32 eigenvalues as they are (the paper's precision), no check
#pragma unroll
                for (int j = 0; j < N; ++j) z[j] = f2d(zq[j]);
            } else if (!__all_sync(0xffffffffu, degenerate)) {
                // the original coefficients again (an L1/L2 hit: this warp read them
                // at the start of the sweep), exactly in FP64 and rounded to FP32
                cx<double> ad[N + 1];
                cx<float> af[N + 1];
                if (!degenerate) {
#pragma unroll
                    for (int k = 0; k <= N; ++k) {
                        if constexpr (std::is_same<In, float2>::value) {
                            af[k] = InLoad<In>::ldf(coeffs, (int64_t)k * n + i);
                            ad[k] = f2d(af[k]);
                        } else {
                            ad[k] = InLoad<In>::ld(coeffs, (int64_t)k * n + i);
                        }
                    }
                    if constexpr (!std::is_same<In, float2>::value) {
                        scale_pow2(ad);
#pragma unroll
                        for (int k = 0; k <= N; ++k) af[k] = d2f(ad[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k <= N; ++k) {
                        ad[k] = {0.0, 0.0};
                        af[k] = {0.0f, 0.0f};
                    }
                    ad[N] = {1.0, 0.0};
                    af[N] = {1.0f, 0.0f};
                }
                // residual_tol <= 0: the default 64 d 2^-53 for this degree
                // MODE_MIXED_DF with complex128 input: the FP32 rounding of each
                // coefficient's remainder (a_k = af_k + alo_k to about 2^-48);
                // complex64 coefficients are exact in FP32 and have none
                constexpr bool LO = MODE == MODE_MIXED_DF && !std::is_same<In, float2>::value;
                cx<float> alo[LO ? N + 1 : 1];
                if constexpr (LO) {
#pragma unroll
                    for (int k = 0; k <= N; ++k)
                        alo[k] = {d2f(ad[k].re - f2d(af[k].re)), d2f(ad[k].im - f2d(af[k].im))};
                }
                const float rtol = A.residual_tol > 0 ? (float)A.residual_tol : (float)(64.0 * N * 0x1p-53);
                // residual test |p(z)| <= residual_tol * sum_k |a_k|_1 |z|^k (1-norms
                // |re| + |im| of the coefficients, at most sqrt(2) above the moduli)
                auto passes = [&](cx<double> p, cx<double> zj) {
                    float az = sqrtf(norm2(d2f(zj)));
                    float den = abs1(af[N]);
#pragma unroll
                    for (int k = N - 1; k >= 0; --k) den = fmaf(den, az, abs1(af[k]));
                    return (sqrtf(norm2(d2f(p))) <= rtol * den) && finite_bits(zj.re) && finite_bits(zj.im);
                };
                unsigned failed = 0;  // bit j: root j failed the residual test
#pragma unroll 1
                for (int j = 0; j < N; ++j) {
                    cx<float> zf = zq[0];
#pragma unroll
                    for (int k = 0; k + 1 < N; ++k) zq[k] = zq[k + 1];
                    cx<double> zj;
                    if constexpr (MODE == MODE_MIXED_DF) {
                        // Newton steps on the FP32 pipe: z kept as a pair zh + zl of
                        // floats; p(z) = p(zh) + p'(zh) zl + p''(zh)/2 zl^2 (the next
                        // term is below 2^-72), p(zh) by the compensated Horner scheme
                        // (twice the working precision), the derivative terms and
                        // the step size in FP32
                        cx<float> zl = {0.0f, 0.0f};
                        for (int step = 0; step < A.polish_steps; ++step) {
                            cx<float> p, err, d1, d2;
                            comp_horner<N, LO>(af, alo, zf, p, err, d1, d2);
                            const cx<float> corr = mul(cfma(d2, zl, d1), zl);
                            const cx<float> r = {__fadd_rn(p.re, __fadd_rn(err.re, corr.re)),
                                                 __fadd_rn(p.im, __fadd_rn(err.im, corr.im))};
                            const cx<float> dz = cdiv(r, d1);
                            if (!finite_c(dz)) break;
                            // z <- z - dz: TwoSum on the high parts, then renormalise
                            const dfl sr = two_sum(zf.re, -dz.re), si = two_sum(zf.im, -dz.im);
                            const dfl nr = fast_two_sum(sr.hi, __fadd_rn(sr.lo, zl.re));
                            const dfl ni = fast_two_sum(si.hi, __fadd_rn(si.lo, zl.im));
                            zf = {nr.hi, ni.hi};
                            zl = {nr.lo, ni.lo};
                            newton += 1;
                        }
                        // zh + zl rounded once to FP64
                        zj = {f2d(zf.re) + f2d(zl.re), f2d(zf.im) + f2d(zl.im)};
                    } else {
                        zj = f2d(zf);
                        // Newton steps: p(z) by FP64 Horner on the original coefficients,
                        // p'(z) and the step size in FP32 (they only scale the correction)
                        for (int step = 0; step < A.polish_steps; ++step) {
                            cx<double> p = ad[N];
#pragma unroll
                            for (int k = N - 1; k >= 0; --k) p = cfma(p, zj, ad[k]);
                            cx<float> pf = af[N], dp = {0.0f, 0.0f};
#pragma unroll
                            for (int k = N - 1; k >= 0; --k) {
                                dp = cfma(dp, zf, pf);
                                pf = cfma(pf, zf, af[k]);
                            }
                            cx<float> dz = cdiv(d2f(p), dp);
                            if (!finite_c(dz)) break;
                            zj = sub(zj, f2d(dz));
                            zf = sub(zf, dz);
                            newton += 1;
                        }
                    }
                    // final FP64 residual
                    cx<double> p = ad[N];
#pragma unroll
                    for (int k = N - 1; k >= 0; --k) p = cfma(p, zj, ad[k]);
                    failed |= (passes(p, zj) ? 0u : 1u) << j;
#pragma unroll
                    for (int k = 0; k + 1 < N; ++k) z[k] = z[k + 1];
                    z[N - 1] = zj;
                }
                if (degenerate) failed = 0;
                // Roots that failed (slow convergence near a close pair, where the
                // FP32 derivative is poor) get up to polish_extra further Newton
                // steps with p and p' both by FP64 Horner. A few roots in a
                // thousand need it, so the warp usually skips this block.
                if (A.polish_extra > 0 && __any_sync(0xffffffffu, failed != 0)) {
#pragma unroll 1
                    for (int j = 0; j < N; ++j) {
                        cx<double> zj = z[0];
#pragma unroll
                        for (int k = 0; k + 1 < N; ++k) z[k] = z[k + 1];
                        for (int it = 0; ((failed >> j) & 1u) && it < A.polish_extra; ++it) {
                            cx<double> p = ad[N], dp = {0.0, 0.0};
#pragma unroll
                            for (int k = N - 1; k >= 0; --k) {
                                dp = cfma(dp, zj, p);
                                p = cfma(p, zj, ad[k]);
                            }
                            cx<double> dz = cdiv(p, dp);
                            if (!(finite_bits(dz.re) && finite_bits(dz.im))) break;
                            zj = sub(zj, dz);
                            newton += 1;
                            cx<double> q = ad[N];
#pragma unroll
                            for (int k = N - 1; k >= 0; --k) q = cfma(q, zj, ad[k]);
                            if (passes(q, zj)) failed &= ~(1u << j);
                        }
                        z[N - 1] = zj;
                    }
                }
                bool reject = failed != 0;
                // separation: two polished roots must not have collapsed onto one.
                // A cheap FP32 screen first (FP32 copies are within ~1e-7 of the
                // FP64 roots); the FP64 test runs only when a lane needs it. The
                // screen's bound, max(1e-4, 2 collapse_tol), passes every pair the
                // FP64 test can reject, the FP32 rounding of both roots included.
                {
                    cx<float> zs[N];
#pragma unroll
                    for (int j = 0; j < N; ++j) zs[j] = d2f(z[j]);
                    const float screen = fmaxf(1e-4f, 2.0f * (float)A.collapse_tol);
                    bool near = false;
#pragma unroll
                    for (int j = 0; j < N; ++j)
#pragma unroll
                        for (int k = j + 1; k < N; ++k)
                            near |= abs1(sub(zs[j], zs[k])) <= screen * fmaxf(1.0f, abs1(zs[j]));
                    if (__any_sync(0xffffffffu, near) && near) {
#pragma unroll
                        for (int j = 0; j < N; ++j)
#pragma unroll
                            for (int k = j + 1; k < N; ++k) {
                                cx<double> d = sub(z[j], z[k]);
                                double lim = A.collapse_tol * fmax(1.0, fabs(z[j].re) + fabs(z[j].im));
                                reject |= (fabs(d.re) + fabs(d.im)) <= lim;
                            }
                    }
                }
                if (reject && st == RD_STATUS_OK && !degenerate) st = RD_STATUS_REJECTED;
            }
            S.add(ST_NEWTON, degenerate ? 0u : newton);
            const unsigned nw = degenerate ? 0u : newton, nr = (degenerate || !polish) ? 0u : (unsigned)N;
            if constexpr (MODE == MODE_MIXED_DF) {
                // compensated Horner per coefficient: 4 TwoProducts (3 flops each),
                // 4 TwoSums (6), 3 error sums, the error recurrence (8) and the
                // derivative recurrences (16) = 66 FP32 flops; per step 50 more
                // (Taylor correction, step size, double-float update). FP64 only for
                // the zh + zl assembly, the final residual and the binning
                S.add(ST_F64, (8u * N + 6u) * nr);
                S.add(ST_F32, (66u * N + 50u) * nw + (2u * N + 4u) * nr);
            } else {
                S.add(ST_F64, (8u * N + 2u) * nw + (8u * N + 4u) * nr);
                S.add(ST_F32, (8u * N + 3u) * nw + (2u * N + 4u) * nr);
            }
        }
        if (degenerate) {
#pragma unroll
            for (int j = 0; j < N; ++j) z[j] = {__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll)};
        }

        if constexpr (!MIXED) S.add(ST_F64, degenerate ? 0u : 4u * N);
        S.add(ST_POLYS, valid ? 1u : 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k) S.add(ST_STATUS0 + k, (valid && st == k) ? 1u : 0u);
        if (valid && A.status) A.status[pid] = st;

        // ---- store and bin the roots (runtime loop, rotating z)
        cx<double> cen = {0.0, 0.0};
        int64_t my_tile = pid;
        if (A.hist && A.clip_on && valid) {
            cen = map.centre(A, pid);
            my_tile = map.tile(A, pid);
        }
        unsigned n_clipped = 0, n_binned = 0, n_oow = 0;
        double2 *R = reinterpret_cast<double2 *>(A.roots);
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
            cx<double> zj = z[0];
#pragma unroll
            for (int k = 0; k + 1 < N; ++k) z[k] = z[k + 1];
            if (R && valid) R[map.root(pid, j)] = make_double2(zj.re, zj.im);
            if (A.hist) {
                double x = zj.re, y = zj.im;
                bool keep = valid;
                if (A.clip_on) {
                    x = __dadd_rn(__dmul_rn(A.radius, x), cen.re);  // z = c + rho w, no contraction
                    y = __dadd_rn(__dmul_rn(A.radius, y), cen.im);
                    int t = pixel_of(A.tiles, x, y);
                    bool in_tile = (t >= 0) && ((int64_t)t == my_tile);
                    n_clipped += (valid && !in_tile) ? 1u : 0u;
                    keep = keep && in_tile;
                }
                int pix = keep ? pixel_of(A.bin, x, y) : -1;
                n_binned += (pix >= 0) ? 1u : 0u;
                n_oow += (keep && pix < 0) ? 1u : 0u;
                hist_add(A.hist, pix);
            }
        }
        if (A.hist) {
            S.add(ST_CLIPPED, n_clipped);
            S.add(ST_BINNED, n_binned);
            S.add(ST_OOW, n_oow);
        }
    }
}

// One warp solves (and bins) the 32 polynomials base .. base+31 of a
// coefficient-major batch `coeffs` of n polynomials of degree N. All 32
// lanes must call it together.
template <int N, typename T, typename In, int MODE, class Map>
__device__ __forceinline__ void solve_warp(const SolveArgs &A, const void *coeffs, int64_t n, int64_t base,
                                           const Map &map, const CtaStats &S)
{
    const int64_t i = base + (threadIdx.x & 31);
    cx<T> d[N];
    bool degenerate, not_conv;
    sweep_lane<N, T, In, MODE>(A, coeffs, n, i, S, d, degenerate, not_conv);
    finish_lane<N, T, In, MODE>(A, coeffs, n, i, map, S, d, degenerate, not_conv);
}

// Uniform batch: warps stride over A.n polynomials, 32 at a time.
template <int N, typename T, typename In, int MODE>
__global__ void __launch_bounds__(256, (MODE != MODE_PLAIN && N <= 6) ? 2 : 1) solve_kernel(SolveArgs A)
{
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, A.stats);
    const UniformMap map{{}, A.n};
    for (int64_t base = warp_id * 32; base < A.n; base += warps_total * 32)
        solve_warp<N, T, In, MODE>(A, A.coeffs, A.n, base, map, S);
    stats_end(S, A.stats);
}

}  // namespace rd
