// rd_solve2.cuh -- the QR solver with two lanes per polynomial, for the
// larger degrees, where one thread cannot keep the whole Hessenberg matrix
// in registers without spilling or starving the SM of warps (degree 12:
// 89 live complex entries per thread).
//
// Same method as rd_solve.cuh (Sec. II-B/II-C, Alg. 1/2): single-shift QR
// sweeps of complex Givens rotations on the companion matrix, deflation of
// the bottom eigenvalue, Newton polish in FP64 (RD_MIXED). Layout: lanes 2k
// and 2k+1 of a warp hold polynomial base + k; the lane of parity P keeps the
// columns c = 2l + P (local index l) of the matrix, rows 0 .. c+1 of each
// (the Hessenberg profile), so a lane holds about half of the entries.
//   * A left rotation on rows r-1, r touches columns >= r-1 of both lanes:
//     each lane rotates its own columns; the lane holding column r-1 computes
//     (c, s) and its partner receives them by warp shuffle.
//   * A right rotation on columns r-1, r has one column in each lane: the two
//     lanes exchange their column entries (rows 0..r) by shuffle and each
//     writes its own new column.
//   * The trailing 2x2 block (deflation test, shift) is gathered from both
//     lanes, so both make the same decisions and keep the same active size.
// Each lane polishes, stores and bins the roots on its own diagonal entries
// (root 2l + P); the pair agrees on the status.
#pragma once

#include "rd_solve.cuh"

namespace rd {

template <typename T>
__device__ __forceinline__ cx<T> shfl_pair(cx<T> v)
{
    return {__shfl_xor_sync(0xffffffffu, v.re, 1), __shfl_xor_sync(0xffffffffu, v.im, 1)};
}

template <int N>
struct TwoLane {
    static constexpr int L = (N + 1) / 2;  // local columns per lane (odd N: lane 1's last is empty)
};

template <typename T>
__device__ __forceinline__ cx<double> widen(cx<T> a)
{
    if constexpr (std::is_same<T, float>::value)
        return f2d(a);
    else
        return a;
}

// One shifted QR sweep of size M (warp-uniform) on the distributed matrix hl
// (hl[l][r] = h[r][2l + P]); rotations r >= m of this pair are the identity.
template <int N, typename T>
__device__ __forceinline__ void qr_sweep2(cx<T> (&hl)[TwoLane<N>::L][N], int m, int M, cx<T> shift, int P)
{
    const int pair_base = (threadIdx.x & 31) & ~1;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < M) {
            bool a = (i < m) && ((i & 1) == P);
            hl[i >> 1][i].re -= a ? shift.re : T(0);
            hl[i >> 1][i].im -= a ? shift.im : T(0);
        }
    T c[N];
    cx<T> s[N];
    // Left rotation Q_r (rows r-1, r; zeroes h[r][r-1]) for r = 1..M-1, each
    // followed by the right rotation Q_{r-1}^H (columns r-2, r-1, rows
    // 0..r-1): Q_{r-1}^H needs column r-1 after Q_r, and no later left
    // rotation touches columns r-2, r-1, so the result is that of all left
    // rotations before all right ones (Appendix A), with two rotations live.
#pragma unroll
    for (int r = 1; r <= N; ++r) {
        if (r < N && r < M) {
            const int O = (r - 1) & 1;  // parity of the lane holding column r-1
            const int l0 = (r - 1) >> 1;
            const bool own = P == O;
            cx<T> top;
            givens(hl[l0][r - 1], hl[l0][r], c[r], s[r], top);
            c[r] = __shfl_sync(0xffffffffu, c[r], pair_base | O);
            s[r].re = __shfl_sync(0xffffffffu, s[r].re, pair_base | O);
            s[r].im = __shfl_sync(0xffffffffu, s[r].im, pair_base | O);
            const bool act = r < m;
            c[r] = act ? c[r] : T(1);
            s[r] = sel(act, s[r], cx<T>{T(0), T(0)});
            // local column l0: column r-1 in the owner (it becomes (top, 0));
            // in the partner column r (O = 0), or column r-2 (O = 1), whose rows
            // r-1, r are zero by then
            cx<T> x = hl[l0][r - 1], y = hl[l0][r];
            cx<T> nx = x, ny = y;
            rot_rows(c[r], s[r], nx, ny);
            hl[l0][r - 1] = own ? sel(act, top, x) : nx;
            hl[l0][r] = own ? sel(act, cx<T>{T(0), T(0)}, y) : ny;
#pragma unroll
            for (int l = l0 + 1; l < TwoLane<N>::L; ++l)
                if (2 * l < M) rot_rows(c[r], s[r], hl[l][r - 1], hl[l][r]);
        }
        // right rotation q = r-1 on columns q-1, q over rows 0..q; column q-1
        // is in lane parity (q-1)&1 at local index (q-1)>>1, column q in
        // parity q&1 at q>>1
        const int q = r - 1;
        if (q >= 1 && q < M) {
            const bool left = ((q - 1) & 1) == P;
            // left column: x' = c x + conj(s) y; right column: y' = c y - s x
            const cx<T> k = left ? cx<T>{s[q].re, -s[q].im} : cx<T>{-s[q].re, -s[q].im};
#pragma unroll
            for (int i = 0; i <= q; ++i) {
                cx<T> mine;
                if (q & 1)
                    mine = hl[q >> 1][i];
                else
                    mine = P ? hl[(q >> 1) - 1][i] : hl[q >> 1][i];
                const cx<T> other = shfl_pair(mine);
                const cx<T> nv = cfma(k, other, scale(c[q], mine));
                if (q & 1) {
                    hl[q >> 1][i] = nv;
                } else {
                    hl[(q >> 1) - 1][i] = P ? nv : hl[(q >> 1) - 1][i];
                    hl[q >> 1][i] = P ? hl[q >> 1][i] : nv;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < M) {
            bool a = (i < m) && ((i & 1) == P);
            hl[i >> 1][i].re += a ? shift.re : T(0);
            hl[i >> 1][i].im += a ? shift.im : T(0);
        }
}

// Trailing 2x2 [[a, b], [c, d]] of the active block of size m >= 2; both
// lanes of the pair receive the same values. All 32 lanes must call it.
template <int N, typename T>
__device__ __forceinline__ void trailing2(const cx<T> (&hl)[TwoLane<N>::L][N], int m, int P, cx<T> &a,
                                          cx<T> &b, cx<T> &c, cx<T> &d)
{
    // this lane's column among m-2, m-1 (col = 2l + P), and its entries in
    // rows m-2, m-1: rows col, col+1 for column m-2; col-1, col for m-1
    const bool has_left = ((m - 2) & 1) == P;
    const int col = has_left ? m - 2 : m - 1;
    const int lc = col >> 1;
    const int top = col - (has_left ? 0 : 1) - 2 * lc;  // first row - 2l: -1, 0 or 1
    cx<T> v1 = {T(0), T(0)}, v2 = {T(0), T(0)};
#pragma unroll
    for (int l = 0; l < TwoLane<N>::L; ++l) {
        if (l == lc) {
            cx<T> e_m1 = l > 0 ? hl[l][2 * l - 1] : cx<T>{T(0), T(0)};
            cx<T> e0 = hl[l][2 * l];
            cx<T> e1 = 2 * l + 1 < N ? hl[l][2 * l + 1] : cx<T>{T(0), T(0)};
            cx<T> e2 = 2 * l + 2 < N ? hl[l][2 * l + 2] : cx<T>{T(0), T(0)};
            v1 = top < 0 ? e_m1 : (top == 0 ? e0 : e1);
            v2 = top < 0 ? e0 : (top == 0 ? e1 : e2);
        }
    }
    const cx<T> w1 = shfl_pair(v1), w2 = shfl_pair(v2);
    a = has_left ? v1 : w1;
    c = has_left ? v2 : w2;
    b = has_left ? w1 : v1;
    d = has_left ? w2 : v2;
}

// Lanes 2k, 2k+1 solve (and bin) polynomial base + k, k < 16, of a
// coefficient-major batch `coeffs` of n polynomials of degree N. All 32
// lanes must call it together.
template <int N, typename T, typename In, int MODE, class Map>
__device__ __forceinline__ void solve_warp2(const SolveArgs &A, const void *coeffs, int64_t n, int64_t base,
                                            const Map &map, const CtaStats &S)
{
    static_assert(MODE != MODE_MIXED_DF, "the two-lane solver polishes in FP64");
    static_assert(N >= 2, "two lanes per polynomial needs degree >= 2");
    constexpr bool MIXED = MODE != MODE_PLAIN;
    constexpr int L = TwoLane<N>::L;
    const int lane = threadIdx.x & 31;
    const int P = lane & 1;
    const T tol = (T)A.tol;
    const int64_t i = base + (lane >> 1);
    const bool valid = i < n;
    const int64_t pid = valid ? map.poly(i) : 0;
    const int nmine = (N + 1 - P) / 2;  // roots (diagonal entries) of this lane
    const int npart = (N + P) / 2;      // roots of the partner lane

    // ---- load a_0..a_N (both lanes of the pair) and normalise
    cx<T> b[N];
    bool degenerate = !valid;
    if (valid) {
        if constexpr (MIXED && std::is_same<In, float2>::value) {
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

    // ---- this lane's columns of the Frobenius companion matrix
    cx<T> hl[L][N];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int r = 0; r < N; ++r) hl[l][r] = {T(0), T(0)};
#pragma unroll
    for (int l = 0; l < L; ++l) {
        // the subdiagonal one of column 2l + P sits in row 2l + P + 1
        if (2 * l + 1 < N) hl[l][2 * l + 1] = P ? hl[l][2 * l + 1] : cx<T>{T(1), T(0)};
        if (2 * l + 2 < N) hl[l][2 * l + 2] = P ? cx<T>{T(1), T(0)} : hl[l][2 * l + 2];
        // the last column -b_0 .. -b_{N-1}
        if (2 * l == N - 1 || 2 * l + 1 == N - 1) {
            const bool last = (2 * l + P) == N - 1 && !degenerate;
#pragma unroll
            for (int r = 0; r < N; ++r) hl[l][r] = last ? cx<T>{-b[r].re, -b[r].im} : hl[l][r];
        }
    }

    // ---- QR iteration with deflation (Alg. 1); both lanes decide alike
    int m = degenerate ? 0 : N;
    int its = 0;
    bool not_conv = false;
    unsigned n_sweeps = 0, n_pairs = 0, n_rots = 0;
    for (;;) {
        {
            cx<T> ta, tb, tc, td;
            trailing2<N, T>(hl, m >= 2 ? m : 2, P, ta, tb, tc, td);
            if (m >= 2) {
                bool small = A.fixed_sweeps > 0 ? (its >= A.fixed_sweeps) : (abs1(tc) <= tol * (abs1(ta) + abs1(td)));
                if (small || its >= A.max_iters) {
                    not_conv |= !small;
                    m -= 1;
                    its = 0;
                }
            }
        }
        const int mm = m >= 2 ? m : 0;
        const int M = __reduce_max_sync(0xffffffffu, mm);
        if (M < 2) break;
        cx<T> ta, tb, tc, td;
        trailing2<N, T>(hl, mm >= 2 ? mm : 2, P, ta, tb, tc, td);
        bool wilk = (A.shift == RD_SHIFT_WILKINSON) || (A.exc_period > 0 && its > 0 && (its % A.exc_period) == 0);
        cx<T> shift = wilk ? wilkinson(ta, tb, tc, td) : td;
        qr_sweep2<N, T>(hl, mm, M, shift, P);
        if (mm >= 2) {
            its += 1;
            n_sweeps += 1;
            n_pairs += (unsigned)(mm * (mm + 1) - 2);
            n_rots += (unsigned)(mm - 1);
        }
    }
    // per polynomial once (lane P = 0 of the pair), as in the one-lane solver
    const unsigned once = P == 0 ? 1u : 0u;
    S.add(ST_SWEEPS, n_sweeps * once);
    S.add(ST_PAIRS, n_pairs * once);
    S.add(ST_ROTS, n_rots * once);
    S.add(MIXED ? ST_F32 : ST_F64, (20u * n_pairs + 24u * n_rots + 60u * n_sweeps) * once);

    // ---- this lane's roots: diagonal entries h[2l+P][2l+P]
    uint8_t st = degenerate ? RD_STATUS_DEGENERATE : (not_conv ? RD_STATUS_NOT_CONVERGED : RD_STATUS_OK);
    cx<double> z[L];
    cx<T> zq[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        zq[l] = P ? (2 * l + 1 < N ? hl[l][2 * l + 1] : cx<T>{T(0), T(0)}) : hl[l][2 * l];
        z[l] = widen(zq[l]);
    }
    bool reject = false;
    if constexpr (MIXED) {
        unsigned newton = 0;
        const bool polish = A.polish_steps > 0 || A.polish_extra > 0;
        if (polish && !__all_sync(0xffffffffu, degenerate)) {
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
                    scale_pow2(ad);  // FP32 copies finite beyond the FP32 range
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
            const float rtol = A.residual_tol > 0 ? (float)A.residual_tol : (float)(64.0 * N * 0x1p-53);
            auto passes = [&](cx<double> p, cx<double> zj) {
                float az = sqrtf(norm2(d2f(zj)));
                float den = abs1(af[N]);
#pragma unroll
                for (int k = N - 1; k >= 0; --k) den = fmaf(den, az, abs1(af[k]));
                return (sqrtf(norm2(d2f(p))) <= rtol * den) && finite_bits(zj.re) && finite_bits(zj.im);
            };
            unsigned failed = 0;  // bit j: root 2j + P failed the residual test
#pragma unroll 1
            for (int j = 0; j < L; ++j) {
                cx<float> zf = zq[0];
#pragma unroll
                for (int k = 0; k + 1 < L; ++k) zq[k] = zq[k + 1];
                cx<double> zj = z[0];
#pragma unroll
                for (int k = 0; k + 1 < L; ++k) z[k] = z[k + 1];
                if (j < nmine) {
                    // FP64 p(z) on the original coefficients, FP32 p'(z) and step
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
                    cx<double> p = ad[N];
#pragma unroll
                    for (int k = N - 1; k >= 0; --k) p = cfma(p, zj, ad[k]);
                    failed |= (passes(p, zj) ? 0u : 1u) << j;
                }
                z[L - 1] = zj;
                zq[L - 1] = zf;
            }
            if (degenerate) failed = 0;
            if (A.polish_extra > 0 && __any_sync(0xffffffffu, failed != 0)) {
#pragma unroll 1
                for (int j = 0; j < L; ++j) {
                    cx<double> zj = z[0];
#pragma unroll
                    for (int k = 0; k + 1 < L; ++k) z[k] = z[k + 1];
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
                    z[L - 1] = zj;
                }
            }
            reject = failed != 0;
            // separation, each pair of the polynomial's roots once with the lower
            // root index g = 2j + P first (the one-lane solver's test): own pairs
            // j < k, and own root j against partner root k when 2j + P < 2k + 1 - P
            {
                cx<float> zs[L], zo[L];
#pragma unroll
                for (int j = 0; j < L; ++j) zs[j] = d2f(z[j]);
#pragma unroll
                for (int j = 0; j < L; ++j) zo[j] = shfl_pair(zs[j]);
                bool near = false;
                // the screen passes every pair the FP64 test can reject (as in finish_lane)
                const float screen = fmaxf(1e-4f, 2.0f * (float)A.collapse_tol);
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const float lim = screen * fmaxf(1.0f, abs1(zs[j]));
#pragma unroll
                    for (int k = j + 1; k < L; ++k) near |= (k < nmine) && abs1(sub(zs[j], zs[k])) <= lim;
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        near |= (j < nmine) && (k < npart) && (2 * j + P < 2 * k + 1 - P) &&
                                abs1(sub(zs[j], zo[k])) <= lim;
                }
                if (__any_sync(0xffffffffu, near)) {
                    cx<double> zp[L];
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        zp[k] = {__shfl_xor_sync(0xffffffffu, z[k].re, 1), __shfl_xor_sync(0xffffffffu, z[k].im, 1)};
                    if (near) {
#pragma unroll
                        for (int j = 0; j < L; ++j) {
                            const double lim = A.collapse_tol * fmax(1.0, fabs(z[j].re) + fabs(z[j].im));
#pragma unroll
                            for (int k = j + 1; k < L; ++k) {
                                cx<double> dd = sub(z[j], z[k]);
                                reject |= (k < nmine) && (fabs(dd.re) + fabs(dd.im)) <= lim;
                            }
#pragma unroll
                            for (int k = 0; k < L; ++k) {
                                cx<double> dd = sub(z[j], zp[k]);
                                reject |= (j < nmine) && (k < npart) && (2 * j + P < 2 * k + 1 - P) &&
                                          (fabs(dd.re) + fabs(dd.im)) <= lim;
                            }
                        }
                    }
                }
            }
        }
        const unsigned nw = degenerate ? 0u : newton, nr = (degenerate || !polish) ? 0u : (unsigned)nmine;
        S.add(ST_NEWTON, nw);
        S.add(ST_F64, (8u * N + 2u) * nw + (8u * N + 4u) * nr);
        S.add(ST_F32, (8u * N + 3u) * nw + (2u * N + 4u) * nr);
    } else {
        S.add(ST_F64, degenerate ? 0u : 4u * (unsigned)nmine);
    }
    // the pair agrees on REJECTED (the shuffle runs in every lane: a
    // short-circuit here would leave lanes out of a full-mask collective)
    const int partner_reject = __shfl_xor_sync(0xffffffffu, reject ? 1 : 0, 1);
    reject = reject || partner_reject != 0;
    if (reject && st == RD_STATUS_OK && !degenerate) st = RD_STATUS_REJECTED;
    if (degenerate) {
#pragma unroll
        for (int j = 0; j < L; ++j)
            z[j] = {__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll)};
    }
    S.add(ST_POLYS, valid ? once : 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) S.add(ST_STATUS0 + k, (valid && st == k) ? once : 0u);
    if (valid && P == 0 && A.status) A.status[pid] = st;

    // ---- store and bin this lane's roots, root index 2j + P
    cx<double> cen = {0.0, 0.0};
    int64_t my_tile = pid;
    if (A.hist && A.clip_on && valid) {
        cen = map.centre(A, pid);
        my_tile = map.tile(A, pid);
    }
    unsigned n_clipped = 0, n_binned = 0, n_oow = 0;
    double2 *R = reinterpret_cast<double2 *>(A.roots);
#pragma unroll 1
    for (int j = 0; j < L; ++j) {
        cx<double> zj = z[0];
#pragma unroll
        for (int k = 0; k + 1 < L; ++k) z[k] = z[k + 1];
        const bool have = valid && j < nmine;
        if (R && have) R[map.root(pid, 2 * j + P)] = make_double2(zj.re, zj.im);
        if (A.hist) {
            double x = zj.re, y = zj.im;
            bool keep = have;
            if (A.clip_on) {
                x = __dadd_rn(__dmul_rn(A.radius, x), cen.re);  // z = c + rho w, no contraction
                y = __dadd_rn(__dmul_rn(A.radius, y), cen.im);
                int t = pixel_of(A.tiles, x, y);
                bool in_tile = (t >= 0) && ((int64_t)t == my_tile);
                n_clipped += (have && !in_tile) ? 1u : 0u;
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

// Registers per thread for the two-lane kernels. FP32 sweeps: 128 (16 warps
// per SM) holds the half matrix up to degree 8; degrees 9..12 need about 150
// live values in the sweep and get 168 (12 warps per SM) rather than spill.
// FP64 sweeps: the half matrix alone is 2 x 47 complex values at degree 12.
constexpr int two_lane_regs(int n, int mode) { return mode != MODE_PLAIN ? (n <= 8 ? 128 : 168) : 255; }

// Uniform batch, two lanes per polynomial: warps stride over A.n, 16 at a time.
template <int N, typename T, typename In, int MODE>
__global__ void __maxnreg__(two_lane_regs(N, MODE)) solve2_kernel(SolveArgs A)
{
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, A.stats);
    const UniformMap map{{}, A.n};
    for (int64_t base = warp_id * 16; base < A.n; base += warps_total * 16)
        solve_warp2<N, T, In, MODE>(A, A.coeffs, A.n, base, map, S);
    stats_end(S, A.stats);
}

// Launch of solve2_kernel for one degree (grid: enough warps for A.n / 16,
// capped at ctas_per_sm per SM, or the occupancy limit when that is 0).
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

}  // namespace rd
