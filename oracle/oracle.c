/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the batched root-density path.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it; the CUDA library shares no code with it.
 *
 * Paper: R. Tang, C. Quan, "Hardware-Accelerated Algorithm for Complex
 * Function Roots Density Graph Plotting", arXiv 2507.02164.
 *   Sec. II-A   L2 approximation on the unit disk (G a = b)
 *   Sec. II-B   roots = eigenvalues of the Frobenius companion matrix; Alg. 1
 *   Sec. II-C   complex Givens rotation; A <- (Q_{n-1}..Q_1) A (Q_1^H..Q_{n-1}^H)
 *   Sec. III    roots converted to pixel coordinates and counted
 *
 * Everything is written out plainly, in C99 complex arithmetic: a QR step is
 * the factorisation A - s I = Q R by Givens matrices followed by A <- R Q + s I,
 * every product a full dense matrix product (no use of the Hessenberg
 * structure, no blocking). Readings where the paper is silent:
 *   - Frobenius form: ones on the subdiagonal, last column -b_0..-b_{n-1}.
 *   - Givens: c = conj(a)/r, s = conj(b)/r, r = hypot(|a|,|b|); r = 0 -> (1,0).
 *   - Stopping: Alg. 1 runs a fixed number of sweeps per level; the oracle
 *     instead deflates the bottom eigenvalue once
 *       |h[m-1][m-2]| <= tol * (|h[m-1][m-1]| + |h[m-2][m-2]|)
 *     and gives up on a level after max_its sweeps (status NOT_CONVERGED,
 *     the diagonal entry is still taken as the eigenvalue).
 *   - Shift: Rayleigh s = h[m-1][m-1] as in Alg. 1; because a real Rayleigh
 *     shift never splits a complex-conjugate pair of a real matrix, every
 *     exc_period-th sweep without deflation uses the Wilkinson shift (the
 *     eigenvalue of the trailing 2x2 nearer h[m-1][m-1]; ties take "+").
 *   - Inner product of Sec. II-A: area measure dA on the unit disk.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx ld(const double *p) { return CMPLX(p[0], p[1]); }
static void st(double *p, cplx z) { p[0] = creal(z); p[1] = cimag(z); }

/* ---------------------------------------------------------------- Sec. II-C */

/* Givens pair: [[c, s], [-conj(s), conj(c)]] (a, b)^T = (r, 0)^T. */
static void givens(cplx a, cplx b, cplx *c, cplx *s)
{
    double r = hypot(cabs(a), cabs(b));
    if (r == 0.0) {
        *c = 1.0;
        *s = 0.0;
        return;
    }
    *c = conj(a) / r;
    *s = conj(b) / r;
}

void or_givens(const double *a, const double *b, double *c, double *s)
{
    cplx cc, ss;
    givens(ld(a), ld(b), &cc, &ss);
    st(c, cc);
    st(s, ss);
}

/* ---------------------------------------------------------------- Sec. II-B */

/* A is n x n row-major; A[i][j] at A[i*n + j]. */
#define AT(A, n, i, j) ((A)[(size_t)(i) * (n) + (j)])

static void companion(const cplx *b, int n, cplx *A)
{
    for (int i = 0; i < n * n; ++i) A[i] = 0.0;
    for (int i = 0; i + 1 < n; ++i) AT(A, n, i + 1, i) = 1.0;
    for (int i = 0; i < n; ++i) AT(A, n, i, n - 1) = -b[i];
}

void or_companion(const double *b, int n, double *A)
{
    cplx bb[OR_MAX_DEGREE], AA[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int i = 0; i < n; ++i) bb[i] = ld(b + 2 * i);
    companion(bb, n, AA);
    for (int i = 0; i < n * n; ++i) st(A + 2 * i, AA[i]);
}

/* Small dense m x m matrices (row-major, m <= OR_MAX_DEGREE) for writing one
 * QR step as the matrix products it is. */
static void mat_identity(int m, cplx *X)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) X[i * m + j] = (i == j) ? 1.0 : 0.0;
}

/* Z = X Y (Z must not alias X or Y) */
static void mat_mul(int m, const cplx *X, const cplx *Y, cplx *Z)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < m; ++k) acc += X[i * m + k] * Y[k * m + j];
            Z[i * m + j] = acc;
        }
}

/* Y = X^H */
static void mat_adjoint(int m, const cplx *X, cplx *Y)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Y[j * m + i] = conj(X[i * m + j]);
}

/* Q_r of Sec. II-C embedded in the m x m identity: the 2 x 2 rotation
 * [[c, s], [-conj(s), conj(c)]] acting on coordinates r-1 and r. */
static void givens_matrix(int m, int r, cplx c, cplx s, cplx *G)
{
    mat_identity(m, G);
    G[(r - 1) * m + (r - 1)] = c;
    G[(r - 1) * m + r] = s;
    G[r * m + (r - 1)] = -conj(s);
    G[r * m + r] = conj(c);
}

/* One shifted QR step (Alg. 1, Sec. II-B/II-C) on the leading m x m block of
 * the n x n matrix A, written as the factorisation it is:
 *   B = A - s I;  Q_1 .. Q_{m-1}, each chosen (Sec. II-C) to zero entry
 *   (r, r-1) of Q_{r-1} .. Q_1 B, give R = Q_{m-1} .. Q_1 B (upper triangular)
 *   and Q^H = Q_{m-1} .. Q_1;  then A <- R Q + s I.
 * Every product is a full dense m x m product; nothing uses the Hessenberg
 * structure (Appendix A shows that the result stays Hessenberg; the tests
 * check it instead of assuming it). */
static void qr_sweep(cplx *A, int n, int m, cplx shift)
{
    cplx B[OR_MAX_DEGREE * OR_MAX_DEGREE], Qh[OR_MAX_DEGREE * OR_MAX_DEGREE];
    cplx G[OR_MAX_DEGREE * OR_MAX_DEGREE], T[OR_MAX_DEGREE * OR_MAX_DEGREE];
    cplx Q[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) B[i * m + j] = AT(A, n, i, j);
    for (int i = 0; i < m; ++i) B[i * m + i] -= shift;
    mat_identity(m, Qh);
    for (int r = 1; r < m; ++r) {
        cplx c, s;
        givens(B[(r - 1) * m + (r - 1)], B[r * m + (r - 1)], &c, &s);
        givens_matrix(m, r, c, s, G);
        mat_mul(m, G, B, T); /* B <- Q_r B */
        memcpy(B, T, sizeof(cplx) * m * m);
        mat_mul(m, G, Qh, T); /* Q^H <- Q_r Q^H */
        memcpy(Qh, T, sizeof(cplx) * m * m);
    }
    mat_adjoint(m, Qh, Q);
    mat_mul(m, B, Q, T); /* R Q */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) AT(A, n, i, j) = T[i * m + j];
    for (int i = 0; i < m; ++i) AT(A, n, i, i) += shift;
}

void or_qr_sweep(double *A, int n, int m, const double *shift)
{
    cplx AA[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int i = 0; i < n * n; ++i) AA[i] = ld(A + 2 * i);
    qr_sweep(AA, n, m, ld(shift));
    for (int i = 0; i < n * n; ++i) st(A + 2 * i, AA[i]);
}

/* Eigenvalue of [[a, b], [c, d]] (trailing 2x2 of the active block) nearer d. */
static cplx wilkinson(const cplx *A, int n, int m)
{
    cplx a = AT(A, n, m - 2, m - 2), b = AT(A, n, m - 2, m - 1);
    cplx c = AT(A, n, m - 1, m - 2), d = AT(A, n, m - 1, m - 1);
    cplx t = 0.5 * (a - d);
    cplx disc = csqrt(t * t + b * c);
    cplx mu_plus = d + t + disc, mu_minus = d + t - disc;
    return cabs(mu_plus - d) <= cabs(mu_minus - d) ? mu_plus : mu_minus;
}

void or_wilkinson_shift(const double *A, int n, int m, double *shift)
{
    cplx AA[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int i = 0; i < n * n; ++i) AA[i] = ld(A + 2 * i);
    st(shift, wilkinson(AA, n, m));
}

static int finite_c(cplx z) { return isfinite(creal(z)) && isfinite(cimag(z)); }

/* Alg. 1 with bottom deflation: returns the status, fills eig[0..d-1]. */
static int solve_one(const cplx *a, int d, double tol, int max_its, int shift_mode,
                     int exc_period, cplx *eig, int32_t *sweeps_out)
{
    int status = OR_OK;
    int32_t sweeps = 0;
    int degenerate = (a[d] == 0.0);
    for (int k = 0; k <= d; ++k)
        if (!finite_c(a[k])) degenerate = 1;
    if (degenerate) {
        for (int j = 0; j < d; ++j) eig[j] = CMPLX(NAN, NAN);
        if (sweeps_out) *sweeps_out = 0;
        return OR_DEGENERATE;
    }

    cplx b[OR_MAX_DEGREE], A[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int k = 0; k < d; ++k) b[k] = a[k] / a[d]; /* monic: P(z) = z^d + b_{d-1} z^{d-1} + ... */
    companion(b, d, A);

    int n = d, m = d, its = 0;
    while (m >= 2) {
        double sub = cabs(AT(A, n, m - 1, m - 2));
        double diag = cabs(AT(A, n, m - 1, m - 1)) + cabs(AT(A, n, m - 2, m - 2));
        if (sub <= tol * diag || its >= max_its) {
            if (!(sub <= tol * diag)) status = OR_NOT_CONVERGED;
            eig[m - 1] = AT(A, n, m - 1, m - 1);
            m -= 1;
            its = 0;
            continue;
        }
        cplx shift;
        if (shift_mode == OR_SHIFT_WILKINSON || (its > 0 && exc_period > 0 && its % exc_period == 0))
            shift = wilkinson(A, n, m);
        else
            shift = AT(A, n, m - 1, m - 1);
        qr_sweep(A, n, m, shift);
        its += 1;
        sweeps += 1;
    }
    eig[0] = AT(A, n, 0, 0);
    if (sweeps_out) *sweeps_out = sweeps;
    return status;
}

int or_solve_one(const double *a, int d, double tol, int max_its, int shift_mode,
                 int exc_period, double *roots, int32_t *sweeps)
{
    cplx aa[OR_MAX_DEGREE + 1], eig[OR_MAX_DEGREE];
    if (d < 1 || d > OR_MAX_DEGREE) return -1;
    for (int k = 0; k <= d; ++k) aa[k] = ld(a + 2 * k);
    int status = solve_one(aa, d, tol, max_its, shift_mode, exc_period, eig, sweeps);
    for (int j = 0; j < d; ++j) st(roots + 2 * j, eig[j]);
    return status;
}

/* The paper's fixed schedule (no deflation test): Alg. 1 with its iteration
 * count T, i.e. T shifted QR steps on each active size m = d, d-1, .., 2, after
 * which the diagonal entry h[m-1][m-1] is taken as an eigenvalue and the
 * block shrinks; the last one is h[0][0]. The shift of step t on size m is
 * chosen as in solve_one with t in place of the stagnation count. */
int or_solve_fixed(const double *a_in, int d, int T, int shift_mode, int exc_period, double *roots)
{
    cplx a[OR_MAX_DEGREE + 1], eig[OR_MAX_DEGREE];
    if (d < 1 || d > OR_MAX_DEGREE || T < 1) return -1;
    for (int k = 0; k <= d; ++k) a[k] = ld(a_in + 2 * k);
    int degenerate = (a[d] == 0.0);
    for (int k = 0; k <= d; ++k)
        if (!finite_c(a[k])) degenerate = 1;
    if (degenerate) {
        for (int j = 0; j < d; ++j) st(roots + 2 * j, CMPLX(NAN, NAN));
        return OR_DEGENERATE;
    }
    cplx b[OR_MAX_DEGREE], A[OR_MAX_DEGREE * OR_MAX_DEGREE];
    for (int k = 0; k < d; ++k) b[k] = a[k] / a[d];
    companion(b, d, A);
    for (int m = d; m >= 2; --m) {
        for (int t = 0; t < T; ++t) {
            cplx shift;
            if (shift_mode == OR_SHIFT_WILKINSON || (t > 0 && exc_period > 0 && t % exc_period == 0))
                shift = wilkinson(A, d, m);
            else
                shift = AT(A, d, m - 1, m - 1);
            qr_sweep(A, d, m, shift);
        }
        eig[m - 1] = AT(A, d, m - 1, m - 1);
    }
    eig[0] = AT(A, d, 0, 0);
    for (int j = 0; j < d; ++j) st(roots + 2 * j, eig[j]);
    return OR_OK;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int pick_threads(int threads)
{
    return threads > 0 ? threads : or_max_threads();
}

int or_solve_batch(const double *coef, int64_t n, int d, double tol, int max_its,
                   int shift_mode, int exc_period, double *roots, uint8_t *status,
                   int32_t *sweeps, int threads)
{
    if (d < 1 || d > OR_MAX_DEGREE) return -1;
    int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        int32_t sw = 0;
        int stt = or_solve_one(coef + 2 * i * (d + 1), d, tol, max_its, shift_mode, exc_period,
                               roots + 2 * i * d, &sw);
        if (status) status[i] = (uint8_t)stt;
        if (sweeps) sweeps[i] = sw;
    }
    return nt;
}

/* ----------------------------------------------------------------- Sec. III */

/* Pixel of a point: column ix = floor((x - xmin) * W/(xmax - xmin)), row
 * iy = floor((ymax - y) * H/(ymax - ymin)) (row 0 at the top); half-open
 * bins, so x = xmax or y = ymin lies outside. Returns 0 outside or NaN. */
static int pixel_of(double x, double y, double xmin, double xmax, double ymin, double ymax,
                    int W, int H, int *ix, int *iy)
{
    double sx = (double)W / (xmax - xmin);
    double sy = (double)H / (ymax - ymin);
    double fx = (x - xmin) * sx;
    double fy = (ymax - y) * sy;
    if (!(fx >= 0.0 && fx < (double)W && fy >= 0.0 && fy < (double)H)) return 0;
    *ix = (int)floor(fx);
    *iy = (int)floor(fy);
    return 1;
}

void or_hist(const double *roots, int64_t n_roots, double xmin, double xmax,
             double ymin, double ymax, int W, int H, uint32_t *hist, uint64_t *oow)
{
    for (int64_t r = 0; r < n_roots; ++r) {
        int ix, iy;
        if (pixel_of(roots[2 * r], roots[2 * r + 1], xmin, xmax, ymin, ymax, W, H, &ix, &iy))
            hist[(size_t)iy * W + ix] += 1;
        else if (oow)
            *oow += 1;
    }
}

void or_hist_tiled(const double *roots, int64_t n_polys, int d, const int64_t *tile_of_poly,
                   int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                   int W, int H, uint32_t *hist, uint64_t *oow, uint64_t *dropped)
{
    for (int64_t i = 0; i < n_polys; ++i) {
        for (int j = 0; j < d; ++j) {
            double x = roots[2 * (i * d + j)], y = roots[2 * (i * d + j) + 1];
            int tx, ty, ix, iy;
            if (!pixel_of(x, y, xmin, xmax, ymin, ymax, nx, ny, &tx, &ty) ||
                (int64_t)ty * nx + tx != tile_of_poly[i]) {
                if (dropped) *dropped += 1;
                continue;
            }
            if (pixel_of(x, y, xmin, xmax, ymin, ymax, W, H, &ix, &iy))
                hist[(size_t)iy * W + ix] += 1;
            else if (oow)
                *oow += 1;
        }
    }
}

void or_affine(double *roots, int64_t n_polys, int d, const double *centres, double rho)
{
    for (int64_t i = 0; i < n_polys; ++i)
        for (int j = 0; j < d; ++j) {
            cplx w = ld(roots + 2 * (i * d + j));
            st(roots + 2 * (i * d + j), ld(centres + 2 * i) + rho * w);
        }
}

/* ---------------------------------------------------------------- Sec. II-A */

/* Legendre P_n(t) and P_n'(t) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}. */
static void legendre(int n, double t, double *p, double *dp)
{
    double p0 = 1.0, p1 = t;
    if (n == 0) {
        *p = 1.0;
        *dp = 0.0;
        return;
    }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (t * p1 - p0) / (t * t - 1.0);
}

/* Nodes: roots of P_n on (-1, 1) by Newton from cos(pi (i + 3/4)/(n + 1/2)),
 * weights 2 / ((1 - t^2) P_n'(t)^2); then mapped to [0, 1]. */
int or_gauss_legendre(int nr, double *x, double *w)
{
    if (nr < 1) return -1;
    for (int i = 0; i < nr; ++i) {
        double t = cos(M_PI * (i + 0.75) / (nr + 0.5));
        double p, dp;
        for (int it = 0; it < 100; ++it) {
            legendre(nr, t, &p, &dp);
            double dt = p / dp;
            t -= dt;
            if (fabs(dt) <= 1e-16) break;
        }
        legendre(nr, t, &p, &dp);
        double wt = 2.0 / ((1.0 - t * t) * dp * dp);
        /* t runs from near +1 down; store ascending on [0, 1] */
        x[nr - 1 - i] = 0.5 * (t + 1.0);
        w[nr - 1 - i] = 0.5 * wt;
    }
    return 0;
}

/* Solve the (k x k) complex system M a = rhs by Gaussian elimination with
 * partial pivoting; M and rhs are overwritten. */
static int gauss_solve(cplx *M, cplx *rhs, int k, cplx *a)
{
    for (int col = 0; col < k; ++col) {
        int piv = col;
        for (int r = col + 1; r < k; ++r)
            if (cabs(M[r * k + col]) > cabs(M[piv * k + col])) piv = r;
        if (M[piv * k + col] == 0.0) return -1;
        if (piv != col) {
            for (int j = 0; j < k; ++j) {
                cplx t = M[col * k + j];
                M[col * k + j] = M[piv * k + j];
                M[piv * k + j] = t;
            }
            cplx t = rhs[col];
            rhs[col] = rhs[piv];
            rhs[piv] = t;
        }
        for (int r = col + 1; r < k; ++r) {
            cplx f = M[r * k + col] / M[col * k + col];
            for (int j = col; j < k; ++j) M[r * k + j] -= f * M[col * k + j];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int r = k - 1; r >= 0; --r) {
        cplx acc = rhs[r];
        for (int j = r + 1; j < k; ++j) acc -= M[r * k + j] * a[j];
        a[r] = acc / M[r * k + r];
    }
    return 0;
}

/* <g, h> = integral over the unit disk of g conj(h) dA, by Gauss-Legendre in r
 * (with the Jacobian r) times the trapezoid rule in theta. The Gram matrix
 * G_jk = <z^j, z^k> and b_j = <g, z^j> come from the same rule; G a = b. */
int or_l2_approx(const double *samples, int64_t n, int nr, int nt, int degree,
                 double *coeffs, double *gram, int threads)
{
    int K = degree + 1;
    if (nr < 1 || nt < 1 || degree < 0 || degree > OR_MAX_DEGREE) return -1;
    double *rn = malloc(sizeof(double) * nr), *wn = malloc(sizeof(double) * nr);
    cplx *wgt = malloc(sizeof(cplx) * nr * nt);  /* quadrature weight of node (p,q) */
    cplx *pw = malloc(sizeof(cplx) * nr * nt * K); /* (r_p e^{i theta_q})^j */
    cplx *G = malloc(sizeof(cplx) * K * K);
    or_gauss_legendre(nr, rn, wn);
    for (int p = 0; p < nr; ++p)
        for (int q = 0; q < nt; ++q) {
            double th = 2.0 * M_PI * q / nt;
            cplx w = rn[p] * CMPLX(cos(th), sin(th));
            wgt[p * nt + q] = wn[p] * rn[p] * (2.0 * M_PI / nt);
            cplx acc = 1.0;
            for (int j = 0; j < K; ++j) {
                pw[(p * nt + q) * K + j] = acc;
                acc *= w;
            }
        }
    for (int j = 0; j < K; ++j)
        for (int k = 0; k < K; ++k) {
            cplx acc = 0.0;
            for (int pq = 0; pq < nr * nt; ++pq)
                acc += wgt[pq] * pw[pq * K + j] * conj(pw[pq * K + k]);
            G[j * K + k] = acc;
        }
    if (gram)
        for (int i = 0; i < K * K; ++i) st(gram + 2 * i, G[i]);

    int bad = 0;
    int ntr = pick_threads(threads);
#pragma omp parallel for schedule(static) num_threads(ntr) reduction(| : bad)
    for (int64_t s = 0; s < n; ++s) {
        cplx bvec[OR_MAX_DEGREE + 1], M[(OR_MAX_DEGREE + 1) * (OR_MAX_DEGREE + 1)], a[OR_MAX_DEGREE + 1];
        const double *g = samples + 2 * s * (int64_t)nr * nt;
        for (int j = 0; j < K; ++j) {
            cplx acc = 0.0;
            for (int pq = 0; pq < nr * nt; ++pq)
                acc += wgt[pq] * ld(g + 2 * pq) * conj(pw[pq * K + j]);
            bvec[j] = acc;
        }
        memcpy(M, G, sizeof(cplx) * K * K);
        if (gauss_solve(M, bvec, K, a) != 0) bad = 1;
        for (int j = 0; j < K; ++j) st(coeffs + 2 * (s * K + j), a[j]);
    }
    free(rn);
    free(wn);
    free(wgt);
    free(pw);
    free(G);
    return bad ? -2 : 0;
}

/* --------------------------------------- implicit differentiation of roots */

/* p'(z) = sum_{k>=1} k a_k z^{k-1} by Horner's rule. */
static cplx dpoly(const double *a, int d, cplx z)
{
    cplx dp = 0.0;
    for (int k = d; k >= 1; --k) dp = dp * z + (double)k * ld(a + 2 * k);
    return dp;
}

/* p(z) = sum_k a_k z^k vanishes at z_j, so p'(z_j) dz_j + sum_k z_j^k da_k = 0:
 * dz_j/da_k = -z_j^k / p'(z_j). For a real loss and PyTorch's gradient
 * convention (grad = dL/dRe + i dL/dIm) the pull-back through a holomorphic
 * map multiplies by the conjugate derivative. */
void or_roots_backward(const double *coef, int64_t n, int d, const double *roots,
                       const double *grad_roots, double *grad_coef, uint8_t *status)
{
    for (int64_t i = 0; i < n; ++i) {
        const double *a = coef + 2 * i * (d + 1);
        cplx g[OR_MAX_DEGREE + 1];
        int stt = OR_OK;
        for (int k = 0; k <= d; ++k) g[k] = 0.0;
        for (int j = 0; j < d; ++j) {
            cplx z = ld(roots + 2 * (i * d + j));
            cplx gz = ld(grad_roots + 2 * (i * d + j));
            cplx dp = dpoly(a, d, z);
            if (!finite_c(dp) || !finite_c(z) || cabs(dp) <= 1e-300) {
                stt = OR_SINGULAR;
                continue;
            }
            cplx zk = 1.0;
            for (int k = 0; k <= d; ++k) {
                g[k] += conj(-zk / dp) * gz;
                zk *= z;
            }
        }
        for (int k = 0; k <= d; ++k) st(grad_coef + 2 * (i * (d + 1) + k), g[k]);
        if (status) status[i] = (uint8_t)stt;
    }
}

/* ------------------------------------------------- soft root density (C4) */

/* The differentiable stand-in for the histogram used by the differentiation
 * workload (not in the paper): W x H pixel centres over the window, pixel
 * (iy, ix) at x = xmin + (ix + 1/2) px, y = ymax - (iy + 1/2) py with
 * px = (xmax - xmin)/W, py = (ymax - ymin)/H. A root at (x, y), in pixel
 * units u = (x - xmin)/px, v = (ymax - y)/py, adds
 *   w = max(0, exp(-r^2 / (2 sigma^2)) - exp(-9/2)),  r^2 = du^2 + dv^2,
 *   du = u - (ix + 1/2), dv = v - (iy + 1/2),
 * times `scale` to pixel (iy, ix); w reaches 0 at r = 3 sigma, so only the
 * pixels whose centres lie within 3 sigma in both axes are visited. A root
 * with a non-finite coordinate adds nothing. */
static int splat_box(double u, double sigma, int n_pix, int *lo, int *hi)
{
    if (!isfinite(u)) return 0;
    double a = ceil(u - 0.5 - 3.0 * sigma), b = floor(u - 0.5 + 3.0 * sigma);
    if (a < 0.0) a = 0.0;
    if (b > n_pix - 1.0) b = n_pix - 1.0;
    if (a > b) return 0;
    *lo = (int)a;
    *hi = (int)b;
    return 1;
}

void or_splat(const double *roots, int64_t n, double xmin, double xmax, double ymin, double ymax, int W, int H,
              double sigma, double scale, double *img)
{
    const double px = (xmax - xmin) / W, py = (ymax - ymin) / H;
    const double cut = exp(-4.5);
    for (int64_t j = 0; j < n; ++j) {
        const double u = (roots[2 * j] - xmin) / px;
        const double v = (ymax - roots[2 * j + 1]) / py;
        int x0, x1, y0, y1;
        if (!splat_box(u, sigma, W, &x0, &x1) || !splat_box(v, sigma, H, &y0, &y1)) continue;
        for (int iy = y0; iy <= y1; ++iy)
            for (int ix = x0; ix <= x1; ++ix) {
                const double du = u - (ix + 0.5);
                const double dv = v - (iy + 0.5);
                const double w = exp(-(du * du + dv * dv) / (2.0 * sigma * sigma)) - cut;
                if (w > 0.0) img[(size_t)iy * W + ix] += scale * w;
            }
    }
}

/* Gradient of L(img) with respect to every root: given G = dL/dimg,
 *   dL/du = scale sum_pix G dw/du,  dw/du = -(du / sigma^2) exp(-r^2/(2 sigma^2))
 * where w > 0 (0 elsewhere), likewise for v; then x = xmin + px u and
 * y = ymax - py v give grad[2j] = dL/dx = (dL/du) / px and
 * grad[2j+1] = dL/dy = -(dL/dv) / py (PyTorch's convention for a complex
 * root: dL/dRe + i dL/dIm). */
void or_splat_grad(const double *roots, int64_t n, double xmin, double xmax, double ymin, double ymax, int W,
                   int H, double sigma, double scale, const double *G, double *grad)
{
    const double px = (xmax - xmin) / W, py = (ymax - ymin) / H;
    const double cut = exp(-4.5);
    for (int64_t j = 0; j < n; ++j) {
        const double u = (roots[2 * j] - xmin) / px, v = (ymax - roots[2 * j + 1]) / py;
        double gu = 0.0, gv = 0.0;
        int x0, x1, y0, y1;
        if (splat_box(u, sigma, W, &x0, &x1) && splat_box(v, sigma, H, &y0, &y1)) {
            for (int iy = y0; iy <= y1; ++iy)
                for (int ix = x0; ix <= x1; ++ix) {
                    const double du = u - (ix + 0.5), dv = v - (iy + 0.5);
                    const double e = exp(-(du * du + dv * dv) / (2.0 * sigma * sigma));
                    if (e - cut > 0.0) {
                        const double g = G[(size_t)iy * W + ix];
                        gu += g * (-du / (sigma * sigma)) * e;
                        gv += g * (-dv / (sigma * sigma)) * e;
                    }
                }
        }
        grad[2 * j] = scale * gu / px;
        grad[2 * j + 1] = -scale * gv / py;
    }
}

void or_root_condition(const double *coef, int64_t n, int d, const double *roots, double *kappa)
{
    for (int64_t i = 0; i < n; ++i) {
        const double *a = coef + 2 * i * (d + 1);
        for (int j = 0; j < d; ++j) {
            cplx z = ld(roots + 2 * (i * d + j));
            double az = cabs(z), num = 0.0, zk = 1.0;
            for (int k = 0; k <= d; ++k) {
                num += cabs(ld(a + 2 * k)) * zk;
                zk *= az;
            }
            cplx dp = dpoly(a, d, z);
            kappa[i * d + j] = num / (fmax(1.0, az) * cabs(dp));
        }
    }
}
