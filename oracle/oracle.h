/*
 * oracle.h -- plain FP64 CPU oracle for the batched polynomial-root /
 * root-density path of "Hardware-Accelerated Algorithm for Complex Function
 * Roots Density Graph Plotting" (Tang & Quan, arXiv 2507.02164).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library. The CUDA library never includes,
 * links or calls it, and it never calls the CUDA library.
 *
 * Complex numbers cross this interface as interleaved (re, im) double pairs.
 * Coefficient arrays are poly-major: polynomial i, coefficient k (power z^k)
 * at coef[2*(i*(d+1)+k)]. Root arrays are poly-major: root j of polynomial i
 * at roots[2*(i*d+j)].
 */
#ifndef ROOTDENSITY_ORACLE_H
#define ROOTDENSITY_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_DEGREE 16

/* status codes, one per polynomial */
#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_SINGULAR 2
#define OR_DEGENERATE 3

/* shift strategies */
#define OR_SHIFT_RAYLEIGH 0  /* Rayleigh h[m-1][m-1]; Wilkinson every exc_period stagnant sweeps */
#define OR_SHIFT_WILKINSON 1 /* Wilkinson on every sweep */

/* Givens coefficients (c, s) with G (a, b)^T = (r, 0), r = sqrt(|a|^2+|b|^2). */
void or_givens(const double *a, const double *b, double *c, double *s);

/* Build the n x n Frobenius companion matrix of the monic polynomial with
 * low coefficients b_0..b_{n-1} into A (row-major n x n complex). */
void or_companion(const double *b, int n, double *A);

/* One shifted QR step on the leading m x m block of the n x n row-major
 * matrix A, with shift `shift`: B = A - s I = Q R by Givens matrices
 * (Sec. II-C), then A <- R Q + s I, as full dense matrix products. */
void or_qr_sweep(double *A, int n, int m, const double *shift);

/* Wilkinson shift of the trailing 2x2 of the leading m x m block of A. */
void or_wilkinson_shift(const double *A, int n, int m, double *shift);

/* Roots of one polynomial a_0..a_d (d >= 1). Returns the status; writes d
 * roots and, if sweeps != 0, the number of QR sweeps performed. */
int or_solve_one(const double *a, int d, double tol, int max_its, int shift_mode,
                 int exc_period, double *roots, int32_t *sweeps);

/* Batch version; poly-major arrays; OpenMP over polynomials with `threads`
 * threads (<= 0: the OpenMP default). Returns the number of threads used. */
int or_solve_batch(const double *coef, int64_t n, int d, double tol, int max_its,
                   int shift_mode, int exc_period, double *roots, uint8_t *status,
                   int32_t *sweeps, int threads);

/* The paper's fixed schedule: T QR steps on each active size d, .., 2 (Alg. 1
 * with its iteration count), no deflation test. Returns the status (OK or
 * DEGENERATE). */
int or_solve_fixed(const double *a, int d, int T, int shift_mode, int exc_period, double *roots);

/* Root-density histogram: hist[iy*W + ix] += 1 for every root inside the
 * window, *oow += 1 for every other root (NaN included). */
void or_hist(const double *roots, int64_t n_roots, double xmin, double xmax,
             double ymin, double ymax, int W, int H, uint32_t *hist, uint64_t *oow);

/* Same binning with a per-root tile test: root r (of polynomial r / d) is kept
 * only if its tile index equals that of its polynomial's tile. Tiles are
 * nx x ny over the same window; tile t = ty*nx + tx. */
void or_hist_tiled(const double *roots, int64_t n_polys, int d, const int64_t *tile_of_poly,
                   int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                   int W, int H, uint32_t *hist, uint64_t *oow, uint64_t *dropped);

/* Map roots in the local variable w to z = c + rho * w (per polynomial). */
void or_affine(double *roots, int64_t n_polys, int d, const double *centres, double rho);

/* Gauss-Legendre rule with nr nodes on [0, 1]: nodes x, weights w. */
int or_gauss_legendre(int nr, double *x, double *w);

/* Least-squares (L2) polynomial approximation on the unit disk. samples holds
 * g(r_p e^{i theta_q}) for p < nr (Gauss-Legendre radii), q < nt (theta_q =
 * 2 pi q / nt), index [s][p*nt + q]. Writes coeffs [s][degree+1]. gram, if
 * non-null, receives the (degree+1)^2 quadrature Gram matrix. */
int or_l2_approx(const double *samples, int64_t n, int nr, int nt, int degree,
                 double *coeffs, double *gram, int threads);

/* Implicit-differentiation adjoint: grad_coef[k] = sum_j conj(-z_j^k / p'(z_j)) grad_z_j. */
void or_roots_backward(const double *coef, int64_t n, int d, const double *roots,
                       const double *grad_roots, double *grad_coef, uint8_t *status);

/* Condition number of each root: sum_k |a_k||z|^k / (max(1,|z|) |p'(z)|). */
void or_root_condition(const double *coef, int64_t n, int d, const double *roots, double *kappa);

/* Soft root density (differentiation workload): img[iy*W + ix] += scale *
 * max(0, exp(-r^2/(2 sigma^2)) - exp(-9/2)) for every root, r the distance in
 * pixels from the root to the centre of pixel (iy, ix) (row 0 at ymax). */
void or_splat(const double *roots, int64_t n, double xmin, double xmax, double ymin, double ymax, int W, int H,
              double sigma, double scale, double *img);

/* dL/dRe z_j, dL/dIm z_j (interleaved) of L(img) for every root, given G = dL/dimg. */
void or_splat_grad(const double *roots, int64_t n, double xmin, double xmax, double ymin, double ymax, int W,
                   int H, double sigma, double scale, const double *G, double *grad);

/* Number of OpenMP threads the batch calls use by default. */
int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
