/*
 * rootdensity.h -- C ABI of libroots, the GB300 (sm_103a) library for
 * batched complex polynomial roots and root-density histograms.
 *
 * Method: R. Tang, C. Quan, "Hardware-Accelerated Algorithm for Complex
 * Function Roots Density Graph Plotting", arXiv 2507.02164.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" must point to device memory of the current
 *     CUDA device; the caller owns it. The library never frees, keeps or
 *     reallocates caller memory, and never allocates device memory itself.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls only enqueue work on it; none synchronises.
 *   - Complex numbers are interleaved (re, im): rd_c64 = 2 x float (8 B),
 *     rd_c128 = 2 x double (16 B).
 *   - Uniform-degree batches are coefficient-major ("structure of arrays"):
 *     coefficient k (of z^k, k = 0..d) of polynomial i is element k*n + i;
 *     root j of polynomial i is element j*n + i. Consecutive polynomials are
 *     consecutive in memory, so a warp reads 32 neighbours in one transaction.
 *   - Return value: RD_OK, or a negative error code. rd_last_error() gives a
 *     thread-local message for the most recent failure on the calling thread.
 *     On error nothing has been enqueued.
 *   - rd_autotune is the one exception to "never allocates, never
 *     synchronises": it allocates its own probe batch and times it with
 *     events. Call it outside any stream capture.
 */
#ifndef ROOTDENSITY_H
#define ROOTDENSITY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_ABI_VERSION 2

/* ---- return codes ---------------------------------------------------- */
#define RD_OK 0
#define RD_EINVAL (-1)        /* null pointer, bad size, degree or window   */
#define RD_ECUDA (-2)         /* CUDA launch or device query failed          */
#define RD_EUNSUPPORTED (-3)  /* dtype / mode / degree combination not built */

/* ---- per-polynomial status (uint8) ----------------------------------- */
#define RD_STATUS_OK 0
#define RD_STATUS_NOT_CONVERGED 1 /* a level used max_iters sweeps; its diagonal entry is still returned */
#define RD_STATUS_REJECTED 2      /* mixed: residual or separation check failed; backward: p'(z) singular */
#define RD_STATUS_DEGENERATE 3    /* a_d == 0 or a non-finite coefficient; roots are NaN */

typedef enum { RD_C64 = 0, RD_C128 = 1 } rd_dtype;

/* RD_PLAIN_FP64: every QR sweep in FP64.
 * RD_MIXED: QR sweeps in FP32, then `polish_steps` FP64 Newton steps per root
 * on the original coefficients and an FP64 residual / separation check. */
typedef enum { RD_PLAIN_FP64 = 0, RD_MIXED = 1 } rd_mode;

/* RD_SHIFT_WILKINSON: eigenvalue of the trailing 2x2 nearer h[m-1][m-1] on
 * every sweep. RD_SHIFT_RAYLEIGH: the paper's shift s = h[m-1][m-1] (Alg. 1),
 * with the Wilkinson shift every exc_period sweeps without deflation. */
typedef enum { RD_SHIFT_WILKINSON = 0, RD_SHIFT_RAYLEIGH = 1 } rd_shift;

typedef struct {
    double tol;            /* deflation: |h[m-1][m-2]| <= tol (|h[m-1][m-1]| + |h[m-2][m-2]|), 1-norms of re/im */
    int32_t max_iters;     /* sweeps per eigenvalue before giving up (>= 1)                     */
    int32_t shift;         /* rd_shift                                                          */
    int32_t exc_period;    /* RD_SHIFT_RAYLEIGH only; 0 = never use the Wilkinson shift        */
    int32_t polish_steps;  /* RD_MIXED: FP64 Newton steps per root (0..8)                       */
    double residual_tol;   /* RD_MIXED: reject when |p(z)| > residual_tol * sum_k |a_k||z|^k;
                              <= 0 means 64 * d * 2^-53                                         */
    double collapse_tol;   /* RD_MIXED: reject when two roots lie within collapse_tol * max(1,|z|) */
    int32_t block;         /* threads per CTA, multiple of 32 in [32, 256] (up to 512 with
                              polish_warps > 0, see below); 0 = the default                  */
    int32_t ctas_per_sm;   /* grid = ctas_per_sm x SM count; 0 = tuned default                   */
    int32_t polish_extra;  /* RD_MIXED: further Newton steps, p and p' both in FP64, for a root
                              that fails the residual check after polish_steps (0..16)          */
    int32_t fixed_sweeps;  /* 0: adaptive deflation (tol). T > 0: the paper's fixed schedule
                              (Alg. 2): exactly T sweeps per eigenvalue, no deflation test       */
    int32_t polish_mode;   /* RD_MIXED: rd_polish                                                */
    int32_t lanes;         /* lanes per polynomial: 0 or 1 = one thread holds the whole matrix;
                              2 = two lanes share it (columns split by parity, rotations
                              exchanged by warp shuffles; degree >= 2 and RD_POLISH_FP64
                              only, degree 1 always runs one lane). Two lanes measured
                              slower on GB300 at degrees 6..12; the autotuner times both   */
    int32_t polish_warps;  /* RD_MIXED (either polish mode), one lane, rd_roots_batched and
                              rd_roots_density: 0 = every warp sweeps and then polishes its
                              own 32 polynomials; P > 0 = warp-specialised CTAs, P warps of
                              each polish, check, store and bin what the other block/32 - P
                              warps sweep, handed over through a shared-memory ring, so the
                              polish (FP64 pipe, or FP32 pipe with RD_POLISH_DF) and the
                              sweeps (FP32 pipe) work at the same time. block may then be up to 512 (degrees <= 6) or 256
                              (degrees >= 7). Same roots bit for bit                       */
    int32_t ring_slots;    /* polish_warps > 0: ring slots of 32 polynomials per CTA (2..64);
                              0 = 2 x block/32                                             */
} rd_params;

/* RD_POLISH_FP64: every Newton step evaluates p(z) by FP64 Horner.
 * RD_POLISH_DF: the Newton steps run on the FP32 pipe, which GB300 runs
 * about 70x faster than its FP64 pipe: z is carried as a pair zh + zl of
 * floats (about 2^-48 relative), p(zh) is evaluated by the compensated
 * Horner scheme (error-free products and sums, as accurate as Horner in
 * twice the working precision) and p(z) = p(zh) + p'(zh) zl + p''(zh)/2 zl^2;
 * the final residual check is still an FP64 Horner evaluation and a root
 * that fails it still gets polish_extra FP64 Newton steps. */
typedef enum { RD_POLISH_FP64 = 0, RD_POLISH_DF = 1 } rd_polish;

/* Defaults: plain tol 1e-13, mixed tol 4 * 2^-24, max_iters 40, Wilkinson
 * shift, exc_period 10, 3 polish steps, 5 extra steps, residual 64 d 2^-53,
 * collapse 1e-9, adaptive deflation. RD_MIXED with polish_steps = 0 and
 * polish_extra = 0 returns the FP32 eigenvalues without polish or check. */
void rd_default_params(rd_mode mode, rd_params *out);

/* Root-density window: pixel column ix = floor((x - xmin) * W / (xmax - xmin)),
 * row iy = floor((ymax - y) * H / (ymax - ymin)) (row 0 at the top), both in
 * FP64; a root is counted when 0 <= ix < W and 0 <= iy < H (half-open bins:
 * x = xmax or y = ymin is outside), otherwise it is out of the window.
 * The paper converts solved roots to screen pixels and counts them in video
 * memory (Sec. III, "Roots to Pixels" and "Video Memory" of Table I). */
typedef struct {
    double xmin, xmax, ymin, ymax;
} rd_window;

/* Counters a solve or binning call adds to (device, all uint64, += semantics). */
typedef struct {
    uint64_t polys;          /* polynomials processed                                    */
    uint64_t status[4];      /* polynomials per status code                              */
    uint64_t sweeps;         /* QR sweeps, summed over polynomials                       */
    uint64_t pair_updates;   /* rotated row/column entry pairs of the Hessenberg sweeps  */
    uint64_t rotations;      /* Givens rotations generated                               */
    uint64_t newton_steps;   /* RD_MIXED: Newton steps taken                             */
    uint64_t binned;         /* roots counted in the histogram                           */
    uint64_t out_of_window;  /* roots outside the window (NaN included)                  */
    uint64_t clipped;        /* roots dropped before binning: by a tile clip, or (standalone
                                binning) because their polynomial's status is not OK     */
    uint64_t flops_fp32;     /* algorithmic FP32 flops of the solve (see below)          */
    uint64_t flops_fp64;     /* algorithmic FP64 flops of the solve                      */
    uint64_t wait_timeouts;  /* polynomials the warp-specialised solver abandoned after a
                                bounded wait (status REJECTED, no roots written or binned);
                                0 unless its hand-off between warps failed                */
} rd_stats;
/* Algorithmic flop convention (the method's own work, not what the hardware
 * executes): a sweep at active size m costs 20 (m(m+1) - 2) for its rotated
 * entry pairs, 24 (m - 1) for its Givens pairs and 60 for shift, unshift,
 * Wilkinson shift and deflation test, in the sweep precision. RD_MIXED adds
 * per Newton step 8d + 2 FP64 (p(z)) and 8d + 3 FP32 (p'(z), step size), and
 * per root 8d + 4 FP64 (final residual, binning) and 2d + 4 FP32 (denominator);
 * with RD_POLISH_DF a Newton step costs 66d + 50 FP32 (compensated Horner
 * and its derivative recurrences: 66 FP32 flops per coefficient) and a root
 * 8d + 6 FP64;
 * RD_PLAIN_FP64 adds 4 FP64 per root (binning). */

/* Optional per-polynomial tile clip of the full pipeline (Sec. II, domain
 * split into subregions D_i): roots are first mapped z = centre_i + radius *
 * w, then kept only if their tile, computed like a pixel on an nx x ny grid
 * over `tiles`, equals tile_index[i]. */
typedef struct {
    const double *centres;     /* device, rd_c128 [n]: centre of polynomial i's sub-disk     */
    double radius;             /* sub-disk radius (the tile half-diagonal)                    */
    const int64_t *tile_index; /* device, [n]; NULL = polynomial i lies in tile i             */
    int32_t nx, ny;            /* tile grid                                                   */
    rd_window tiles;           /* window the tile grid covers                                 */
} rd_clip;

int rd_abi_version(void);
const char *rd_last_error(void);

/* Number of streaming multiprocessors of the current device (0 on failure). */
int rd_device_sm_count(void);

/* ---- roots of a uniform-degree batch (Sec. II-B, Alg. 1 / Alg. 2) ----------
 * Roots of p_i(z) = sum_k a_ik z^k for i < n: eigenvalues of the Frobenius
 * companion matrix of the monic p_i / a_id, by single-shift QR sweeps built
 * from complex Givens rotations (Sec. II-C) applied in place to the Hessenberg
 * matrix, with bottom deflation (tol) and at most max_iters sweeps per root.
 *   coeffs  device, [degree+1][n] of `dtype` (rd_c64 or rd_c128)
 *   degree  1..12
 *   n       >= 0 (n = 0 is a no-op)
 *   params  host pointer; NULL = rd_default_params(mode)
 *   roots   device, rd_c128 [degree][n], or NULL
 *   status  device, uint8 [n], or NULL
 *   stats   device rd_stats (accumulated), or NULL
 * Order of the roots of one polynomial is unspecified. */
int rd_roots_batched(const void *coeffs, rd_dtype dtype, int degree, int64_t n, rd_mode mode,
                     const rd_params *params, double *roots, uint8_t *status, rd_stats *stats,
                     void *stream);

/* ---- self-test of the warp-specialised solver's bounded waits ------------
 * Runs the degree-6 complex64 warp-specialised kernel (params.polish_warps)
 * on coeffs [7][n] with every warp of its CTAs in the polish role, so that no
 * ring slot is ever filled: each CTA's first wait runs out after 2 s and sets
 * the CTA's abort flag, no later wait starts, and the kernel returns with
 * status[i] = RD_STATUS_REJECTED for every i < n and stats->wait_timeouts and
 * stats->status[RD_STATUS_REJECTED] increased by n. It exercises the failure
 * path of the hand-off without a GPU fault. 1 <= n <= 1024 (one wave of
 * CTAs: about 2 s); coeffs, status and stats are device pointers (required).
 * Returns RD_EINVAL on bad arguments; does not synchronise. */
int rd_ws_selftest_timeout(const void *coeffs, int64_t n, uint8_t *status, rd_stats *stats, void *stream);

/* ---- fused roots + root-density histogram ---------------------------------
 * rd_roots_batched, then every root is binned into hist (+=, uint32, row-major
 * [H][W]) with warp-aggregated atomics, without a trip through memory. clip
 * (host pointer, may be NULL) selects the full-pipeline tile clip. roots and
 * status may be NULL. The caller zeroes hist (rd_hist_clear) when it wants a
 * fresh image: calls accumulate, so a long batch may be split into chunks. */
int rd_roots_density(const void *coeffs, rd_dtype dtype, int degree, int64_t n, rd_mode mode,
                     const rd_params *params, const rd_clip *clip, rd_window window, int W, int H,
                     uint32_t *hist, double *roots, uint8_t *status, rd_stats *stats,
                     void *stream);

/* ---- standalone binning (Sec. III, Roots to Pixels) -------------------------
 * hist[iy*W + ix] += 1 for each of the n_roots roots (device rd_c128 array)
 * inside the window; others (NaN included) add to stats->out_of_window.
 *   n_polys  0: the roots stand alone (status and clip must be NULL).
 *            n > 0: the roots are a solve's output for n polynomials, root r
 *            belonging to polynomial r mod n (the [degree][n] layout of
 *            rd_roots_batched); n_roots must be a multiple of n.
 *   status   device uint8 [n_polys] or NULL: when given, only the roots of
 *            polynomials with status RD_STATUS_OK are binned.
 *   clip     host pointer or NULL: the roots are points w of their
 *            polynomials' unit disks (Sec. II, subregions D_i); root r of
 *            polynomial i is mapped to z = clip->centres[i] + clip->radius w
 *            and binned only when z lies in polynomial i's own tile
 *            (clip->tile_index[i], or i), as the fused solve's clip does.
 * Roots dropped by the status mask or the clip add to stats->clipped. The
 * pixel arithmetic is the fused solve's, operation for operation. */
int rd_density_accumulate(const double *roots, const uint8_t *status, int64_t n_roots, int64_t n_polys,
                          rd_window window, int W, int H, const rd_clip *clip, uint32_t *hist,
                          rd_stats *stats, void *stream);

/* Zero `words` 32-bit words of device memory (histogram or rd_stats). */
int rd_hist_clear(uint32_t *hist, int64_t words, void *stream);

/* ---- inputs in page-locked host memory ---------------------------------------
 * Every input array of the solve entry points (coefficients, degrees,
 * offsets, samples) is read by the kernels through its address, so it may be
 * device memory or page-locked host memory that the CUDA runtime maps into the
 * device address space at the same address (unified addressing): the kernels
 * then read it across the host link while they compute (zero copy). Passing
 * any other host address faults the kernel. rd_pointer_is_device_accessible
 * returns 1 for device or managed memory and for page-locked host memory whose
 * device address equals its host address, 0 otherwise (also when no GPU is
 * present). Host-side only; it enqueues nothing. */
int rd_pointer_is_device_accessible(const void *p);

/* ---- uneven degrees (1..12) in one pass -------------------------------------
 * Packed poly-major batch: polynomial i has degree degrees[i] and its
 * coefficients a_0..a_d are coeffs[offsets[i] .. offsets[i+1]-1] (offsets has
 * n+1 entries; n_coeffs = offsets[n] elements of `dtype`). Roots are packed
 * the same way without the leading coefficient: root j of polynomial i is
 * roots[offsets[i] - i + j] (rd_c128). The call bins the batch by degree
 * into the workspace, then solves every degree bin with a persistent kernel
 * that takes 32-polynomial tasks (16 with two lanes per polynomial) from the
 * bin's atomic queue, binning roots into hist when it is given.
 * roots (when not NULL) holds n_coeffs - n elements.
 * Polynomial i is solved when degrees[i] is 1..12 and its offsets are
 * consistent: offsets[i+1] - offsets[i] = degrees[i] + 1, offsets[i] >= i and
 * offsets[i+1] <= n_coeffs - (n - 1 - i) (its roots then lie inside the root
 * array). An inconsistent polynomial gets RD_STATUS_DEGENERATE and nothing
 * else is written for it; a consistent one of another degree gets
 * RD_STATUS_DEGENERATE and NaN roots. If the solvable polynomials need more
 * than n_coeffs coefficients in all (their ranges overlap: offsets that are
 * not monotone), none of them is solved: each gets RD_STATUS_DEGENERATE and
 * NaN roots. A well-formed batch (offsets[0] = 0, increasing, offsets[n] =
 * n_coeffs) is always consistent.
 *   ws        device scratch of at least rd_uneven_workspace_bytes(n, n_coeffs,
 *             dtype) bytes, 256-byte aligned; overwritten; must not be shared
 *             by two calls in flight at once
 *   window    host pointer; NULL with hist NULL = no binning
 *   tuning    host pointer or NULL (params.block / ctas_per_sm / lanes for every
 *             degree); see rd_uneven_tuning
 * n < 2^32 and n_coeffs <= 2^40 (RD_EINVAL otherwise;
 * rd_uneven_workspace_bytes returns 0 outside these limits). Only enqueues
 * work (16 kernel launches): the degree bins run as two chains, one on
 * `stream` and one on a helper stream of the calling host thread, forked from
 * and joined back to `stream` with events, so the whole call can be captured
 * in a CUDA graph (as two parallel branches) and `stream` orders everything
 * before and after it. The first call on a device from a host thread creates
 * the helper stream and its two events; make that call outside capture. */
typedef struct {
    /* Launch shape of each degree bin's solve kernel, indexed by the degree
     * (entries 1..12; entries 0 and 13..15 are ignored). 0 = the default.   */
    int32_t block[16];        /* threads per CTA, a multiple of 32 in [32, 256]                  */
    int32_t ctas_per_sm[16];  /* resident CTAs per SM (0 = the occupancy maximum)                 */
    int32_t lanes[16];        /* lanes per polynomial, 1 or 2 (0 = params.lanes)                  */
    int32_t polish_warps[16]; /* RD_MIXED, degrees 1..8: P > 0 runs the bin in warp-specialised
                                 CTAs of block[d] threads (a multiple of 32 up to 512 at degrees
                                 <= 6, 256 at 7 and 8; 0 = the largest), P warps of each polishing
                                 what the others sweep (see rd_params.polish_warps), one lane per
                                 polynomial, ctas_per_sm ignored; 0 = every warp sweeps and then
                                 polishes. The same roots either way                                */
} rd_uneven_tuning;

size_t rd_uneven_workspace_bytes(int64_t n, int64_t n_coeffs, rd_dtype dtype);
int rd_roots_uneven(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets,
                    int64_t n, int64_t n_coeffs, rd_mode mode, const rd_params *params,
                    const rd_uneven_tuning *tuning, const rd_window *window, int W, int H, uint32_t *hist,
                    double *roots, uint8_t *status, rd_stats *stats, void *ws, size_t ws_bytes, void *stream);

/* ---- uneven degrees without a caller-provided workspace ----------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory where they need roots: code running under
 * an allocator owned by a host framework, loops where cudaMalloc/cudaFree
 * would synchronise the device, deployments with a device-memory budget
 * fixed in advance. It behaves like rd_roots_uneven (same arguments without
 * ws/ws_bytes, same results; its degree bins all run on `stream`, so it makes
 * no helper stream either) but uses a scratch array of
 * RD_STATIC_SCRATCH_BYTES bytes built into the library: that memory is held
 * on every GPU that loads the library until the process exits, and the call
 * itself allocates and frees nothing.
 *   - A batch whose rd_uneven_workspace_bytes(n, n_coeffs, dtype) exceeds
 *     RD_STATIC_SCRATCH_BYTES is rejected with RD_EINVAL and a message; split
 *     it, or use rd_roots_uneven.
 *   - A call outside stream capture looks up the scratch array's device
 *     address (cudaGetSymbolAddress) with its device current, so the
 *     address stays right after a cudaDeviceReset; a call under capture uses
 *     the address the last call outside capture found on that device. Make
 *     the first call on each device before any stream capture begins (a
 *     first call under capture returns RD_EINVAL).
 *   - All calls on a device share the one array and each leaves its contents
 *     behind (the next call clears what must start at zero). Two calls whose
 *     work overlaps on the GPU (different streams, or different host threads)
 *     race on it and give wrong results: serialise them. */
#define RD_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int rd_roots_uneven_static(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets,
                           int64_t n, int64_t n_coeffs, rd_mode mode, const rd_params *params,
                           const rd_uneven_tuning *tuning, const rd_window *window, int W, int H,
                           uint32_t *hist, double *roots, uint8_t *status, rd_stats *stats, void *stream);

/* ---- implicit-differentiation adjoint ---------------------------------------
 * grad_coeffs[k*n+i] = sum_j conj(-z_ij^k / p_i'(z_ij)) * grad_roots[j*n+i],
 * k = 0..degree (p(z) = 0 defines z(a); dz/da_k = -z^k / p'(z)), the gradient
 * convention of PyTorch (grad = dL/dRe + i dL/dIm). Nothing from the forward
 * QR sweeps is needed. A root with |p'(z)| <= 1e-300 (or non-finite) adds
 * nothing and sets status RD_STATUS_REJECTED.
 *   coeffs, grad_coeffs  device, [degree+1][n] of dtype (grad_coeffs overwritten)
 *   roots, grad_roots    device, rd_c128 [degree][n]
 *   status               device uint8 [n] or NULL
 * rd_c128 computes in FP64, rd_c64 in FP32. */
int rd_roots_backward(const void *coeffs, rd_dtype dtype, int degree, int64_t n,
                      const double *roots, const double *grad_roots, void *grad_coeffs,
                      uint8_t *status, void *stream);

/* The same adjoint for a packed batch of uneven degrees (the layout of
 * rd_roots_uneven): polynomial i has degree degrees[i] and coefficients
 * coeffs[offsets[i] .. offsets[i+1]-1]; its roots and their gradients are
 * roots[offsets[i] - i + j], grad_roots[offsets[i] - i + j] (rd_c128, n_coeffs
 * - n elements each); grad_coeffs (n_coeffs elements of dtype) is written
 * like coeffs. A polynomial is differentiated under the consistency rule of
 * rd_roots_uneven; an inconsistent one gets RD_STATUS_DEGENERATE and nothing
 * is written for it, a consistent one of degree 0 or above 12 gets
 * RD_STATUS_DEGENERATE and zero gradients. n < 2^32, n_coeffs <= 2^40. */
int rd_roots_backward_uneven(const void *coeffs, rd_dtype dtype, const uint8_t *degrees,
                             const int64_t *offsets, int64_t n, int64_t n_coeffs, const double *roots,
                             const double *grad_roots, void *grad_coeffs, uint8_t *status, void *stream);

/* ---- L2 approximation on sub-disks (Sec. II-A) ------------------------------
 * Nodes of the quadrature on the unit disk: radii r_p (Gauss-Legendre on
 * [0,1], p < nr, ascending) with weights w_p, and angles theta_q = 2 pi q / nt
 * (q < nt), so that f is sampled at c + rho r_p e^{i theta_q}.
 * Host function; r and w are host arrays of nr doubles, theta a host array of
 * nt doubles or NULL. 1 <= nr <= 32, 1 <= nt <= 4096. */
int rd_l2_nodes(int nr, int nt, double *r, double *theta, double *w);

/* For each sub-disk s < n, samples[s][p*nt + q] = g_s(r_p e^{i theta_q})
 * (device rd_c128; g_s(w) = f(c_s + rho w)). Computes the degree-`degree`
 * least-squares polynomial of g_s on the unit disk for the inner product
 * <g, h> = integral g conj(h) dA, whose Gram matrix is diagonal:
 * a_j = (j+1)/pi <g, w^j>. coeffs: device rd_c128, coefficient-major
 * [degree+1][n] (ready for rd_roots_*). nt must be 32; nr <= 32; degree <= 12.
 * The coefficients stay in the local variable w of each sub-disk (expanding
 * them in z would scale a_j by rho^-j). centres (device rd_c128 [n], the
 * sub-disk centres c_s) and radius (rho) describe that map z = c_s + rho w:
 * when map is not NULL they are checked and written into map->centres and
 * map->radius, which the caller completes with its tile grid and passes to
 * rd_roots_density or rd_density_accumulate; the kernel does not read them.
 * centres may be NULL only when map is NULL. */
int rd_l2_approx(const double *samples, int64_t n, int nr, int nt, int degree, int precision,
                 const double *centres, double radius, double *coeffs, rd_clip *map, void *stream);
/* precision: RD_L2_FP64 sums in FP64 (the FP64 pipe bounds the kernel);
 * RD_L2_DF sums in double-float arithmetic on the FP32 pipe (about 2^-48
 * relative per term, ~1e-14 on the coefficients relative to the largest of a
 * sub-disk), after scaling each sub-disk's samples by a power of two. */
#define RD_L2_FP64 0
#define RD_L2_DF 1

/* ---- soft root density (the differentiation workload's loss) ------------------
 * Not in the paper, which counts roots into pixels (Sec. III): a loss needs an
 * image that moves smoothly with the roots. Pixel (iy, ix) of the W x H image
 * has its centre at x = xmin + (ix + 1/2) px, y = ymax - (iy + 1/2) py
 * (px = (xmax - xmin)/W, py = (ymax - ymin)/H, row 0 at ymax, as the
 * histogram). rd_splat adds, for every root z_j,
 *   img[iy*W + ix] += scale * max(0, exp(-r^2 / (2 sigma^2)) - exp(-9/2)),
 * r the distance from z_j to the pixel centre in pixel units (zero beyond
 * 3 sigma); a non-finite root adds nothing. FP64 atomic adds: repeated calls
 * agree to rounding, not bit for bit.
 *   roots       device rd_c128 [n]
 *   img         device double [H][W], accumulated (the caller zeroes it)
 *   0 < sigma <= 2 (the stencil is at most 13 x 13 pixels); scale >= 0;
 *   W, H >= 1.
 * rd_splat_backward writes grad_roots[j] = dL/dRe z_j + i dL/dIm z_j (PyTorch's
 * gradient convention) of a loss L(img), given grad_img = dL/dimg (device
 * double [H][W]); grad_roots: device rd_c128 [n], overwritten. */
int rd_splat(const double *roots, int64_t n, rd_window window, int W, int H, double sigma, double scale,
             int precision, double *img, void *stream);
int rd_splat_backward(const double *roots, int64_t n, rd_window window, int W, int H, double sigma, double scale,
                      int precision, const double *grad_img, double *grad_roots, void *stream);
/* precision: RD_SPLAT_FP64 computes the stencil in FP64 (~1e-14 relative);
 * RD_SPLAT_FP32 in FP32 on the FP32 pipe (~1e-6 relative; for complex64
 * coefficients, whose roots carry ~1e-7 anyway). Image and gradients are
 * float64 in both. */
#define RD_SPLAT_FP64 0
#define RD_SPLAT_FP32 1

/* ---- the whole path for an analytic f, one launch -----------------------------
 * Sec. II: the region is covered by sub-disks; on each, f is approximated by a
 * polynomial g (Sec. II-A, least squares on the disk, a_j = (j+1)/pi <g, w^j>
 * in the local variable w, z = c + rho w), the roots of g are found (Sec.
 * II-B/II-C) and a root is counted in the tile whose sub-disk produced it
 * (each zero of f once). rd_field_density does all of it in one kernel: it
 * evaluates f in FP64 at the 16 x 32 polar nodes of every tile's sub-disk
 * (the rd_l2_nodes radii, theta_q = 2 pi q / 32), forms the coefficients with
 * double-float sums (as RD_L2_DF), solves them (rd_roots_density, `mode`),
 * keeps the roots that fall in their own tile and bins them. No sample array
 * is read or written.
 * Tiles: nx x ny over spec->tiles, tile t = iy * nx + ix from the top-left
 * corner, centre (xmin + (ix + 1/2) w, ymax - (iy + 1/2) h), w = (xmax - xmin)
 * / nx, h = (ymax - ymin) / ny, each product and sum rounded once.
 *   f         RD_F_SIN_CUBE: f(z) = sin(z^3) + z/2; RD_F_POLY: f(z) = sum_k
 *             poly[k] z^k, k <= poly_degree <= 12
 *   spec      host pointer; nr must be 16 and degree 6
 *   coeffs    device rd_c128 [degree+1][nx*ny] (local variable w) or NULL
 *   roots     device rd_c128 [degree][nx*ny] (local variable w) or NULL
 *   status    device uint8 [nx*ny] or NULL
 *   hist      device uint32 [H][W] over window (accumulated, never cleared);
 *             required
 * params: as rd_roots_density; lanes must be 0 or 1 and polish_mode
 * RD_POLISH_FP64. Errors: RD_EINVAL for a bad spec, window or pointer,
 * RD_EUNSUPPORTED for another nr or degree. */
typedef enum { RD_F_SIN_CUBE = 0, RD_F_POLY = 1 } rd_field;
typedef struct {
    rd_window tiles;        /* the tiled region                                     */
    int32_t nx, ny;         /* tile grid, nx * ny < 2^31                            */
    double radius;          /* sub-disk radius; <= 0: half the tile diagonal        */
    int32_t nr;             /* radial nodes: 16                                     */
    int32_t degree;         /* degree of g: 6                                       */
    int32_t poly_degree;    /* RD_F_POLY: degree of f, 0..12                        */
    int32_t reserved;       /* must be 0                                            */
    double poly[26];        /* RD_F_POLY: c_0 .. c_12 as (re, im) pairs             */
} rd_field_spec;
int rd_field_density(rd_field f, const rd_field_spec *spec, rd_mode mode, const rd_params *params,
                     rd_window window, int W, int H, uint32_t *hist, double *coeffs, double *roots,
                     uint8_t *status, rd_stats *stats, void *stream);

/* ---- launch-shape autotuner ---------------------------------------------------
 * Times the launch shapes of rd_roots_density for one degree, mode, polish
 * mode (rd_polish; RD_MIXED only, else ignored) and storage type on a probe batch of n_probe complex-Gaussian polynomials (real and
 * imaginary parts N(0,1), drawn on the device from a fixed seed per degree)
 * binned into a 1920 x 1080 histogram over [-3,3] x [-1.6875,1.6875], and
 * returns the fastest. Candidates: lanes per polynomial (1; 2 from degree 2 on,
 * with the FP64 polish), threads per CTA 32, 64, 128, 256, resident CTAs per
 * SM (the occupancy maximum or fewer), each with every warp sweeping then
 * polishing; and for RD_MIXED the warp-specialised shapes (polish_warps > 0),
 * a set for each polish mode. Two lanes are not a candidate with RD_POLISH_DF.
 * Each shape runs once untimed, then `reps` times (1..15) timed with CUDA
 * events; its time is the median. A shape that cannot be launched (too many
 * registers for the block) is recorded with ms < 0 and skipped. This is the
 * one entry point that allocates (the probe batch and its histogram, freed
 * before it returns) and synchronises: call it outside any stream capture.
 *   out        host; the fastest shape, and the fastest with polish_warps = 0
 *              (the form the uneven-degree bins run)
 *   table      host array of table_cap entries or NULL; receives every timed
 *              shape (at most table_cap), *table_len their number
 * 1 <= degree <= 12, 1024 <= n_probe <= 2^24. */
typedef struct {
    int32_t lanes, block, ctas_per_sm, polish_warps;
    float ms;      /* median milliseconds of one rd_roots_density call on the probe, < 0: not launchable */
} rd_tune_entry;
typedef struct {
    rd_tune_entry best;      /* fastest shape overall                                      */
    rd_tune_entry one_role;  /* fastest shape with polish_warps = 0                         */
    int32_t n_candidates;    /* shapes timed (launchable or not)                           */
    int32_t reserved;
} rd_tuning;
int rd_autotune(int degree, rd_mode mode, int polish_mode, rd_dtype dtype, int64_t n_probe, int reps,
                rd_tuning *out, rd_tune_entry *table, int table_cap, int *table_len);

/* ---- ALU throughput probe ------------------------------------------------------
 * Not part of the method: the denominator of its roofline. Enqueues one kernel
 * of independent fused multiply-add chains, RD_PEAK_FP32 (packed FP32 pairs,
 * fma.rn.f32x2, on the FP32 pipe) or RD_PEAK_FP64 (DFMA on the FP64 pipe):
 * ctas_per_sm x SM count CTAs of 256 threads, each thread `iters` x 16 steps
 * of 8 independent chains, i.e. iters x 256 FP32 or iters x 128 FP64 FMAs.
 * *flops (host) receives the
 * flops the launch performs (2 per FMA); the caller times it with events on
 * `stream`. sink: device, 8 bytes, written only if a chain ends on a value it
 * cannot reach (it keeps the chains from being optimised away).
 * 1 <= iters <= 2^24, 1 <= ctas_per_sm <= 32. */
#define RD_PEAK_FP32 0
#define RD_PEAK_FP64 1
int rd_alu_peak(int kind, int64_t iters, int ctas_per_sm, double *sink, uint64_t *flops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ROOTDENSITY_H */
