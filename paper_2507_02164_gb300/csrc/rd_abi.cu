// rd_abi.cu -- the extern "C" entry points of libroots: argument checks,
// defaults and dispatch to the kernels. Every call only enqueues work on the
// caller's stream; nothing here allocates device memory or synchronises.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rd_common.cuh"
#include "rd_solve.cuh"

namespace rd {
int launch_solve_mixed(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st);
int launch_solve_plain(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st);
int launch_solve2(int degree, rd_dtype dt, bool mixed, const SolveArgs &a, int block, int ctas_per_sm, cudaStream_t st);
int launch_solve_ws(int degree, rd_dtype dt, const SolveArgs &a, int block, int ctas_per_sm, int polish_warps,
                    int ring_slots, cudaStream_t st);
int launch_solve_ws_selftest(const SolveArgs &a, cudaStream_t st);
int lanes_for(int degree, bool mixed, int polish_mode, int requested);
int launch_density(const double *roots, int64_t n, const DensityArgs &D, uint32_t *hist, rd_stats *stats,
                   cudaStream_t st);
int launch_backward_uneven(rd_dtype dt, const void *coeffs, const uint8_t *degrees, const int64_t *offsets,
                           int64_t n, int64_t n_coeffs, const double *roots, const double *grad_roots,
                           void *grad_coeffs, uint8_t *status, cudaStream_t st);
int launch_clear(uint32_t *p, int64_t words, cudaStream_t st);
int launch_backward(int degree, rd_dtype dt, const void *coeffs, const double *roots, const double *grad_roots,
                    void *grad_coeffs, uint8_t *status, int64_t n, cudaStream_t st);
int l2_nodes_host(int nr, double *r, double *w);
size_t uneven_workspace_bytes(int64_t n, int64_t n_coeffs, rd_dtype dt);
int launch_uneven(const SolveArgs &a, rd_dtype dt, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                  int64_t n_coeffs, bool mixed, void *ws, const int *block, const int *cps, const int *lanes,
                  const int *pw, bool fork, cudaStream_t st);
int launch_l2(const double *samples, int64_t n, int nr, int degree, double *coeffs, int precision,
              cudaStream_t st);
int roots_uneven_common(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                        int64_t n_coeffs, rd_mode mode, const rd_params *params, const rd_uneven_tuning *tuning,
                        const rd_window *window, int W, int H, uint32_t *hist, double *roots, uint8_t *status,
                        rd_stats *stats, void *ws, size_t ws_bytes, bool fork, void *stream);
int launch_field(const SolveArgs &a, const rd_field_spec &spec, int func, double rho, bool mixed, double *coeffs,
                 int ctas_per_sm, cudaStream_t st);
int launch_splat(const double *roots, int64_t n, const rd_window &w, int W, int H, double sigma, double scale,
                 int precision, double *img, cudaStream_t st);
int launch_splat_backward(const double *roots, int64_t n, const rd_window &w, int W, int H, double sigma,
                          double scale, int precision, const double *G, double *grad, cudaStream_t st);
}  // namespace rd

static thread_local char g_err[512] = "";

int rd_set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int rd_check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_set_error(RD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return RD_OK;
}

// SM count of the current device, queried once per device.
int rd_sm_count_cached()
{
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        cache[dev] = v;
    }
    return cache[dev];
}

namespace {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool window_ok(const rd_window &w)
{
    return std::isfinite(w.xmin) && std::isfinite(w.xmax) && std::isfinite(w.ymin) && std::isfinite(w.ymax) &&
           w.xmin < w.xmax && w.ymin < w.ymax;
}

rd::Binner make_binner(const rd_window &w, int W, int H)
{
    rd::Binner b;
    b.xmin = w.xmin;
    b.ymax = w.ymax;
    b.sx = (double)W / (w.xmax - w.xmin);
    b.sy = (double)H / (w.ymax - w.ymin);
    b.W = W;
    b.H = H;
    return b;
}

int check_params(const rd_params &p)
{
    if (!(p.tol >= 0.0) || !std::isfinite(p.tol)) return rd_set_error(RD_EINVAL, "params.tol must be finite and >= 0");
    if (p.max_iters < 1 || p.max_iters > 100000) return rd_set_error(RD_EINVAL, "params.max_iters must be in [1, 100000]");
    if (p.shift != RD_SHIFT_WILKINSON && p.shift != RD_SHIFT_RAYLEIGH) return rd_set_error(RD_EINVAL, "params.shift invalid");
    if (p.exc_period < 0) return rd_set_error(RD_EINVAL, "params.exc_period must be >= 0");
    if (p.polish_steps < 0 || p.polish_steps > 8) return rd_set_error(RD_EINVAL, "params.polish_steps must be in [0, 8]");
    if (!std::isfinite(p.residual_tol) || !std::isfinite(p.collapse_tol) || p.collapse_tol < 0)
        return rd_set_error(RD_EINVAL, "params.residual_tol / collapse_tol invalid");
    if (p.polish_warps < 0 || p.polish_warps > 15) return rd_set_error(RD_EINVAL, "params.polish_warps must be in [0, 15]");
    if (p.ring_slots != 0 && (p.ring_slots < 2 || p.ring_slots > 64))
        return rd_set_error(RD_EINVAL, "params.ring_slots must be 0 or in [2, 64]");
    const int block_max = p.polish_warps > 0 ? 512 : 256;
    if (p.block != 0 && (p.block < 32 || p.block > block_max || p.block % 32 != 0))
        return rd_set_error(RD_EINVAL, "params.block must be 0 or a multiple of 32 in [32, %d]", block_max);
    if (p.ctas_per_sm < 0 || p.ctas_per_sm > 64) return rd_set_error(RD_EINVAL, "params.ctas_per_sm must be in [0, 64]");
    if (p.polish_extra < 0 || p.polish_extra > 16) return rd_set_error(RD_EINVAL, "params.polish_extra must be in [0, 16]");
    if (p.polish_mode != RD_POLISH_FP64 && p.polish_mode != RD_POLISH_DF)
        return rd_set_error(RD_EINVAL, "params.polish_mode must be RD_POLISH_FP64 or RD_POLISH_DF");
    if (p.lanes < 0 || p.lanes > 2) return rd_set_error(RD_EINVAL, "params.lanes must be 0, 1 or 2");
    if (p.lanes == 2 && p.polish_mode != RD_POLISH_FP64)
        return rd_set_error(RD_EINVAL, "params.lanes = 2 needs polish_mode RD_POLISH_FP64");
    if (p.fixed_sweeps < 0 || p.fixed_sweeps > p.max_iters)
        return rd_set_error(RD_EINVAL, "params.fixed_sweeps must be in [0, max_iters]");
    if (p.polish_warps > 0 && p.lanes == 2)
        return rd_set_error(RD_EINVAL, "params.polish_warps > 0 needs one lane per polynomial");
    return RD_OK;
}

// Validate a tile clip (host struct, device arrays) for n polynomials.
int check_clip(const rd_clip &c, int64_t n)
{
    if (!c.centres || !aligned(c.centres, 16)) return rd_set_error(RD_EINVAL, "clip.centres null or misaligned");
    if (!(c.radius > 0) || !std::isfinite(c.radius)) return rd_set_error(RD_EINVAL, "clip.radius must be > 0");
    if (c.nx < 1 || c.ny < 1 || !window_ok(c.tiles)) return rd_set_error(RD_EINVAL, "clip tile grid invalid");
    if (c.tile_index && !aligned(c.tile_index, 8)) return rd_set_error(RD_EINVAL, "clip.tile_index misaligned");
    if (!c.tile_index && n > (int64_t)c.nx * c.ny)
        return rd_set_error(RD_EINVAL, "clip: n exceeds nx*ny without tile_index");
    return RD_OK;
}

// Validate the arguments shared by every solve entry point and fill the
// kernel argument block (everything except the coefficient layout).
int build_solve_args(rd_dtype dtype, int degree_for_tol, rd_mode mode, const rd_params *params, const rd_clip *clip,
                     const rd_window *window, int W, int H, uint32_t *hist, double *roots, uint8_t *status,
                     rd_stats *stats, rd::SolveArgs &a, rd_params &p)
{
    if (dtype != RD_C64 && dtype != RD_C128) return rd_set_error(RD_EINVAL, "dtype must be RD_C64 or RD_C128");
    if (mode != RD_PLAIN_FP64 && mode != RD_MIXED) return rd_set_error(RD_EINVAL, "mode must be RD_PLAIN_FP64 or RD_MIXED");
    if (roots && !aligned(roots, 16)) return rd_set_error(RD_EINVAL, "roots misaligned (16 B)");
    if (stats && !aligned(stats, 8)) return rd_set_error(RD_EINVAL, "stats misaligned (8 B)");
    if (params) p = *params;
    else rd_default_params(mode, &p);
    int rc = check_params(p);
    if (rc) return rc;
    std::memset(&a, 0, sizeof(a));
    a.tol = p.tol;
    a.max_iters = p.max_iters;
    a.shift = p.shift;
    a.exc_period = p.exc_period;
    a.polish_steps = p.polish_steps;
    a.polish_extra = p.polish_extra;
    a.fixed_sweeps = p.fixed_sweeps;
    a.polish_mode = p.polish_mode;
    a.residual_tol = p.residual_tol > 0 ? p.residual_tol : 64.0 * degree_for_tol * std::ldexp(1.0, -53);
    a.collapse_tol = p.collapse_tol;
    a.roots = roots;
    a.status = status;
    a.stats = stats;
    if (hist) {
        if (!window || !window_ok(*window)) return rd_set_error(RD_EINVAL, "window must be finite with xmin < xmax, ymin < ymax");
        if (W < 1 || H < 1 || (int64_t)W * H > ((int64_t)1 << 31)) return rd_set_error(RD_EINVAL, "bad histogram size %d x %d", W, H);
        if (!aligned(hist, 4)) return rd_set_error(RD_EINVAL, "hist misaligned");
        a.hist = hist;
        a.bin = make_binner(*window, W, H);
        if (clip) {
            if (!clip->centres || !aligned(clip->centres, 16)) return rd_set_error(RD_EINVAL, "clip.centres null or misaligned");
            if (!(clip->radius > 0) || !std::isfinite(clip->radius)) return rd_set_error(RD_EINVAL, "clip.radius must be > 0");
            if (clip->nx < 1 || clip->ny < 1 || !window_ok(clip->tiles)) return rd_set_error(RD_EINVAL, "clip tile grid invalid");
            if (clip->tile_index && !aligned(clip->tile_index, 8)) return rd_set_error(RD_EINVAL, "clip.tile_index misaligned");
            a.clip_on = 1;
            a.centres = clip->centres;
            a.radius = clip->radius;
            a.tile_index = clip->tile_index;
            a.tiles = make_binner(clip->tiles, clip->nx, clip->ny);
        }
    } else if (clip) {
        return rd_set_error(RD_EINVAL, "clip needs a histogram");
    }
    return RD_OK;
}

int solve_common(const void *coeffs, rd_dtype dtype, int degree, int64_t n, rd_mode mode, const rd_params *params,
                 const rd_clip *clip, const rd_window *window, int W, int H, uint32_t *hist, double *roots,
                 uint8_t *status, rd_stats *stats, void *stream)
{
    if (degree < 1 || degree > 12) return rd_set_error(RD_EUNSUPPORTED, "degree %d outside 1..12", degree);
    if (n < 0) return rd_set_error(RD_EINVAL, "n < 0");
    if (n > ((int64_t)1 << 40)) return rd_set_error(RD_EINVAL, "n too large");
    size_t el = dtype == RD_C64 ? 8 : 16;
    if (n > 0 && (!coeffs || !aligned(coeffs, el))) return rd_set_error(RD_EINVAL, "coeffs null or misaligned");
    rd::SolveArgs a;
    rd_params p;
    int rc = build_solve_args(dtype, degree, mode, params, clip, window, W, H, hist, roots, status, stats, a, p);
    if (rc) return rc;
    if (clip && !clip->tile_index && n > (int64_t)clip->nx * clip->ny)
        return rd_set_error(RD_EINVAL, "clip: n exceeds nx*ny without tile_index");
    a.coeffs = coeffs;
    a.n = n;
    if (n == 0) return RD_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p.polish_warps > 0) {
        if (mode != RD_MIXED) return rd_set_error(RD_EINVAL, "params.polish_warps > 0 needs RD_MIXED");
        return rd::launch_solve_ws(degree, dtype, a, p.block, p.ctas_per_sm, p.polish_warps, p.ring_slots, st);
    }
    int block = p.block ? p.block : 128;
    if (rd::lanes_for(degree, mode == RD_MIXED, p.polish_mode, p.lanes) == 2)
        return rd::launch_solve2(degree, dtype, mode == RD_MIXED, a, block, p.ctas_per_sm, st);
    if (mode == RD_MIXED) return rd::launch_solve_mixed(degree, dtype, a, block, p.ctas_per_sm, st);
    return rd::launch_solve_plain(degree, dtype, a, block, p.ctas_per_sm, st);
}

}  // namespace

extern "C" {

int rd_abi_version(void) { return RD_ABI_VERSION; }

int rd_pointer_is_device_accessible(const void *p)
{
    if (!p) return 0;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of the query
        return 0;
    }
    switch (attr.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
        return 1;
    case cudaMemoryTypeHost:
        return attr.devicePointer == p ? 1 : 0;
    default:
        return 0;
    }
}

const char *rd_last_error(void) { return g_err; }

int rd_device_sm_count(void)
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return v;
}

void rd_default_params(rd_mode mode, rd_params *out)
{
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->tol = mode == RD_MIXED ? 4.0 * std::ldexp(1.0, -24) : 1e-13;
    out->max_iters = 40;
    out->shift = RD_SHIFT_WILKINSON;
    out->exc_period = 10;
    out->polish_steps = 3;
    out->residual_tol = 0.0;
    out->collapse_tol = 1e-9;
    out->block = 0;
    out->ctas_per_sm = 0;
    out->polish_extra = 5;
    out->fixed_sweeps = 0;
    out->polish_mode = RD_POLISH_FP64;
    out->lanes = 0;
    out->polish_warps = 0;
    out->ring_slots = 0;
}

int rd_ws_selftest_timeout(const void *coeffs, int64_t n, uint8_t *status, rd_stats *stats, void *stream)
{
    if (n < 1 || n > 1024) return rd_set_error(RD_EINVAL, "n must be in [1, 1024]");
    if (!coeffs || !aligned(coeffs, 8)) return rd_set_error(RD_EINVAL, "coeffs null or misaligned");
    if (!status || !stats || !aligned(stats, 8)) return rd_set_error(RD_EINVAL, "status and stats are required");
    rd::SolveArgs a;
    rd_params p;
    int rc = build_solve_args(RD_C64, 6, RD_MIXED, nullptr, nullptr, nullptr, 0, 0, nullptr, nullptr, status, stats,
                              a, p);
    if (rc) return rc;
    a.coeffs = coeffs;
    a.n = n;
    return rd::launch_solve_ws_selftest(a, reinterpret_cast<cudaStream_t>(stream));
}

int rd_roots_batched(const void *coeffs, rd_dtype dtype, int degree, int64_t n, rd_mode mode, const rd_params *params,
                     double *roots, uint8_t *status, rd_stats *stats, void *stream)
{
    return solve_common(coeffs, dtype, degree, n, mode, params, nullptr, nullptr, 0, 0, nullptr, roots, status, stats,
                        stream);
}

int rd_roots_density(const void *coeffs, rd_dtype dtype, int degree, int64_t n, rd_mode mode, const rd_params *params,
                     const rd_clip *clip, rd_window window, int W, int H, uint32_t *hist, double *roots,
                     uint8_t *status, rd_stats *stats, void *stream)
{
    if (!hist) return rd_set_error(RD_EINVAL, "hist is null");
    return solve_common(coeffs, dtype, degree, n, mode, params, clip, &window, W, H, hist, roots, status, stats,
                        stream);
}

int rd_density_accumulate(const double *roots, const uint8_t *status, int64_t n_roots, int64_t n_polys,
                          rd_window window, int W, int H, const rd_clip *clip, uint32_t *hist, rd_stats *stats,
                          void *stream)
{
    if (n_roots < 0 || n_polys < 0) return rd_set_error(RD_EINVAL, "n_roots and n_polys must be >= 0");
    if (!hist || !aligned(hist, 4)) return rd_set_error(RD_EINVAL, "hist null or misaligned");
    if (n_roots > 0 && (!roots || !aligned(roots, 16))) return rd_set_error(RD_EINVAL, "roots null or misaligned");
    if (!window_ok(window)) return rd_set_error(RD_EINVAL, "window must be finite with xmin < xmax, ymin < ymax");
    if (W < 1 || H < 1 || (int64_t)W * H > ((int64_t)1 << 31)) return rd_set_error(RD_EINVAL, "bad histogram size");
    if (stats && !aligned(stats, 8)) return rd_set_error(RD_EINVAL, "stats misaligned");
    if ((status || clip) && n_polys == 0) return rd_set_error(RD_EINVAL, "status and clip need n_polys > 0");
    if (n_polys > 0 && n_roots % n_polys != 0)
        return rd_set_error(RD_EINVAL, "n_roots (%lld) must be a multiple of n_polys (%lld)", (long long)n_roots,
                            (long long)n_polys);
    rd::DensityArgs D;
    std::memset(&D, 0, sizeof(D));
    D.bin = make_binner(window, W, H);
    D.status = status;
    D.n_polys = n_polys;
    if (clip) {
        int rc = check_clip(*clip, n_polys);
        if (rc) return rc;
        D.clip_on = 1;
        D.centres = clip->centres;
        D.radius = clip->radius;
        D.tile_index = clip->tile_index;
        D.tiles = make_binner(clip->tiles, clip->nx, clip->ny);
    }
    if (n_roots == 0) return RD_OK;
    return rd::launch_density(roots, n_roots, D, hist, stats, reinterpret_cast<cudaStream_t>(stream));
}

int rd_hist_clear(uint32_t *hist, int64_t words, void *stream)
{
    if (words < 0) return rd_set_error(RD_EINVAL, "words < 0");
    if (words == 0) return RD_OK;
    if (!hist || !aligned(hist, 4)) return rd_set_error(RD_EINVAL, "hist null or misaligned");
    return rd::launch_clear(hist, words, reinterpret_cast<cudaStream_t>(stream));
}

size_t rd_uneven_workspace_bytes(int64_t n, int64_t n_coeffs, rd_dtype dtype)
{
    if (dtype != RD_C64 && dtype != RD_C128) return 0;
    return rd::uneven_workspace_bytes(n, n_coeffs, dtype);  // 0 outside n < 2^32, n_coeffs <= 2^40
}

int rd_roots_uneven(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                    int64_t n_coeffs, rd_mode mode, const rd_params *params, const rd_uneven_tuning *tuning,
                    const rd_window *window, int W, int H, uint32_t *hist, double *roots, uint8_t *status,
                    rd_stats *stats, void *ws, size_t ws_bytes, void *stream)
{
    return rd::roots_uneven_common(coeffs, dtype, degrees, offsets, n, n_coeffs, mode, params, tuning, window, W, H,
                                   hist, roots, status, stats, ws, ws_bytes, true, stream);
}

}  // extern "C"

namespace rd {

// rd_roots_uneven's work; fork = false keeps every degree bin on `stream`
// (no helper stream is made: the allocation-free entry point).
int roots_uneven_common(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                        int64_t n_coeffs, rd_mode mode, const rd_params *params, const rd_uneven_tuning *tuning,
                        const rd_window *window, int W, int H, uint32_t *hist, double *roots, uint8_t *status,
                        rd_stats *stats, void *ws, size_t ws_bytes, bool fork, void *stream)
{
    if (n < 0 || n_coeffs < 0) return rd_set_error(RD_EINVAL, "n and n_coeffs must be >= 0");
    if (n >= ((int64_t)1 << 32)) return rd_set_error(RD_EINVAL, "n must be below 2^32");
    if (n_coeffs > ((int64_t)1 << 40)) return rd_set_error(RD_EINVAL, "n_coeffs must be at most 2^40");
    if ((hist == nullptr) != (window == nullptr)) return rd_set_error(RD_EINVAL, "hist and window go together");
    rd::SolveArgs a;
    rd_params p;
    int rc = build_solve_args(dtype, 12, mode, params, nullptr, window, W, H, hist, roots, status, stats, a, p);
    if (rc) return rc;
    if (p.residual_tol <= 0) a.residual_tol = -1.0;  // per-degree default 64 d 2^-53, set in the kernel
    if (p.polish_warps != 0) return rd_set_error(RD_EINVAL, "params.polish_warps must be 0 for uneven batches");
    if (n == 0) return RD_OK;
    size_t el = dtype == RD_C64 ? 8 : 16;
    if (!coeffs || !aligned(coeffs, el)) return rd_set_error(RD_EINVAL, "coeffs null or misaligned");
    if (!degrees || !offsets || !aligned(offsets, 8)) return rd_set_error(RD_EINVAL, "degrees / offsets null or misaligned");
    if (!ws || !aligned(ws, 256)) return rd_set_error(RD_EINVAL, "workspace null or not 256-byte aligned");
    size_t need = rd::uneven_workspace_bytes(n, n_coeffs, dtype);
    if (ws_bytes < need) return rd_set_error(RD_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    int block[16], cps[16], lanes[16], pw[16];
    for (int d = 0; d < 16; ++d) {
        block[d] = p.block ? p.block : 128;
        cps[d] = p.ctas_per_sm;
        lanes[d] = p.lanes;
        pw[d] = 0;
        if (tuning && d >= 1 && d <= 12 && tuning->polish_warps[d] != 0) {
            // the warp-specialised form of this bin
            const int P = tuning->polish_warps[d];
            const int maxb = d <= 6 ? 512 : 256;
            const int b = tuning->block[d] ? tuning->block[d] : maxb;
            if (d > 8) return rd_set_error(RD_EINVAL, "tuning.polish_warps[%d]: built for degrees up to 8", d);
            if (mode != RD_MIXED) return rd_set_error(RD_EINVAL, "tuning.polish_warps[%d] needs RD_MIXED", d);
            if (b < 64 || b > maxb || b % 32)
                return rd_set_error(RD_EINVAL, "tuning.block[%d] must be a multiple of 32 in [64, %d] with polish warps",
                                    d, maxb);
            if (P < 1 || P >= b / 32)
                return rd_set_error(RD_EINVAL, "tuning.polish_warps[%d] must be in [1, %d]", d, b / 32 - 1);
            if (tuning->lanes[d] == 2) return rd_set_error(RD_EINVAL, "tuning.polish_warps[%d] needs one lane", d);
            block[d] = b;
            pw[d] = P;
            continue;
        }
        if (tuning && d >= 1 && d <= 12) {
            if (tuning->block[d] != 0 && (tuning->block[d] < 32 || tuning->block[d] > 256 || tuning->block[d] % 32))
                return rd_set_error(RD_EINVAL, "tuning.block[%d] must be 0 or a multiple of 32 in [32, 256]", d);
            if (tuning->ctas_per_sm[d] < 0 || tuning->ctas_per_sm[d] > 64)
                return rd_set_error(RD_EINVAL, "tuning.ctas_per_sm[%d] must be in [0, 64]", d);
            if (tuning->lanes[d] < 0 || tuning->lanes[d] > 2)
                return rd_set_error(RD_EINVAL, "tuning.lanes[%d] must be 0, 1 or 2", d);
            if (tuning->lanes[d] == 2 && mode == RD_MIXED && p.polish_mode != RD_POLISH_FP64)
                return rd_set_error(RD_EINVAL, "tuning.lanes[%d] = 2 needs polish_mode RD_POLISH_FP64", d);
            if (tuning->block[d]) block[d] = tuning->block[d];
            if (tuning->ctas_per_sm[d]) cps[d] = tuning->ctas_per_sm[d];
            if (tuning->lanes[d]) lanes[d] = tuning->lanes[d];
        }
    }
    a.coeffs = coeffs;
    a.n = n;
    return rd::launch_uneven(a, dtype, degrees, offsets, n, n_coeffs, mode == RD_MIXED, ws, block, cps, lanes, pw,
                             fork, reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace rd

extern "C" {

int rd_roots_backward(const void *coeffs, rd_dtype dtype, int degree, int64_t n, const double *roots,
                      const double *grad_roots, void *grad_coeffs, uint8_t *status, void *stream)
{
    if (dtype != RD_C64 && dtype != RD_C128) return rd_set_error(RD_EINVAL, "dtype must be RD_C64 or RD_C128");
    if (degree < 1 || degree > 12) return rd_set_error(RD_EUNSUPPORTED, "degree %d outside 1..12", degree);
    if (n < 0) return rd_set_error(RD_EINVAL, "n < 0");
    if (n == 0) return RD_OK;
    size_t el = dtype == RD_C64 ? 8 : 16;
    if (!coeffs || !aligned(coeffs, el) || !grad_coeffs || !aligned(grad_coeffs, el))
        return rd_set_error(RD_EINVAL, "coeffs / grad_coeffs null or misaligned");
    if (!roots || !aligned(roots, 16) || !grad_roots || !aligned(grad_roots, 16))
        return rd_set_error(RD_EINVAL, "roots / grad_roots null or misaligned");
    return rd::launch_backward(degree, dtype, coeffs, roots, grad_roots, grad_coeffs, status, n,
                               reinterpret_cast<cudaStream_t>(stream));
}

int rd_roots_backward_uneven(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets,
                             int64_t n, int64_t n_coeffs, const double *roots, const double *grad_roots,
                             void *grad_coeffs, uint8_t *status, void *stream)
{
    if (dtype != RD_C64 && dtype != RD_C128) return rd_set_error(RD_EINVAL, "dtype must be RD_C64 or RD_C128");
    if (n < 0 || n_coeffs < 0) return rd_set_error(RD_EINVAL, "n and n_coeffs must be >= 0");
    if (n >= ((int64_t)1 << 32)) return rd_set_error(RD_EINVAL, "n must be below 2^32");
    if (n_coeffs > ((int64_t)1 << 40)) return rd_set_error(RD_EINVAL, "n_coeffs must be at most 2^40");
    if (n == 0) return RD_OK;
    size_t el = dtype == RD_C64 ? 8 : 16;
    if (!coeffs || !aligned(coeffs, el) || !grad_coeffs || !aligned(grad_coeffs, el))
        return rd_set_error(RD_EINVAL, "coeffs / grad_coeffs null or misaligned");
    if (!degrees || !offsets || !aligned(offsets, 8)) return rd_set_error(RD_EINVAL, "degrees / offsets null or misaligned");
    if (!roots || !aligned(roots, 16) || !grad_roots || !aligned(grad_roots, 16))
        return rd_set_error(RD_EINVAL, "roots / grad_roots null or misaligned");
    return rd::launch_backward_uneven(dtype, coeffs, degrees, offsets, n, n_coeffs, roots, grad_roots, grad_coeffs,
                                      status, reinterpret_cast<cudaStream_t>(stream));
}

int rd_l2_nodes(int nr, int nt, double *r, double *theta, double *w)
{
    if (nr < 1 || nr > 32) return rd_set_error(RD_EINVAL, "nr must be in 1..32");
    if (nt < 1 || nt > 4096) return rd_set_error(RD_EINVAL, "nt must be in 1..4096");
    if (!r || !w) return rd_set_error(RD_EINVAL, "r / w null");
    int rc = rd::l2_nodes_host(nr, r, w);
    if (rc) return rc;
    const double pi = 3.14159265358979323846;
    if (theta)
        for (int q = 0; q < nt; ++q) theta[q] = 2.0 * pi * q / nt;
    return RD_OK;
}

int rd_l2_approx(const double *samples, int64_t n, int nr, int nt, int degree, int precision, const double *centres,
                 double radius, double *coeffs, rd_clip *map, void *stream)
{
    if (precision != RD_L2_FP64 && precision != RD_L2_DF) return rd_set_error(RD_EINVAL, "precision must be RD_L2_FP64 or RD_L2_DF");
    if (nt != 32) return rd_set_error(RD_EUNSUPPORTED, "nt must be 32 (one angle per lane)");
    if (nr < 1 || nr > 32) return rd_set_error(RD_EINVAL, "nr must be in 1..32");
    if (degree < 0 || degree > 12) return rd_set_error(RD_EINVAL, "degree must be in 0..12");
    if (n < 0) return rd_set_error(RD_EINVAL, "n < 0");
    if (map) {
        if (!centres || !aligned(centres, 16)) return rd_set_error(RD_EINVAL, "centres null or misaligned (16 B)");
        if (!(radius > 0) || !std::isfinite(radius)) return rd_set_error(RD_EINVAL, "radius must be finite and > 0");
    }
    if (n > 0 && (!samples || !aligned(samples, 16) || !coeffs || !aligned(coeffs, 16)))
        return rd_set_error(RD_EINVAL, "samples / coeffs null or misaligned");
    if (n > 0) {
        int rc = rd::launch_l2(samples, n, nr, degree, coeffs, precision, reinterpret_cast<cudaStream_t>(stream));
        if (rc) return rc;
    }
    if (map) {
        map->centres = centres;
        map->radius = radius;
    }
    return RD_OK;
}

namespace {
int check_splat(const double *roots, int64_t n, const rd_window &window, int W, int H, double sigma, double scale,
                int precision)
{
    if (precision != RD_SPLAT_FP64 && precision != RD_SPLAT_FP32)
        return rd_set_error(RD_EINVAL, "precision must be RD_SPLAT_FP64 or RD_SPLAT_FP32");
    if (n < 0) return rd_set_error(RD_EINVAL, "n < 0");
    if (n > 0 && (!roots || !aligned(roots, 16))) return rd_set_error(RD_EINVAL, "roots null or misaligned (16 B)");
    if (!window_ok(window)) return rd_set_error(RD_EINVAL, "window must be finite with xmin < xmax, ymin < ymax");
    if (W < 1 || H < 1 || (int64_t)W * H > ((int64_t)1 << 31)) return rd_set_error(RD_EINVAL, "bad image size %d x %d", W, H);
    if (!(sigma > 0.0 && sigma <= 2.0)) return rd_set_error(RD_EINVAL, "sigma must be in (0, 2]");
    if (!(scale >= 0.0) || !std::isfinite(scale)) return rd_set_error(RD_EINVAL, "scale must be finite and >= 0");
    return RD_OK;
}
}  // namespace

int rd_splat(const double *roots, int64_t n, rd_window window, int W, int H, double sigma, double scale,
             int precision, double *img, void *stream)
{
    int rc = check_splat(roots, n, window, W, H, sigma, scale, precision);
    if (rc) return rc;
    if (!img || !aligned(img, 8)) return rd_set_error(RD_EINVAL, "img null or misaligned");
    if (n == 0) return RD_OK;
    return rd::launch_splat(roots, n, window, W, H, sigma, scale, precision, img,
                            reinterpret_cast<cudaStream_t>(stream));
}

int rd_splat_backward(const double *roots, int64_t n, rd_window window, int W, int H, double sigma, double scale,
                      int precision, const double *grad_img, double *grad_roots, void *stream)
{
    int rc = check_splat(roots, n, window, W, H, sigma, scale, precision);
    if (rc) return rc;
    if (!grad_img || !aligned(grad_img, 8)) return rd_set_error(RD_EINVAL, "grad_img null or misaligned");
    if (n > 0 && (!grad_roots || !aligned(grad_roots, 16)))
        return rd_set_error(RD_EINVAL, "grad_roots null or misaligned (16 B)");
    if (n == 0) return RD_OK;
    return rd::launch_splat_backward(roots, n, window, W, H, sigma, scale, precision, grad_img, grad_roots,
                                     reinterpret_cast<cudaStream_t>(stream));
}

int rd_field_density(rd_field f, const rd_field_spec *spec, rd_mode mode, const rd_params *params,
                     rd_window window, int W, int H, uint32_t *hist, double *coeffs, double *roots,
                     uint8_t *status, rd_stats *stats, void *stream)
{
    if (f != RD_F_SIN_CUBE && f != RD_F_POLY) return rd_set_error(RD_EINVAL, "f must be RD_F_SIN_CUBE or RD_F_POLY");
    if (!spec) return rd_set_error(RD_EINVAL, "spec is null");
    const rd_field_spec &sp = *spec;
    if (!window_ok(sp.tiles)) return rd_set_error(RD_EINVAL, "spec.tiles must be finite with xmin < xmax, ymin < ymax");
    if (sp.nx < 1 || sp.ny < 1 || (int64_t)sp.nx * sp.ny >= ((int64_t)1 << 31))
        return rd_set_error(RD_EINVAL, "spec.nx, spec.ny must be >= 1 with nx * ny < 2^31");
    if (sp.nr != 16) return rd_set_error(RD_EUNSUPPORTED, "spec.nr must be 16");
    if (sp.degree != 6) return rd_set_error(RD_EUNSUPPORTED, "spec.degree must be 6");
    if (sp.reserved != 0) return rd_set_error(RD_EINVAL, "spec.reserved must be 0");
    if (f == RD_F_POLY) {
        if (sp.poly_degree < 0 || sp.poly_degree > 12) return rd_set_error(RD_EINVAL, "spec.poly_degree must be in 0..12");
        for (int k = 0; k < 26; ++k)
            if (!std::isfinite(sp.poly[k])) return rd_set_error(RD_EINVAL, "spec.poly must be finite");
    }
    if (!std::isfinite(sp.radius)) return rd_set_error(RD_EINVAL, "spec.radius must be finite");
    const double tw = (sp.tiles.xmax - sp.tiles.xmin) / sp.nx, th = (sp.tiles.ymax - sp.tiles.ymin) / sp.ny;
    const double rho = sp.radius > 0 ? sp.radius : 0.5 * std::hypot(tw, th);
    if (!hist) return rd_set_error(RD_EINVAL, "hist is required");
    if (coeffs && !aligned(coeffs, 16)) return rd_set_error(RD_EINVAL, "coeffs misaligned (16 B)");
    rd::SolveArgs a;
    rd_params p;
    int rc = build_solve_args(RD_C128, sp.degree, mode, params, nullptr, &window, W, H, hist, roots, status, stats, a, p);
    if (rc) return rc;
    if (p.lanes == 2) return rd_set_error(RD_EINVAL, "params.lanes must be 0 or 1 here");
    if (p.polish_warps != 0) return rd_set_error(RD_EINVAL, "params.polish_warps must be 0 here");
    if (mode == RD_MIXED && p.polish_mode != RD_POLISH_FP64)
        return rd_set_error(RD_EINVAL, "params.polish_mode must be RD_POLISH_FP64 here");
    a.n = (int64_t)sp.nx * sp.ny;
    a.clip_on = 1;
    a.radius = rho;
    a.tiles = make_binner(sp.tiles, sp.nx, sp.ny);
    return rd::launch_field(a, sp, (int)f, rho, mode == RD_MIXED, coeffs, p.ctas_per_sm,
                            reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
