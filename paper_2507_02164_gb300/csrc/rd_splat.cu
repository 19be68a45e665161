// rd_splat.cu -- soft root density: the differentiable stand-in for the
// root-density histogram that the differentiation workload's loss uses (the
// paper bins hard counts, Sec. III; a loss needs an image that moves
// smoothly with the roots).
//
// Image: W x H pixel centres over the window, pixel (iy, ix) at
// x = xmin + (ix + 1/2) px, y = ymax - (iy + 1/2) py. A root at pixel
// coordinates u = (x - xmin)/px, v = (ymax - y)/py adds
//   w = max(0, exp(-(du^2 + dv^2) / (2 sigma^2)) - exp(-9/2)) * scale,
//   du = u - (ix + 1/2), dv = v - (iy + 1/2),
// which reaches 0 at 3 sigma: the pixels visited are those with centres
// within 3 sigma of the root in both axes, at most 13 x 13 for sigma <= 2.
//
// The Gaussian separates, exp(-(du^2 + dv^2)/(2 s^2)) = e(du) e(dv), and
// along one axis the 13 values e(du0 - k) follow from two exponentials by the
// ratio recurrence (fast Gaussian gridding, Greengard & Lee 2004):
//   e_{k+1} = e_k q_k,  q_k = exp((2 (du0 - k) - 1) / (2 s^2)),
//   q_{k+1} = q_k exp(-1 / s^2),
// about 13 ulp of rounding at the far end: 4 exponentials per root instead
// of 169.
//   * forward: one thread per root, FP64 atomic adds into the image (an
//     L2-resident 295 KB at 256 x 144); the order of the adds varies, so
//     the image is reproducible to rounding, not bit for bit;
//   * backward: one thread per root gathers dL/dimg over the same stencil:
//     dL/du = scale sum G dw/du with dw/du = -(du / s^2) e(du) e(dv) where
//     w > 0; dL/dx = (dL/du) / px, dL/dy = -(dL/dv) / py (PyTorch's
//     convention for a complex root: dL/dRe + i dL/dIm).
#include <atomic>
#include <cmath>

#include "rd_common.cuh"

namespace rd {

constexpr int SPLAT_K = 13;  // stencil width for sigma <= 2

struct SplatGeom {
    double xmin, ymax, px, py;
    double inv_px, inv_py;  // 1 / px, 1 / py: products instead of FP64 divisions per root
    int W, H;
    double sigma, inv_2s2, inv_s2, step, cut, scale, cut_s;  // cut_s = cut * scale
};

// First pixel index and the count along one axis, and the K Gaussian
// factors e(d0 - k), d0 = u - (i0 + 1/2). K = floor(6 sigma) + 1 covers the
// pixels within 3 sigma (a count above K, which only FP64 rounding of the box
// ends can give, adds a pixel whose weight is 0). Returns 0 when nothing is
// visited (non-finite coordinate or the box outside the image).
template <int K>
__device__ __forceinline__ int splat_axis(const SplatGeom &g, double u, int n_pix, int &i0, double (&e)[K],
                                          double &d0)
{
    if (!finite_bits(u)) return 0;
    double a = ceil(u - 0.5 - 3.0 * g.sigma), b = floor(u - 0.5 + 3.0 * g.sigma);
    a = fmax(a, 0.0);
    b = fmin(b, n_pix - 1.0);
    if (!(a <= b)) return 0;
    i0 = (int)a;
    const int cnt = (int)(b - a) + 1;
    d0 = u - (a + 0.5);
    double ek = exp(-d0 * d0 * g.inv_2s2);
    double q = exp((2.0 * d0 - 1.0) * g.inv_2s2);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        e[k] = ek;
        ek *= q;
        q *= g.step;
    }
    return cnt;
}

template <int K>
__global__ void __launch_bounds__(256) splat_kernel(const double2 *__restrict__ roots, int64_t n, SplatGeom g,
                                                    double *img)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        double ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis<K>(g, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis<K>(g, v, g.H, y0, ey, dy0) : 0;
        if (!ny) continue;
        // scale * (e(du) e(dv) - cut) = e(du) (scale e(dv)) - scale cut: one FMA
        // per pixel; w > 0 is read off the sign and magnitude bits (an
        // integer compare: FP64 compares issue to the FP64 pipe)
#pragma unroll
        for (int ky = 0; ky < K; ++ky) {
            if (ky >= ny) break;
            double *row = img + (size_t)(y0 + ky) * g.W + x0;
            const double eys = ey[ky] * g.scale;
#pragma unroll
            for (int kx = 0; kx < K; ++kx) {
                const double w = fma(ex[kx], eys, -g.cut_s);
                if (kx < nx && __double_as_longlong(w) > 0) atomicAdd(row + kx, w);
            }
        }
    }
}

template <int K>
__global__ void __launch_bounds__(256) splat_backward_kernel(const double2 *__restrict__ roots, int64_t n, SplatGeom g,
                                                             const double *__restrict__ G, double2 *grad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        double ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis<K>(g, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis<K>(g, v, g.H, y0, ey, dy0) : 0;
        double gu = 0.0, gv = 0.0;
        if (ny) {
            // the Gaussian separates: sum G e(du) e(dv) du over a row is
            // e(dv) sum G (e(du) du), so per pixel two FMAs on column factors
            // fixed per root, and e(du) e(dv) only for the cut test
            double edx[K];
#pragma unroll
            for (int kx = 0; kx < K; ++kx) edx[kx] = ex[kx] * (dx0 - kx);
            const long long cut_bits = __double_as_longlong(g.cut);
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                if (ky >= ny) break;
                const double *row = G + (size_t)(y0 + ky) * g.W + x0;
                double su = 0.0, sv = 0.0;
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const double e = ex[kx] * ey[ky];
                    // e > cut for positive doubles, on the bits (integer pipe)
                    if (kx < nx && __double_as_longlong(e) > cut_bits) {
                        const double gp = __ldg(row + kx);
                        su = fma(gp, edx[kx], su);
                        sv = fma(gp, ex[kx], sv);
                    }
                }
                gu = fma(ey[ky], su, gu);
                gv = fma(ey[ky] * (dy0 - ky), sv, gv);
            }
        }
        // dw/du = -(du / s^2) e, dw/dv = -(dv / s^2) e
        const double k = -g.scale * g.inv_s2;
        grad[j] = make_double2(k * gu * g.inv_px, -k * gv * g.inv_py);
    }
}

// ---- FP32 variant: the stencil arithmetic on the FP32 pipe -----------------
// The same stencil, recurrence and tests in float (about 1e-6 relative on
// the image and the gradient); the root's pixel coordinates u, v stay FP64
// (two FP64 operations per root), the image stays float64: weights are
// widened and the image gradient narrowed with integer bit operations (a
// conversion instruction would issue to the FP64 pipe again), and the atomic
// adds are FP64 additions in L2, not on the SM's FP64 pipe.
struct SplatGeomF {
    float sigma, inv_2s2, inv_s2, step, cut, scale, cut_s;
};

template <int K>
__device__ __forceinline__ int splat_axis_f(const SplatGeomF &g, double u, int n_pix, int &i0, float (&e)[K],
                                            float &d0)
{
    if (!finite_bits(u)) return 0;
    double a = ceil(u - 0.5 - 3.0 * (double)g.sigma), b = floor(u - 0.5 + 3.0 * (double)g.sigma);
    a = fmax(a, 0.0);
    b = fmin(b, n_pix - 1.0);
    if (!(a <= b)) return 0;
    i0 = (int)a;
    const int cnt = (int)(b - a) + 1;
    d0 = d2f(u - (a + 0.5));
    float ek = __expf(-d0 * d0 * g.inv_2s2);
    float q = __expf((2.0f * d0 - 1.0f) * g.inv_2s2);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        e[k] = ek;
        ek *= q;
        q *= g.step;
    }
    return cnt;
}

template <int K>
__global__ void __launch_bounds__(256) splat_kernel_f32(const double2 *__restrict__ roots, int64_t n, SplatGeom g,
                                                        SplatGeomF gf, double *img)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        float ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis_f<K>(gf, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis_f<K>(gf, v, g.H, y0, ey, dy0) : 0;
        if (!ny) continue;
#pragma unroll
        for (int ky = 0; ky < K; ++ky) {
            if (ky >= ny) break;
            double *row = img + (size_t)(y0 + ky) * g.W + x0;
            const float eys = ey[ky] * gf.scale;
#pragma unroll
            for (int kx = 0; kx < K; ++kx) {
                const float w = fmaf(ex[kx], eys, -gf.cut_s);
                if (kx < nx && __float_as_int(w) > 0) atomicAdd(row + kx, f2d(w));
            }
        }
    }
}

// The same FP32 forward with the image accumulated per CTA in shared memory
// (float, W x H <= SPLAT_SMEM_PIXELS): shared-memory atomic adds per root and
// pixel, then one FP64 global atomic add per touched pixel per CTA instead
// of one per root and pixel (at sigma 1.5 a root touches about 70 pixels).
// The partial sums stay within the FP32 variant's 1e-6.
constexpr int SPLAT_SMEM_PIXELS = 48 * 1024;  // 192 KB of floats

template <int K>
__global__ void __launch_bounds__(1024, 1) splat_kernel_f32_smem(const double2 *__restrict__ roots, int64_t n,
                                                                 SplatGeom g, SplatGeomF gf, double *img)
{
    extern __shared__ float s_img[];
    const int npix = g.W * g.H;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) s_img[p] = 0.0f;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        float ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis_f<K>(gf, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis_f<K>(gf, v, g.H, y0, ey, dy0) : 0;
        if (!ny) continue;
#pragma unroll
        for (int ky = 0; ky < K; ++ky) {
            if (ky >= ny) break;
            float *row = s_img + (y0 + ky) * g.W + x0;
            const float eys = ey[ky] * gf.scale;
#pragma unroll
            for (int kx = 0; kx < K; ++kx) {
                const float w = fmaf(ex[kx], eys, -gf.cut_s);
                if (kx < nx && __float_as_int(w) > 0) atomicAdd(row + kx, w);
            }
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < npix; p += blockDim.x) {
        const float w = s_img[p];
        if (w != 0.0f) atomicAdd(img + p, f2d(w));
    }
}

template <int K>
__global__ void __launch_bounds__(256) splat_backward_kernel_f32(const double2 *__restrict__ roots, int64_t n,
                                                                 SplatGeom g, SplatGeomF gf,
                                                                 const double *__restrict__ G, double2 *grad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        float ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis_f<K>(gf, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis_f<K>(gf, v, g.H, y0, ey, dy0) : 0;
        float gu = 0.0f, gv = 0.0f;
        if (ny) {
            const int cut_bits = __float_as_int(gf.cut);
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                if (ky >= ny) break;
                const double *row = G + (size_t)(y0 + ky) * g.W + x0;
                float su = 0.0f, sv = 0.0f;
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const float e = ex[kx] * ey[ky];
                    if (kx < nx && __float_as_int(e) > cut_bits) {
                        const float ge = d2f(__ldg(row + kx)) * e;
                        su = fmaf(ge, dx0 - (float)kx, su);
                        sv += ge;
                    }
                }
                gu += su;
                gv = fmaf(sv, dy0 - (float)ky, gv);
            }
        }
        const float k = -gf.scale * gf.inv_s2;
        grad[j] = make_double2(f2d(k * gu) * g.inv_px, -f2d(k * gv) * g.inv_py);
    }
}

// The same FP32 pull-back with dL/dimg staged once per CTA in shared memory
// as float (W x H <= SPLAT_SMEM_PIXELS): the stencil then reads floats from
// shared memory instead of converting an FP64 global value per pixel.
template <int K>
__global__ void __launch_bounds__(1024, 1) splat_backward_kernel_f32_smem(const double2 *__restrict__ roots,
                                                                          int64_t n, SplatGeom g, SplatGeomF gf,
                                                                          const double *__restrict__ G, double2 *grad)
{
    extern __shared__ float s_g[];
    const int npix = g.W * g.H;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) s_g[p] = d2f(__ldg(G + p));
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double2 z = __ldg(roots + j);
        const double u = (z.x - g.xmin) * g.inv_px, v = (g.ymax - z.y) * g.inv_py;
        float ex[K], ey[K], dx0, dy0;
        int x0, y0;
        const int nx = splat_axis_f<K>(gf, u, g.W, x0, ex, dx0);
        const int ny = nx ? splat_axis_f<K>(gf, v, g.H, y0, ey, dy0) : 0;
        float gu = 0.0f, gv = 0.0f;
        if (ny) {
            const int cut_bits = __float_as_int(gf.cut);
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                if (ky >= ny) break;
                const float *row = s_g + (y0 + ky) * g.W + x0;
                float su = 0.0f, sv = 0.0f;
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const float e = ex[kx] * ey[ky];
                    if (kx < nx && __float_as_int(e) > cut_bits) {
                        const float ge = row[kx] * e;
                        su = fmaf(ge, dx0 - (float)kx, su);
                        sv += ge;
                    }
                }
                gu += su;
                gv = fmaf(sv, dy0 - (float)ky, gv);
            }
        }
        const float k = -gf.scale * gf.inv_s2;
        grad[j] = make_double2(f2d(k * gu) * g.inv_px, -f2d(k * gv) * g.inv_py);
    }
}

static SplatGeom splat_geom(const rd_window &w, int W, int H, double sigma, double scale)
{
    SplatGeom g;
    g.xmin = w.xmin;
    g.ymax = w.ymax;
    g.px = (w.xmax - w.xmin) / W;
    g.py = (w.ymax - w.ymin) / H;
    g.inv_px = 1.0 / g.px;
    g.inv_py = 1.0 / g.py;
    g.W = W;
    g.H = H;
    g.sigma = sigma;
    g.inv_2s2 = 1.0 / (2.0 * sigma * sigma);
    g.inv_s2 = 1.0 / (sigma * sigma);
    g.step = std::exp(-1.0 / (sigma * sigma));
    g.cut = std::exp(-4.5);
    g.scale = scale;
    g.cut_s = g.cut * scale;
    return g;
}

static unsigned splat_grid(int64_t n)
{
    int64_t ctas = (n + 255) / 256;
    const int64_t cap = (int64_t)rd_sm_count_cached() * 8;
    if (ctas > cap) ctas = cap;
    return (unsigned)(ctas < 1 ? 1 : ctas);
}

static SplatGeomF splat_geom_f(const SplatGeom &g)
{
    SplatGeomF f;
    f.sigma = (float)g.sigma;
    f.inv_2s2 = (float)g.inv_2s2;
    f.inv_s2 = (float)g.inv_s2;
    f.step = (float)g.step;
    f.cut = (float)g.cut;
    f.scale = (float)g.scale;
    f.cut_s = (float)g.cut_s;
    return f;
}

// Stencil width built for sigma: floor(6 sigma) + 1 pixels per axis, rounded
// up to a built width (sigma in (0, 2]: at most 13).
static int splat_width(double sigma)
{
    const int k = (int)std::floor(6.0 * sigma) + 1;
    return k <= 4 ? 4 : (k <= 7 ? 7 : (k <= 10 ? 10 : SPLAT_K));
}

// Shared memory above 48 KB for the *_f32_smem kernels: opted in per
// device, kernel and width, once, to the largest size asked for.
template <typename Kern>
static int splat_allow_smem(Kern kern, int slot, size_t bytes)
{
    static std::atomic<size_t> allowed[64][8];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return rd_check_launch("cudaGetDevice");
    if (dev < 0 || dev >= 64) return rd_set_error(RD_EUNSUPPORTED, "device %d: at most 64 devices", dev);
    if (bytes <= 48 * 1024 || bytes <= allowed[dev][slot].load()) return RD_OK;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return rd_check_launch("cudaFuncSetAttribute(splat smem kernel)");
    size_t cur = allowed[dev][slot].load();
    while (cur < bytes && !allowed[dev][slot].compare_exchange_weak(cur, bytes)) {
    }
    return RD_OK;
}

static int splat_slot(int K) { return K == 4 ? 0 : (K == 7 ? 1 : (K == 10 ? 2 : 3)); }

// One CTA of 1024 threads per SM at most (the shared image).
static unsigned splat_smem_grid(int64_t n)
{
    int64_t ctas = (n + 1023) / 1024;
    const int64_t cap = rd_sm_count_cached();
    if (ctas > cap) ctas = cap;
    return (unsigned)(ctas < 1 ? 1 : ctas);
}

int launch_splat(const double *roots, int64_t n, const rd_window &w, int W, int H, double sigma, double scale,
                 int precision, double *img, cudaStream_t st)
{
    const SplatGeom g = splat_geom(w, W, H, sigma, scale);
    const int K = splat_width(sigma);
    auto z = reinterpret_cast<const double2 *>(roots);
    if (precision == RD_SPLAT_FP32) {
        if ((int64_t)W * H <= SPLAT_SMEM_PIXELS) {
            const size_t smem = (size_t)W * H * sizeof(float);
#define RD_SPLAT_S(KK)                                                                                  \
    if (K == KK) {                                                                                      \
        int rc = splat_allow_smem(splat_kernel_f32_smem<KK>, splat_slot(KK), smem);                     \
        if (rc) return rc;                                                                              \
        splat_kernel_f32_smem<KK><<<splat_smem_grid(n), 1024, smem, st>>>(z, n, g, splat_geom_f(g), img); \
    }
            RD_SPLAT_S(4) RD_SPLAT_S(7) RD_SPLAT_S(10) RD_SPLAT_S(13)
#undef RD_SPLAT_S
            return rd_check_launch("splat_kernel_f32_smem");
        }
#define RD_SPLAT_F(KK) \
    if (K == KK) splat_kernel_f32<KK><<<splat_grid(n), 256, 0, st>>>(z, n, g, splat_geom_f(g), img);
        RD_SPLAT_F(4) RD_SPLAT_F(7) RD_SPLAT_F(10) RD_SPLAT_F(13)
#undef RD_SPLAT_F
        return rd_check_launch("splat_kernel_f32");
    }
#define RD_SPLAT_D(KK) \
    if (K == KK) splat_kernel<KK><<<splat_grid(n), 256, 0, st>>>(z, n, g, img);
    RD_SPLAT_D(4) RD_SPLAT_D(7) RD_SPLAT_D(10) RD_SPLAT_D(13)
#undef RD_SPLAT_D
    return rd_check_launch("splat_kernel");
}

int launch_splat_backward(const double *roots, int64_t n, const rd_window &w, int W, int H, double sigma,
                          double scale, int precision, const double *G, double *grad, cudaStream_t st)
{
    const SplatGeom g = splat_geom(w, W, H, sigma, scale);
    const int K = splat_width(sigma);
    auto z = reinterpret_cast<const double2 *>(roots);
    auto gr = reinterpret_cast<double2 *>(grad);
    if (precision == RD_SPLAT_FP32) {
        if ((int64_t)W * H <= SPLAT_SMEM_PIXELS) {
            const size_t smem = (size_t)W * H * sizeof(float);
#define RD_SPLAT_BS(KK)                                                                                       \
    if (K == KK) {                                                                                            \
        int rc = splat_allow_smem(splat_backward_kernel_f32_smem<KK>, 4 + splat_slot(KK), smem);              \
        if (rc) return rc;                                                                                    \
        splat_backward_kernel_f32_smem<KK><<<splat_smem_grid(n), 1024, smem, st>>>(z, n, g, splat_geom_f(g), G, gr); \
    }
            RD_SPLAT_BS(4) RD_SPLAT_BS(7) RD_SPLAT_BS(10) RD_SPLAT_BS(13)
#undef RD_SPLAT_BS
            return rd_check_launch("splat_backward_kernel_f32_smem");
        }
#define RD_SPLAT_BF(KK) \
    if (K == KK) splat_backward_kernel_f32<KK><<<splat_grid(n), 256, 0, st>>>(z, n, g, splat_geom_f(g), G, gr);
        RD_SPLAT_BF(4) RD_SPLAT_BF(7) RD_SPLAT_BF(10) RD_SPLAT_BF(13)
#undef RD_SPLAT_BF
        return rd_check_launch("splat_backward_kernel_f32");
    }
#define RD_SPLAT_BD(KK) \
    if (K == KK) splat_backward_kernel<KK><<<splat_grid(n), 256, 0, st>>>(z, n, g, G, gr);
    RD_SPLAT_BD(4) RD_SPLAT_BD(7) RD_SPLAT_BD(10) RD_SPLAT_BD(13)
#undef RD_SPLAT_BD
    return rd_check_launch("splat_backward_kernel");
}

}  // namespace rd
