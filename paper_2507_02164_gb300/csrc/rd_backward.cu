// rd_backward.cu -- adjoint of the roots with respect to the coefficients.
//
// p(z(a), a) = 0 with p(z) = sum_k a_k z^k gives p'(z) dz + sum_k z^k da_k = 0,
// so dz_j/da_k = -z_j^k / p'(z_j): the gradient needs only the roots, not the
// QR sweeps that produced them. For a real loss and PyTorch's convention
// (grad = dL/dRe + i dL/dIm), a holomorphic map pulls gradients back through
// the conjugate derivative:
//   grad_a_k = sum_j conj(-z_j^k / p'(z_j)) grad_z_j
//            = sum_j conj(z_j)^k u_j,    u_j = conj(-1 / p'(z_j)) grad_z_j.
#include "rd_common.cuh"

namespace rd {

template <typename T>
struct CLoad;
template <>
struct CLoad<float> {
    using V = float2;
};
template <>
struct CLoad<double> {
    using V = double2;
};

template <int N, typename T>
__global__ void __launch_bounds__(256) backward_kernel(const void *coeffs, const double2 *__restrict__ roots,
                                                       const double2 *__restrict__ grad_roots, void *grad_coeffs,
                                                       uint8_t *status, int64_t n)
{
    using V = typename CLoad<T>::V;
    const V *A = reinterpret_cast<const V *>(coeffs);
    V *G = reinterpret_cast<V *>(grad_coeffs);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T tiny = sizeof(T) == 8 ? (T)1e-300 : (T)0;  // |p'| at or below this is singular
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        cx<T> a[N + 1];
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            V v = A[(int64_t)k * n + i];
            a[k] = {v.x, v.y};
        }
        cx<T> g[N + 1];
#pragma unroll
        for (int k = 0; k <= N; ++k) g[k] = {T(0), T(0)};
        bool singular = false;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double2 zr = roots[(int64_t)j * n + i];
            double2 gr = grad_roots[(int64_t)j * n + i];
            cx<T> z = {(T)zr.x, (T)zr.y};
            cx<T> gz = {(T)gr.x, (T)gr.y};
            // p'(z) by Horner
            cx<T> dp = scale((T)N, a[N]);
#pragma unroll
            for (int k = N - 1; k >= 1; --k) dp = cfma(dp, z, scale((T)k, a[k]));
            // singular: |p'(z)| <= 1e-300 (0 in FP32) or anything non-finite. The
            // larger component m decides almost always (|p'| > tiny when m > tiny,
            // |p'| <= tiny when m <= tiny / sqrt 2); hypot only in between.
            const T m = fmax(fabs(dp.re), fabs(dp.im));
            bool big = m > tiny;
            if (!big && m > tiny * (T)0.70710678118654752) big = hypot(dp.re, dp.im) > tiny;
            bool bad = !(isfinite(dp.re) && isfinite(dp.im) && isfinite(z.re) && isfinite(z.im)) || !big;
            singular |= bad;
            if (bad) continue;
            // u = conj(-1/dp) * gz = -(dp / |dp|^2) * gz
            cx<T> inv = cdiv(cx<T>{T(1), T(0)}, dp);
            cx<T> u = mul(cx<T>{-inv.re, inv.im}, gz);
            cx<T> zc = {z.re, -z.im};
            cx<T> pw = {T(1), T(0)};
#pragma unroll
            for (int k = 0; k <= N; ++k) {
                g[k] = cfma(pw, u, g[k]);
                pw = mul(pw, zc);
            }
        }
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            V v;
            v.x = g[k].re;
            v.y = g[k].im;
            G[(int64_t)k * n + i] = v;
        }
        if (status) status[i] = singular ? RD_STATUS_REJECTED : RD_STATUS_OK;
    }
}

template <typename T>
static int launch_bw(int degree, const void *coeffs, const double *roots, const double *grad_roots,
                     void *grad_coeffs, uint8_t *status, int64_t n, cudaStream_t st)
{
    const int block = 128;
    int64_t ctas = (n + block - 1) / block;
    int64_t cap = (int64_t)rd_sm_count_cached() * 16;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    auto R = reinterpret_cast<const double2 *>(roots);
    auto GR = reinterpret_cast<const double2 *>(grad_roots);
#define RD_BW_CASE(D) \
    case D: backward_kernel<D, T><<<(unsigned)ctas, block, 0, st>>>(coeffs, R, GR, grad_coeffs, status, n); break;
    switch (degree) {
        RD_BW_CASE(1) RD_BW_CASE(2) RD_BW_CASE(3) RD_BW_CASE(4) RD_BW_CASE(5) RD_BW_CASE(6)
        RD_BW_CASE(7) RD_BW_CASE(8) RD_BW_CASE(9) RD_BW_CASE(10) RD_BW_CASE(11) RD_BW_CASE(12)
    default: return rd_set_error(RD_EUNSUPPORTED, "roots_backward: degree %d not built", degree);
    }
#undef RD_BW_CASE
    return rd_check_launch("backward_kernel");
}

// Packed batch of uneven degrees (the layout of rd_roots_uneven): one thread
// per polynomial with its degree d (1..12) a runtime value. The coefficient
// and gradient arrays are sized for degree 12 and indexed only by unrolled
// constants under k <= d predicates, so they stay in registers; the
// arithmetic is the uniform kernel's operation for operation (p'(z) starts
// from 0 z + d a_d = d a_d exactly), so a batch of one degree gives the same
// bits either way. A polynomial is differentiated under rd_roots_uneven's
// consistency rule, which keeps every read and write inside the arrays.
template <typename T>
__global__ void __launch_bounds__(128) backward_uneven_kernel(const void *coeffs, const uint8_t *__restrict__ degrees,
                                                              const int64_t *__restrict__ offsets, int64_t n,
                                                              int64_t n_coeffs, const double2 *__restrict__ roots,
                                                              const double2 *__restrict__ grad_roots,
                                                              void *grad_coeffs, uint8_t *status)
{
    constexpr int NMAX = 12;
    using V = typename CLoad<T>::V;
    const V *A = reinterpret_cast<const V *>(coeffs);
    V *G = reinterpret_cast<V *>(grad_coeffs);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T tiny = sizeof(T) == 8 ? (T)1e-300 : (T)0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int d = __ldg(degrees + i);
        const int64_t o0 = __ldg(offsets + i), o1 = __ldg(offsets + i + 1);
        const bool consistent = (o0 >= i) && (o1 >= o0) && (o1 <= n_coeffs - (n - 1 - i)) && (o1 - o0 == (int64_t)d + 1);
        if (!consistent) {
            if (status) status[i] = RD_STATUS_DEGENERATE;
            continue;
        }
        if (d < 1 || d > NMAX) {
            for (int k = 0; k <= d; ++k) G[o0 + k] = V{T(0), T(0)};
            if (status) status[i] = RD_STATUS_DEGENERATE;
            continue;
        }
        cx<T> a[NMAX + 1], g[NMAX + 1];
#pragma unroll
        for (int k = 0; k <= NMAX; ++k) {
            V v = k <= d ? A[o0 + k] : V{T(0), T(0)};
            a[k] = {v.x, v.y};
            g[k] = {T(0), T(0)};
        }
        const int64_t r0 = o0 - i;
        bool singular = false;
        for (int j = 0; j < d; ++j) {
            double2 zr = roots[r0 + j];
            double2 gr = grad_roots[r0 + j];
            cx<T> z = {(T)zr.x, (T)zr.y};
            cx<T> gz = {(T)gr.x, (T)gr.y};
            cx<T> dp = {T(0), T(0)};
#pragma unroll
            for (int k = NMAX; k >= 1; --k)
                if (k <= d) dp = cfma(dp, z, scale((T)k, a[k]));
            const T m = fmax(fabs(dp.re), fabs(dp.im));
            bool big = m > tiny;
            if (!big && m > tiny * (T)0.70710678118654752) big = hypot(dp.re, dp.im) > tiny;
            bool bad = !(isfinite(dp.re) && isfinite(dp.im) && isfinite(z.re) && isfinite(z.im)) || !big;
            singular |= bad;
            if (bad) continue;
            cx<T> inv = cdiv(cx<T>{T(1), T(0)}, dp);
            cx<T> u = mul(cx<T>{-inv.re, inv.im}, gz);
            cx<T> zc = {z.re, -z.im};
            cx<T> pw = {T(1), T(0)};
#pragma unroll
            for (int k = 0; k <= NMAX; ++k)
                if (k <= d) {
                    g[k] = cfma(pw, u, g[k]);
                    pw = mul(pw, zc);
                }
        }
#pragma unroll
        for (int k = 0; k <= NMAX; ++k)
            if (k <= d) {
                V v;
                v.x = g[k].re;
                v.y = g[k].im;
                G[o0 + k] = v;
            }
        if (status) status[i] = singular ? RD_STATUS_REJECTED : RD_STATUS_OK;
    }
}

int launch_backward_uneven(rd_dtype dt, const void *coeffs, const uint8_t *degrees, const int64_t *offsets,
                           int64_t n, int64_t n_coeffs, const double *roots, const double *grad_roots,
                           void *grad_coeffs, uint8_t *status, cudaStream_t st)
{
    const int block = 128;
    int64_t ctas = (n + block - 1) / block;
    int64_t cap = (int64_t)rd_sm_count_cached() * 16;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    auto R = reinterpret_cast<const double2 *>(roots);
    auto GR = reinterpret_cast<const double2 *>(grad_roots);
    if (dt == RD_C64)
        backward_uneven_kernel<float><<<(unsigned)ctas, block, 0, st>>>(coeffs, degrees, offsets, n, n_coeffs, R, GR,
                                                                         grad_coeffs, status);
    else
        backward_uneven_kernel<double><<<(unsigned)ctas, block, 0, st>>>(coeffs, degrees, offsets, n, n_coeffs, R, GR,
                                                                          grad_coeffs, status);
    return rd_check_launch("backward_uneven_kernel");
}

int launch_backward(int degree, rd_dtype dt, const void *coeffs, const double *roots, const double *grad_roots,
                    void *grad_coeffs, uint8_t *status, int64_t n, cudaStream_t st)
{
    if (dt == RD_C64) return launch_bw<float>(degree, coeffs, roots, grad_roots, grad_coeffs, status, n, st);
    return launch_bw<double>(degree, coeffs, roots, grad_roots, grad_coeffs, status, n, st);
}

}  // namespace rd
