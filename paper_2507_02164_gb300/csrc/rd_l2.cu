// rd_l2.cu -- least-squares (L2) polynomial approximation on sub-disks.
//
// Paper: Tang & Quan, arXiv 2507.02164, Sec. II: the domain is split into
// small subregions and f is approximated on each by a polynomial g; Sec. II-A:
// with <g, h> = integral over the unit disk of g conj(h), the coefficients
// solve G a = b with G_jk = <z^j, z^k>, b_j = <f, z^j>. Taking the measure as
// area (dA = r dr dtheta), G is diagonal with G_jj = pi/(j+1), so
//   a_j = (j+1)/pi * <g, w^j>.
// Quadrature: Gauss-Legendre in r on [0,1] (nr nodes, the Jacobian r folded
// into the weights), the trapezoid rule in theta (nt = 32 equispaced angles,
// exact for trigonometric degree < 32). Per sub-disk:
//   <g, w^j> ~ sum_p w_p r_p^{j+1} (2 pi / nt) sum_q g(r_p e^{i theta_q}) e^{-i j theta_q}.
//
// Kernel: one warp per sub-disk, lane q owns angle theta_q; the radial sums
// u_j(q) = sum_p (w_p r_p^{j+1}) g_pq use real weights (2 FMA per term), then
// v_j = sum_q u_j(q) e^{-i j theta_q} is a warp reduce-scatter. The 512 samples of a
// sub-disk (8 KB) are read once, 32 consecutive doubles2 per load.
#include <cmath>

#include "rd_common.cuh"

namespace rd {

constexpr int L2_NT = 32;
constexpr int L2_MAX_NR = 32;
constexpr int L2_MAX_DEG = 12;

struct L2Tables {
    double wr[L2_MAX_NR][L2_MAX_DEG + 1];   // w_p r_p^{j+1} * (2 pi / nt) * (j+1) / pi
    double tw[L2_MAX_DEG + 1][L2_NT][2];    // e^{-i j theta_q}
};

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
static void legendre_pair(int n, double x, double &pn, double &pn1)
{
    double pm1 = 1.0, p = x;  // P_0, P_1
    if (n == 0) {
        pn = 1.0;
        pn1 = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        double next = ((2 * k - 1) * x * p - (k - 1) * pm1) / k;
        pm1 = p;
        p = next;
    }
    pn = p;
    pn1 = pm1;
}

// Gauss-Legendre on [0, 1]: nodes are the zeros of P_n mapped from [-1, 1],
// found by Newton's method from Tricomi's first-order estimate; the weights are
// 2 / ((1 - x^2) P_n'(x)^2) on [-1, 1], halved for [0, 1], with
// P_n'(x) = n (P_{n-1}(x) - x P_n(x)) / (1 - x^2).
int l2_nodes_host(int nr, double *r, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= nr; ++k) {
        double x = (1.0 - (nr - 1.0) / (8.0 * nr * nr * nr)) * std::cos(pi * (4.0 * k - 1.0) / (4.0 * nr + 2.0));
        for (int it = 0; it < 60; ++it) {
            double pn, pn1;
            legendre_pair(nr, x, pn, pn1);
            double dpn = nr * (pn1 - x * pn) / ((1.0 - x) * (1.0 + x));
            double dx = pn / dpn;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        double pn, pn1;
        legendre_pair(nr, x, pn, pn1);
        double omx2 = (1.0 - x) * (1.0 + x);
        double dpn = nr * (pn1 - x * pn) / omx2;
        double wt = 2.0 / (omx2 * dpn * dpn);
        // k = 1 is the largest node: fill from the top so r ascends
        r[nr - k] = 0.5 * (1.0 + x);
        w[nr - k] = 0.5 * wt;
    }
    return 0;
}

// Sum each of the V values of every lane over the warp (reduce-scatter).
// Level by level (offsets 16, 8, 4, 2) a lane keeps one half of its values,
// sends the other half to its partner and adds what it receives; the last
// level (offset 1) adds the partner's copy of the same value. Afterwards lane
// L holds the warp sum of value (L >> 1) & (V - 1); V = 16: 16 additions per
// lane instead of 5 V for V separate butterflies.
template <int V>
__device__ __forceinline__ double warp_reduce_scatter(double (&v)[V])
{
    const int lane = threadIdx.x & 31;
    static_assert(V == 16, "four halving levels");
#pragma unroll
    for (int lev = 0; lev < 4; ++lev) {
        const int o = 16 >> lev, half = V >> (lev + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            double send = upper ? v[i] : v[i + half];
            double keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// NR > 0, DEG >= 0: a build for that node count and degree; NR = 0, DEG = -1:
// runtime bounds (the same operations in the same order).
template <int NR, int DEG>
__global__ void __launch_bounds__(256) l2_kernel(const double2 *__restrict__ samples, int64_t n, int nr_arg,
                                                 int degree_arg, double2 *coeffs, const L2Tables T)
{
    constexpr int JMAX = DEG >= 0 ? DEG : L2_MAX_DEG;
    const int nr = NR > 0 ? NR : nr_arg;
    const int degree = DEG >= 0 ? DEG : degree_arg;
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    // this lane's twiddles, read once (lanes read different entries, which
    // the constant bank would serialise inside the loop)
    double twr[JMAX + 1], twi[JMAX + 1];
#pragma unroll
    for (int j = 0; j <= JMAX; ++j) {
        twr[j] = T.tw[j][lane][0];
        twi[j] = T.tw[j][lane][1];
    }
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n; s += warps_total) {
        const double2 *g = samples + s * (int64_t)nr * L2_NT;
        double ur[JMAX + 1], ui[JMAX + 1];
#pragma unroll
        for (int j = 0; j <= JMAX; ++j) ur[j] = ui[j] = 0.0;
#pragma unroll 4
        for (int p = 0; p < nr; ++p) {
            double2 v = __ldg(g + p * L2_NT + lane);
#pragma unroll
            for (int j = 0; j <= JMAX; ++j)
                if (j <= degree) {
                    ur[j] = fma(T.wr[p][j], v.x, ur[j]);
                    ui[j] = fma(T.wr[p][j], v.y, ui[j]);
                }
        }
        // angular sums v_j = sum_q u_j(q) e^{-i j theta_q}: this lane's term, then
        // warp sums, 8 coefficients (16 reals) per reduce-scatter pass
#pragma unroll
        for (int j0 = 0; j0 <= JMAX; j0 += 8) {
            if (j0 > degree) break;
            double val[16];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + jj;
                double vr = 0.0, vi = 0.0;
                if (j <= JMAX && j <= degree) {
                    vr = fma(ur[j], twr[j], -ui[j] * twi[j]);
                    vi = fma(ur[j], twi[j], ui[j] * twr[j]);
                }
                val[2 * jj] = vr;
                val[2 * jj + 1] = vi;
            }
            // lane 4 jj holds Re of coefficient j0 + jj, lane 4 jj + 2 its Im
            double sum = warp_reduce_scatter<16>(val);
            double im = __shfl_down_sync(0xffffffffu, sum, 2);
            const int jj = lane >> 2;
            if ((lane & 3) == 0 && j0 + jj <= degree) coeffs[(int64_t)(j0 + jj) * n + s] = make_double2(sum, im);
        }
    }
}

// ---- double-float variant on the FP32 pipe --------------------------------
// Same sums, each term a double-float (hi + lo floats): GB300 runs FP32 64x
// faster than FP64. Samples are first scaled by a power of two per sub-disk
// (the largest exponent of its 512 samples becomes 0; sin(z^3) reaches 1e41,
// beyond FP32) and split into hi + lo floats with integer operations, then
// the scale is applied back to the FP64 coefficients exactly.

// The radial weights are stored as (w, w) pairs: the real and imaginary
// parts of a sample go through the same operations with the same weight, as
// the two halves of packed FP32 instructions (FFMA2 / FMUL2 / FADD2, each
// half rounded as its scalar form), one issue slot for both.
struct L2TablesDF {
    float2 whi[L2_MAX_NR][L2_MAX_DEG + 1], wlo[L2_MAX_NR][L2_MAX_DEG + 1];
    float thi[L2_MAX_DEG + 1][L2_NT][2], tlo[L2_MAX_DEG + 1][L2_NT][2];
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&r);
}

// two_sum on both halves: s = a + b and its exact rounding error e
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// NR > 0, DEG >= 0: a build for that radial node count and degree (loops of
// fixed length, arrays of DEG + 1 coefficients); NR = 0, DEG = -1: the runtime
// nr and degree, with arrays for L2_MAX_DEG. Both do the same operations in
// the same order.
template <int NR, int DEG>
__global__ void __launch_bounds__(256, 2) l2_kernel_df(const double2 *__restrict__ samples, int64_t n, int nr_arg,
                                                    int degree_arg, double2 *coeffs, const L2TablesDF T)
{
    constexpr int JMAX = DEG >= 0 ? DEG : L2_MAX_DEG;
    const int nr = NR > 0 ? NR : nr_arg;
    const int degree = DEG >= 0 ? DEG : degree_arg;
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    dfl twr[JMAX + 1], twi[JMAX + 1];
#pragma unroll
    for (int j = 0; j <= JMAX; ++j) {
        twr[j] = {T.thi[j][lane][0], T.tlo[j][lane][0]};
        twi[j] = {T.thi[j][lane][1], T.tlo[j][lane][1]};
    }
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n; s += warps_total) {
        const double2 *g = samples + s * (int64_t)nr * L2_NT;
        // per sub-disk scale: the largest biased exponent of its samples
        unsigned emax = 0;
#pragma unroll(NR > 0 ? NR : 1)
        for (int p = 0; p < nr; ++p) {
            double2 v = __ldg(g + p * L2_NT + lane);
            unsigned ex = ((unsigned)__double2hiint(v.x) >> 20) & 0x7ffu;
            unsigned ey = ((unsigned)__double2hiint(v.y) >> 20) & 0x7ffu;
            emax = max(emax, max(ex, ey));
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        const int shift = (int)emax - 1023;
        // accumulators as (real, imaginary) pairs: ah[j] the high parts, al[j] the low
        float2 ah[JMAX + 1], al[JMAX + 1];
#pragma unroll
        for (int j = 0; j <= JMAX; ++j) ah[j] = al[j] = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int p = 0; p < nr; ++p) {
            double2 v = __ldg(g + p * L2_NT + lane);
            const dfl gx = split_scaled(v.x, shift), gy = split_scaled(v.y, shift);
            const float2 gh = make_float2(gx.hi, gy.hi), gl = make_float2(gx.lo, gy.lo);
#pragma unroll
            for (int j = 0; j <= JMAX; ++j)
                if (j <= degree) {
                    const float2 wh = T.whi[p][j], wl = T.wlo[p][j];
                    // exact product hi and its error, then TwoSum into the accumulator
                    const float2 ph = __fmul2_rn(wh, gh);
                    float2 pe = __ffma2_rn(wh, gh, make_float2(-ph.x, -ph.y));
                    pe = __ffma2_rn(wh, gl, pe);
                    pe = __ffma2_rn(wl, gh, pe);
                    float2 t, te;
                    two_sum2(ah[j], ph, t, te);
                    ah[j] = t;
                    al[j] = __fadd2_rn(al[j], __fadd2_rn(te, pe));
                }
        }
        dfl ur[JMAX + 1], ui[JMAX + 1];
#pragma unroll
        for (int j = 0; j <= JMAX; ++j) {
            ur[j] = {ah[j].x, al[j].x};
            ui[j] = {ah[j].y, al[j].y};
        }
#pragma unroll
        for (int j0 = 0; j0 <= JMAX; j0 += 8) {
            if (j0 > degree) break;
            dfl val[16];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + jj;
                dfl vr = {0.0f, 0.0f}, vi = {0.0f, 0.0f};
                if (j <= JMAX && j <= degree) {
                    dfl a = fast_two_sum(ur[j].hi, ur[j].lo), b = fast_two_sum(ui[j].hi, ui[j].lo);
                    vr = df_add(df_mul(a, twr[j]), df_neg(df_mul(b, twi[j])));
                    vi = df_add(df_mul(a, twi[j]), df_mul(b, twr[j]));
                }
                val[2 * jj] = vr;
                val[2 * jj + 1] = vi;
            }
            // double-float reduce-scatter (see warp_reduce_scatter)
#pragma unroll
            for (int lev = 0; lev < 4; ++lev) {
                const int o = 16 >> lev, half = 16 >> (lev + 1);
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    dfl send = upper ? val[i] : val[i + half];
                    dfl keep = upper ? val[i + half] : val[i];
                    dfl got = {__shfl_xor_sync(0xffffffffu, send.hi, o), __shfl_xor_sync(0xffffffffu, send.lo, o)};
                    val[i] = df_add(keep, got);
                }
            }
            dfl got = {__shfl_xor_sync(0xffffffffu, val[0].hi, 1), __shfl_xor_sync(0xffffffffu, val[0].lo, 1)};
            dfl sum = df_add(val[0], got);
            // back to FP64 and to the sub-disk's scale (a power of two: exact)
            double d = (f2d(sum.hi) + f2d(sum.lo)) * __longlong_as_double((long long)(shift + 1023) << 52);
            double im = __shfl_down_sync(0xffffffffu, d, 2);
            const int jj = lane >> 2;
            if ((lane & 3) == 0 && j0 + jj <= degree) coeffs[(int64_t)(j0 + jj) * n + s] = make_double2(d, im);
        }
    }
}

int launch_l2(const double *samples, int64_t n, int nr, int degree, double *coeffs, int precision,
              cudaStream_t st)
{
    if (precision == 1) {
        L2TablesDF T;
        double r[L2_MAX_NR], w[L2_MAX_NR];
        l2_nodes_host(nr, r, w);
        const double pi = 3.14159265358979323846;
        for (int p = 0; p < L2_MAX_NR; ++p)
            for (int j = 0; j <= L2_MAX_DEG; ++j) {
                double v = 0.0;
                if (p < nr && j <= degree) v = w[p] * std::pow(r[p], j + 1) * (2.0 * pi / L2_NT) * (j + 1) / pi;
                const float h = (float)v, l = (float)(v - (double)h);
                T.whi[p][j] = make_float2(h, h);
                T.wlo[p][j] = make_float2(l, l);
            }
        for (int j = 0; j <= L2_MAX_DEG; ++j)
            for (int q = 0; q < L2_NT; ++q) {
                int t = (j * q) % L2_NT;
                double ang = 2.0 * pi * t / L2_NT;
                double c = std::cos(ang), sn = -std::sin(ang);
                T.thi[j][q][0] = (float)c;
                T.tlo[j][q][0] = (float)(c - (double)T.thi[j][q][0]);
                T.thi[j][q][1] = (float)sn;
                T.tlo[j][q][1] = (float)(sn - (double)T.thi[j][q][1]);
            }
        const int block = 256;
        int64_t ctas = (n + 7) / 8;
        int64_t cap = (int64_t)rd_sm_count_cached() * 8;
        if (ctas > cap) ctas = cap;
        if (ctas < 1) ctas = 1;
        const double2 *sp = reinterpret_cast<const double2 *>(samples);
        double2 *cp = reinterpret_cast<double2 *>(coeffs);
        if (nr == 16 && degree == 6)  // the full pipeline's 16 x 32 nodes and degree-6 fits
            l2_kernel_df<16, 6><<<(unsigned)ctas, block, 0, st>>>(sp, n, nr, degree, cp, T);
        else
            l2_kernel_df<0, -1><<<(unsigned)ctas, block, 0, st>>>(sp, n, nr, degree, cp, T);
        return rd_check_launch("l2_kernel_df");
    }
    L2Tables T;
    double r[L2_MAX_NR], w[L2_MAX_NR];
    l2_nodes_host(nr, r, w);
    const double pi = 3.14159265358979323846;
    for (int p = 0; p < L2_MAX_NR; ++p)
        for (int j = 0; j <= L2_MAX_DEG; ++j) {
            double v = 0.0;
            if (p < nr && j <= degree) v = w[p] * std::pow(r[p], j + 1) * (2.0 * pi / L2_NT) * (j + 1) / pi;
            T.wr[p][j] = v;
        }
    for (int j = 0; j <= L2_MAX_DEG; ++j)
        for (int q = 0; q < L2_NT; ++q) {
            // e^{-i j theta_q}, theta_q = 2 pi q / nt, reduced exactly: (j q) mod nt
            int t = (j * q) % L2_NT;
            double ang = 2.0 * pi * t / L2_NT;
            T.tw[j][q][0] = std::cos(ang);
            T.tw[j][q][1] = -std::sin(ang);
        }
    const int block = 256;
    int64_t ctas = (n + 7) / 8;
    int64_t cap = (int64_t)rd_sm_count_cached() * 8;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    const double2 *sp = reinterpret_cast<const double2 *>(samples);
    double2 *cp = reinterpret_cast<double2 *>(coeffs);
    if (nr == 16 && degree == 6)
        l2_kernel<16, 6><<<(unsigned)ctas, block, 0, st>>>(sp, n, nr, degree, cp, T);
    else
        l2_kernel<0, -1><<<(unsigned)ctas, block, 0, st>>>(sp, n, nr, degree, cp, T);
    return rd_check_launch("l2_kernel");
}

}  // namespace rd
