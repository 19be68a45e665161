// rd_field.cu -- the whole method for an analytic f in one launch: samples
// of f at the quadrature nodes of every sub-disk, the L2 polynomial
// approximation, the roots, the tile clip and the histogram.
//
// Paper: Tang & Quan, arXiv 2507.02164. Sec. II: the region is covered by
// small disks D_i; on each, f is approximated by a polynomial g and the roots
// of g stand for the zeros of f in D_i. Sec. II-A: least squares on the disk,
// with the area measure G is diagonal and a_j = (j+1)/pi <g, w^j>, where
// g(w) = f(c + rho w) in the local variable w. Sec. II-B/II-C: roots by
// single-shift QR on the companion matrix.
//
// The split path (rd_l2_approx, then rd_roots_density with a clip) reads an
// array of 16 x 32 samples per sub-disk (1.06 GB for the 480 x 270 tiles)
// that the caller must have made. Here nothing but the histogram (and, if
// asked, coefficients, roots and status) touches memory:
//   * one warp takes 32 consecutive tiles; for each tile, lane q evaluates f
//     in FP64 at the 16 nodes r_p e^{i theta_q} of its angle and stages them
//     in shared memory; the radial sums are double-float sums on the FP32
//     pipe (the samples scaled by the tile's largest power of two, as in
//     l2_kernel_df), the angular sums a warp reduce-scatter; the 7
//     coefficients of the tile go to shared memory;
//   * after 32 tiles the same warp solves them, one lane per tile
//     (solve_warp: FP32 sweeps + FP64 polish, or FP64 sweeps), maps each root
//     to z = c + rho w, keeps it when it lies in the tile's own cell of the
//     grid and bins it.
// The FP64 pipe is the bound: the transcendental functions in f.
#include <cmath>
#include <cstring>

#include "rd_solve.cuh"

namespace rd {

int l2_nodes_host(int nr, double *r, double *w);

constexpr int FIELD_NR = 16;     // radial nodes
constexpr int FIELD_NT = 32;     // angles, one per lane
constexpr int FIELD_WARPS = 8;   // warps per CTA
constexpr int FIELD_MAX_POLY = 12;

template <int N>
struct FieldArgs {
    int func;         // rd_field
    int poly_degree;  // RD_F_POLY
    double poly[FIELD_MAX_POLY + 1][2];
    double xmin, ymax, tw, th;  // tile grid: top-left corner, tile width and height
    int nx, ny;
    double rho;                              // sub-disk radius
    double r[FIELD_NR];                      // Gauss-Legendre radii on [0, 1]
    double ct[FIELD_NT], st[FIELD_NT];       // cos, sin theta_q, theta_q = 2 pi q / 32
    float whi[FIELD_NR][N + 1], wlo[FIELD_NR][N + 1];      // w_p r_p^{j+1} (2 pi / 32) (j+1) / pi
    float thi[N + 1][FIELD_NT][2], tlo[N + 1][FIELD_NT][2];  // e^{-i j theta_q}
    double2 *coeffs;  // [N+1][nx*ny] (local variable w) or null
};

// f(z) for the built-in functions
template <int N>
__device__ __forceinline__ cx<double> field_eval(const FieldArgs<N> &F, cx<double> z)
{
    if (F.func == RD_F_SIN_CUBE) {
        // sin(x + iy) = sin x cosh y + i cos x sinh y, with cosh y and sinh y
        // from one exponential: (e^y +- e^-y) / 2. For small |y| the
        // difference loses relative accuracy in sinh y but not absolute
        // accuracy (about 1e-16), which is what the L2 fit of f needs.
        // z^3 = x (x^2 - 3 y^2) + i y (3 x^2 - y^2)
        const double x2 = z.re * z.re, y2 = z.im * z.im;
        const cx<double> z3 = {z.re * fma(-3.0, y2, x2), z.im * fma(3.0, x2, -y2)};
        double sa, ca;
        sincos(z3.re, &sa, &ca);
        const double e = exp(z3.im), ei = 1.0 / e;
        const double ch = 0.5 * (e + ei), sh = 0.5 * (e - ei);
        return {fma(sa, ch, 0.5 * z.re), fma(ca, sh, 0.5 * z.im)};
    }
    cx<double> p = {F.poly[F.poly_degree][0], F.poly[F.poly_degree][1]};
    for (int k = F.poly_degree - 1; k >= 0; --k) p = cfma(p, z, cx<double>{F.poly[k][0], F.poly[k][1]});
    return p;
}

// Tile t of the grid: centre (x0 + (ix + 1/2) w, y1 - (iy + 1/2) h), each
// product and sum rounded once (the values a host computes the same way).
struct TileMap {
    int64_t base;  // first tile of the warp's group
    int64_t ntiles;
    int nx;
    double xmin, ymax, tw, th;
    __device__ int64_t poly(int64_t i) const { return base + i; }
    __device__ int64_t root(int64_t p, int j) const { return (int64_t)j * ntiles + p; }
    __device__ cx<double> centre(const SolveArgs &, int64_t p) const
    {
        const int64_t iy = p / nx, ix = p - iy * nx;
        return {__dadd_rn(xmin, __dmul_rn((double)ix + 0.5, tw)), __dsub_rn(ymax, __dmul_rn((double)iy + 0.5, th))};
    }
    __device__ int64_t tile(const SolveArgs &, int64_t p) const { return p; }
};

// Dynamic shared memory of one CTA: twiddles, then per warp the coefficients
// of its 32 tiles and the samples of the tile in hand.
template <int N>
struct FieldSmem {
    static constexpr size_t tw_bytes = (size_t)(N + 1) * FIELD_NT * 4 * sizeof(float);
    static constexpr size_t node_bytes = (size_t)FIELD_NR * FIELD_NT * sizeof(double2);  // rho r_p e^{i theta_q}
    static constexpr size_t coef_per_warp = (size_t)(N + 1) * 32;      // double2
    static constexpr size_t samp_per_warp = (size_t)FIELD_NR * FIELD_NT;  // double2
    static constexpr size_t bytes =
        tw_bytes + node_bytes + FIELD_WARPS * (coef_per_warp + samp_per_warp) * sizeof(double2);
};

template <int N, int MODE>
__global__ void __launch_bounds__(FIELD_WARPS * 32, MODE != MODE_PLAIN ? 2 : 1)
    field_kernel(SolveArgs A, const __grid_constant__ FieldArgs<N> F)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long acc[ST_WORDS];
    using T = typename std::conditional<MODE != MODE_PLAIN, float, double>::type;
    using SM = FieldSmem<N>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float(*s_tw)[FIELD_NT][4] = reinterpret_cast<float(*)[FIELD_NT][4]>(smem);  // hi re, hi im, lo re, lo im
    double2 *s_node = reinterpret_cast<double2 *>(smem + SM::tw_bytes);        // [p][q]
    double2 *s_coef = reinterpret_cast<double2 *>(smem + SM::tw_bytes + SM::node_bytes) + wid * SM::coef_per_warp;
    double2 *s_samp = reinterpret_cast<double2 *>(smem + SM::tw_bytes + SM::node_bytes) +
                      FIELD_WARPS * SM::coef_per_warp + wid * SM::samp_per_warp;
    for (int i = threadIdx.x; i < (N + 1) * FIELD_NT; i += blockDim.x) {
        const int j = i / FIELD_NT, q = i % FIELD_NT;
        s_tw[j][q][0] = F.thi[j][q][0];
        s_tw[j][q][1] = F.thi[j][q][1];
        s_tw[j][q][2] = F.tlo[j][q][0];
        s_tw[j][q][3] = F.tlo[j][q][1];
    }
    // node offsets rho (r_p cos theta_q, r_p sin theta_q), once per CTA
    for (int i = threadIdx.x; i < FIELD_NR * FIELD_NT; i += blockDim.x) {
        const int p = i / FIELD_NT, q = i % FIELD_NT;
        s_node[i] = make_double2(__dmul_rn(F.rho, F.r[p] * F.ct[q]), __dmul_rn(F.rho, F.r[p] * F.st[q]));
    }
    const CtaStats S = stats_begin(acc, A.stats);  // its barrier (when stats are kept) publishes s_tw
    if (!A.stats) __syncthreads();
    const int64_t ntiles = (int64_t)F.nx * F.ny;
    const int64_t groups = (ntiles + 31) / 32;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; g < groups; g += warps_total) {
        const int64_t base = g * 32;
        const int count = (int)(ntiles - base < 32 ? ntiles - base : 32);
#pragma unroll 1
        for (int t = 0; t < count; ++t) {
            const int64_t tile = base + t;
            const int64_t iy = tile / F.nx, ix = tile - iy * F.nx;
            const double cxr = __dadd_rn(F.xmin, __dmul_rn((double)ix + 0.5, F.tw));
            const double cxi = __dsub_rn(F.ymax, __dmul_rn((double)iy + 0.5, F.th));
            // samples g(r_p e^{i theta_q}) = f(c + rho r_p e^{i theta_q}), this lane's angle
            unsigned emax = 0;
#pragma unroll 1
            for (int p = 0; p < FIELD_NR; ++p) {
                const double2 w = s_node[p * FIELD_NT + lane];
                const cx<double> z = {__dadd_rn(cxr, w.x), __dadd_rn(cxi, w.y)};
                const cx<double> v = field_eval(F, z);
                s_samp[p * FIELD_NT + lane] = make_double2(v.re, v.im);
                const unsigned ex = ((unsigned)__double2hiint(v.re) >> 20) & 0x7ffu;
                const unsigned ey = ((unsigned)__double2hiint(v.im) >> 20) & 0x7ffu;
                emax = max(emax, max(ex, ey));
            }
            emax = __reduce_max_sync(0xffffffffu, emax);
            const int shift = (int)emax - 1023;
            // radial sums u_j(q) = sum_p (w_p r_p^{j+1} ...) g_pq, double-float
            dfl ur[N + 1], ui[N + 1];
#pragma unroll
            for (int j = 0; j <= N; ++j) ur[j] = ui[j] = dfl{0.0f, 0.0f};
#pragma unroll 4
            for (int p = 0; p < FIELD_NR; ++p) {
                const double2 v = s_samp[p * FIELD_NT + lane];
                const dfl gx = split_scaled(v.x, shift), gy = split_scaled(v.y, shift);
#pragma unroll
                for (int j = 0; j <= N; ++j) {
                    const float wh = F.whi[p][j], wl = F.wlo[p][j];
                    float ph = __fmul_rn(wh, gx.hi);
                    float pe = __fmaf_rn(wh, gx.hi, -ph);
                    pe = __fmaf_rn(wh, gx.lo, pe);
                    pe = __fmaf_rn(wl, gx.hi, pe);
                    dfl s2 = two_sum(ur[j].hi, ph);
                    ur[j] = {s2.hi, __fadd_rn(ur[j].lo, __fadd_rn(s2.lo, pe))};
                    ph = __fmul_rn(wh, gy.hi);
                    pe = __fmaf_rn(wh, gy.hi, -ph);
                    pe = __fmaf_rn(wh, gy.lo, pe);
                    pe = __fmaf_rn(wl, gy.hi, pe);
                    s2 = two_sum(ui[j].hi, ph);
                    ui[j] = {s2.hi, __fadd_rn(ui[j].lo, __fadd_rn(s2.lo, pe))};
                }
            }
            // angular sums: this lane's term times e^{-i j theta_q}, then a
            // double-float reduce-scatter of the 2 (N+1) <= 16 values
            dfl val[16];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                dfl vr = {0.0f, 0.0f}, vi = {0.0f, 0.0f};
                if (jj <= N) {
                    const dfl twr = {s_tw[jj][lane][0], s_tw[jj][lane][2]};
                    const dfl twi = {s_tw[jj][lane][1], s_tw[jj][lane][3]};
                    const dfl a = fast_two_sum(ur[jj].hi, ur[jj].lo), b = fast_two_sum(ui[jj].hi, ui[jj].lo);
                    vr = df_add(df_mul(a, twr), df_neg(df_mul(b, twi)));
                    vi = df_add(df_mul(a, twi), df_mul(b, twr));
                }
                val[2 * jj] = vr;
                val[2 * jj + 1] = vi;
            }
#pragma unroll
            for (int lev = 0; lev < 4; ++lev) {
                const int o = 16 >> lev, half = 16 >> (lev + 1);
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const dfl send = upper ? val[i] : val[i + half];
                    const dfl keep = upper ? val[i + half] : val[i];
                    const dfl got = {__shfl_xor_sync(0xffffffffu, send.hi, o), __shfl_xor_sync(0xffffffffu, send.lo, o)};
                    val[i] = df_add(keep, got);
                }
            }
            const dfl got = {__shfl_xor_sync(0xffffffffu, val[0].hi, 1), __shfl_xor_sync(0xffffffffu, val[0].lo, 1)};
            const dfl sum = df_add(val[0], got);
            // lane 4 jj holds Re of coefficient jj, lane 4 jj + 2 its Im
            const double d = (f2d(sum.hi) + f2d(sum.lo)) * __longlong_as_double((long long)(shift + 1023) << 52);
            const double im = __shfl_down_sync(0xffffffffu, d, 2);
            const int jj = lane >> 2;
            if ((lane & 3) == 0 && jj <= N) {
                s_coef[jj * count + t] = make_double2(d, im);
                if (F.coeffs) F.coeffs[(int64_t)jj * ntiles + tile] = make_double2(d, im);
            }
        }
        __syncwarp();
        // the group's roots: lane i solves tile base + i (coefficient-major, stride count)
        const TileMap map{base, ntiles, F.nx, F.xmin, F.ymax, F.tw, F.th};
        solve_warp<N, T, SharedC128, MODE>(A, s_coef, count, 0, map, S);
        __syncwarp();
    }
    stats_end(S, A.stats);
}

// Host tables for degree N (the same quadrature as rd_l2_approx).
template <int N>
static void field_tables(FieldArgs<N> &F)
{
    double w[FIELD_NR];
    l2_nodes_host(FIELD_NR, F.r, w);
    const double pi = 3.14159265358979323846;
    for (int p = 0; p < FIELD_NR; ++p)
        for (int j = 0; j <= N; ++j) {
            const double v = w[p] * std::pow(F.r[p], j + 1) * (2.0 * pi / FIELD_NT) * (j + 1) / pi;
            F.whi[p][j] = (float)v;
            F.wlo[p][j] = (float)(v - (double)F.whi[p][j]);
        }
    for (int q = 0; q < FIELD_NT; ++q) {
        const double ang = 2.0 * pi * q / FIELD_NT;
        F.ct[q] = std::cos(ang);
        F.st[q] = std::sin(ang);
    }
    for (int j = 0; j <= N; ++j)
        for (int q = 0; q < FIELD_NT; ++q) {
            const int t = (j * q) % FIELD_NT;  // e^{-i j theta_q}, angle reduced exactly
            const double ang = 2.0 * pi * t / FIELD_NT;
            const double c = std::cos(ang), sn = -std::sin(ang);
            F.thi[j][q][0] = (float)c;
            F.tlo[j][q][0] = (float)(c - (double)F.thi[j][q][0]);
            F.thi[j][q][1] = (float)sn;
            F.tlo[j][q][1] = (float)(sn - (double)F.thi[j][q][1]);
        }
}

template <int N, int MODE>
static int launch_field_n(const SolveArgs &a, const rd_field_spec &spec, int func, double rho, double *coeffs,
                          int ctas_per_sm, cudaStream_t st)
{
    FieldArgs<N> F;
    std::memset(&F, 0, sizeof(F));
    F.func = func;
    F.poly_degree = spec.poly_degree;
    for (int k = 0; k <= FIELD_MAX_POLY; ++k) {
        F.poly[k][0] = spec.poly[2 * k];
        F.poly[k][1] = spec.poly[2 * k + 1];
    }
    F.nx = spec.nx;
    F.ny = spec.ny;
    F.xmin = spec.tiles.xmin;
    F.ymax = spec.tiles.ymax;
    F.tw = (spec.tiles.xmax - spec.tiles.xmin) / spec.nx;
    F.th = (spec.tiles.ymax - spec.tiles.ymin) / spec.ny;
    F.rho = rho;
    F.coeffs = reinterpret_cast<double2 *>(coeffs);
    field_tables<N>(F);
    auto kern = field_kernel<N, MODE>;
    const size_t smem = FieldSmem<N>::bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return rd_set_error(RD_ECUDA, "field_kernel shared memory: %s", cudaGetErrorString(e));
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FIELD_WARPS * 32, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int64_t groups = ((int64_t)spec.nx * spec.ny + 31) / 32;
    int64_t grid = (int64_t)per_sm * rd_sm_count_cached();
    const int64_t need = (groups + FIELD_WARPS - 1) / FIELD_WARPS;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, FIELD_WARPS * 32, smem, st>>>(a, F);
    return rd_check_launch("field_kernel");
}

int launch_field(const SolveArgs &a, const rd_field_spec &spec, int func, double rho, bool mixed, double *coeffs,
                 int ctas_per_sm, cudaStream_t st)
{
    if (spec.degree != 6) return rd_set_error(RD_EUNSUPPORTED, "field degree %d not built (6)", spec.degree);
    if (mixed) return launch_field_n<6, MODE_MIXED_FP64>(a, spec, func, rho, coeffs, ctas_per_sm, st);
    return launch_field_n<6, MODE_PLAIN>(a, spec, func, rho, coeffs, ctas_per_sm, st);
}

}  // namespace rd
