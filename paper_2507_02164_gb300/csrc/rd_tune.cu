// rd_tune.cu -- the launch-shape autotuner (rd_autotune) and the ALU
// throughput probe (rd_alu_peak) of libroots.
//
// Neither is part of the paper's method. The autotuner picks, per degree,
// the launch shape of the solve kernels (lanes per polynomial, threads per
// CTA, resident CTAs per SM, and for the mixed mode the split of each CTA
// into sweep and polish warps) by timing every candidate on a probe batch;
// the probe measures what the roofline divides by: the throughput of
// independent FFMA / DFMA chains on this GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rd_common.cuh"

namespace rd {

// ---- probe batch -----------------------------------------------------------
// Complex-Gaussian coefficients (real and imaginary parts N(0,1)), drawn from
// SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator,
// and the Box-Muller transform. Coefficient-major [degree + 1][n].

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ double unit_open(uint64_t bits)  // (0, 1)
{
    return ((double)(bits >> 11) + 0.5) * 0x1p-53;
}

template <typename V>
__global__ void __launch_bounds__(256) probe_kernel(V *out, int64_t count, uint64_t seed)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride) {
        const uint64_t key = splitmix64(seed) ^ ((uint64_t)e * 0xD1B54A32D192ED03ull);
        const double u1 = unit_open(splitmix64(key)), u2 = unit_open(splitmix64(key + 1));
        const double r = sqrt(-2.0 * log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        V v;
        v.x = r * c;
        v.y = r * s;
        out[e] = v;
    }
}

// ---- ALU throughput probe ------------------------------------------------------
// Eight independent FMA chains per thread, 16 steps unrolled per iteration.
// FP64: DFMA, 128 FMAs per iteration. FP32: each chain is a pair of floats
// stepped by one packed fma.rn.f32x2 (two FMAs per instruction, so the loop
// and issue overhead cannot hide the FMA pipe's limit), 256 FMAs per
// iteration. b and c are kernel arguments, so nothing folds; the sink is
// written only if the sum hits a value the chains never reach, so the chains
// stay live.
constexpr int PEAK_STEPS = 16;
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(256) alu_peak_f64_kernel(int iters, double b, double c, double never,
                                                           double *sink)
{
    double a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < PEAK_STEPS; ++s)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) sum += a[k];
    if (sum == never) *sink = sum;
}

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack_f32x2(float x, float y)
{
    return ((unsigned long long)__float_as_uint(y) << 32) | __float_as_uint(x);
}

__global__ void __launch_bounds__(256) alu_peak_f32_kernel(int iters, float b, float c, float never, double *sink)
{
    unsigned long long a[PEAK_CHAINS];
    const unsigned long long B = pack_f32x2(b, b), C = pack_f32x2(c, c);
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = pack_f32x2((threadIdx.x + 2 * k) * 1e-3f, (threadIdx.x + 2 * k + 1) * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < PEAK_STEPS; ++s)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma_f32x2(a[k], B, C);
    }
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k)
        sum += __uint_as_float((unsigned)a[k]) + __uint_as_float((unsigned)(a[k] >> 32));
    if (sum == never) *sink = (double)sum;
}

}  // namespace rd

namespace {

struct Shape {
    int lanes, block, cps, pw;
};

// The candidates: one-role shapes (lanes 1, and 2 from degree 2; 32..256
// threads; the occupancy maximum or fewer CTAs per SM), then for RD_MIXED the
// warp-specialised shapes: up to 16 warps per CTA at degrees <= 6 (about 128
// registers), up to 8 above (255). A polish warp keeps about one FP64
// instruction in flight, so the FP64 pipe wants about ten polish warps per SM.
std::vector<Shape> candidates(int degree, rd_mode mode, int polish_mode)
{
    std::vector<Shape> v;
    const int blocks[4] = {32, 64, 128, 256};
    // two lanes per polynomial only with the FP64 polish (or no polish: plain)
    const int max_lanes = (degree >= 2 && (mode == RD_PLAIN_FP64 || polish_mode == RD_POLISH_FP64)) ? 2 : 1;
    for (int lanes = 1; lanes <= max_lanes; ++lanes)
        for (int b : blocks) {
            const int cps_big[3] = {0, 1, 2}, cps_small[3] = {0, 2, 4};
            const int *cps = b >= 128 ? cps_big : cps_small;
            for (int k = 0; k < 3; ++k) v.push_back({lanes, b, cps[k], 0});
        }
    if (mode == RD_MIXED) {
        // the FP64 polish wants about ten polish warps (one FP64 instruction in
        // flight per warp); the compensated polish is FP32 work of about the
        // sweeps' size and wants an even split
        static const int ws_small[][2] = {{512, 8}, {512, 9}, {512, 10}, {512, 11}, {256, 4}, {256, 5}, {192, 3}, {192, 4}};
        static const int ws_large[][2] = {{96, 1}, {96, 2}, {128, 1}, {128, 2}, {192, 2}, {192, 3}, {192, 4},
                                          {256, 3}, {256, 4}};
        static const int df_small[][2] = {{512, 6}, {512, 7}, {512, 8}, {512, 9}, {512, 10}, {384, 5}, {384, 6},
                                          {384, 7}, {256, 3}, {256, 4}, {256, 5}};
        static const int df_large[][2] = {{128, 1}, {128, 2}, {192, 2}, {192, 3}, {256, 2}, {256, 3}, {256, 4},
                                          {256, 5}};
        const bool df = polish_mode == RD_POLISH_DF;
        if (degree <= 6) {
            if (df)
                for (auto &s : df_small) v.push_back({1, s[0], 0, s[1]});
            else
                for (auto &s : ws_small) v.push_back({1, s[0], 0, s[1]});
        } else {
            if (df)
                for (auto &s : df_large) v.push_back({1, s[0], 0, s[1]});
            else
                for (auto &s : ws_large) v.push_back({1, s[0], 0, s[1]});
        }
    }
    return v;
}

struct TuneScratch {
    void *coeffs = nullptr;
    uint32_t *hist = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneScratch()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        if (hist) cudaFree(hist);
        if (coeffs) cudaFree(coeffs);
    }
};

int cuda_fail(const char *what, cudaError_t e)
{
    return rd_set_error(RD_ECUDA, "rd_autotune: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" int rd_autotune(int degree, rd_mode mode, int polish_mode, rd_dtype dtype, int64_t n_probe, int reps,
                           rd_tuning *out, rd_tune_entry *table, int table_cap, int *table_len)
{
    if (degree < 1 || degree > 12) return rd_set_error(RD_EUNSUPPORTED, "degree %d outside 1..12", degree);
    if (mode != RD_PLAIN_FP64 && mode != RD_MIXED) return rd_set_error(RD_EINVAL, "mode must be RD_PLAIN_FP64 or RD_MIXED");
    if (polish_mode != RD_POLISH_FP64 && polish_mode != RD_POLISH_DF)
        return rd_set_error(RD_EINVAL, "polish_mode must be RD_POLISH_FP64 or RD_POLISH_DF");
    if (dtype != RD_C64 && dtype != RD_C128) return rd_set_error(RD_EINVAL, "dtype must be RD_C64 or RD_C128");
    if (n_probe < 1024 || n_probe > ((int64_t)1 << 24)) return rd_set_error(RD_EINVAL, "n_probe must be in [1024, 2^24]");
    if (reps < 1 || reps > 15) return rd_set_error(RD_EINVAL, "reps must be in 1..15");
    if (!out) return rd_set_error(RD_EINVAL, "out is null");
    if (table && table_cap < 0) return rd_set_error(RD_EINVAL, "table_cap < 0");
    const int W = 1920, H = 1080;
    const rd_window win = {-3.0, 3.0, -1.6875, 1.6875};
    const size_t elem = dtype == RD_C64 ? 8 : 16;
    const int64_t count = n_probe * (degree + 1);

    TuneScratch S;
    cudaError_t e;
    if ((e = cudaMalloc(&S.coeffs, (size_t)count * elem)) != cudaSuccess) return cuda_fail("cudaMalloc(probe)", e);
    if ((e = cudaMalloc(reinterpret_cast<void **>(&S.hist), (size_t)W * H * 4)) != cudaSuccess)
        return cuda_fail("cudaMalloc(hist)", e);
    if ((e = cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail("stream", e);
    if ((e = cudaEventCreate(&S.e0)) != cudaSuccess || (e = cudaEventCreate(&S.e1)) != cudaSuccess)
        return cuda_fail("events", e);
    const uint64_t seed = 977 + (uint64_t)degree;
    const int gen_ctas = std::max(1, std::min(rd_sm_count_cached() * 8, (int)((count + 255) / 256)));
    if (dtype == RD_C64)
        rd::probe_kernel<float2><<<gen_ctas, 256, 0, S.st>>>(reinterpret_cast<float2 *>(S.coeffs), count, seed);
    else
        rd::probe_kernel<double2><<<gen_ctas, 256, 0, S.st>>>(reinterpret_cast<double2 *>(S.coeffs), count, seed);
    int rc = rd_check_launch("probe_kernel");
    if (rc) return rc;
    if ((rc = rd_hist_clear(S.hist, (int64_t)W * H, S.st))) return rc;

    const std::vector<Shape> cand = candidates(degree, mode, polish_mode);
    rd_tune_entry best = {0, 0, 0, 0, -1.0f}, one = {0, 0, 0, 0, -1.0f};
    int stored = 0;
    for (const Shape &sh : cand) {
        rd_params p;
        rd_default_params(mode, &p);
        if (mode == RD_MIXED) p.polish_mode = polish_mode;
        p.lanes = sh.lanes;
        p.block = sh.block;
        p.ctas_per_sm = sh.cps;
        p.polish_warps = sh.pw;
        float ms = -1.0f;
        // untimed first run: launch check and warm-up
        rc = rd_roots_density(S.coeffs, dtype, degree, n_probe, mode, &p, nullptr, win, W, H, S.hist, nullptr,
                              nullptr, nullptr, S.st);
        if (rc == RD_OK) {
            std::vector<float> t;
            for (int r = 0; r < reps && rc == RD_OK; ++r) {
                if ((e = cudaEventRecord(S.e0, S.st)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
                rc = rd_roots_density(S.coeffs, dtype, degree, n_probe, mode, &p, nullptr, win, W, H, S.hist,
                                      nullptr, nullptr, nullptr, S.st);
                if ((e = cudaEventRecord(S.e1, S.st)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
                if ((e = cudaEventSynchronize(S.e1)) != cudaSuccess) return cuda_fail("cudaEventSynchronize", e);
                float x = 0.0f;
                if ((e = cudaEventElapsedTime(&x, S.e0, S.e1)) != cudaSuccess) return cuda_fail("elapsed time", e);
                t.push_back(x);
            }
            if (rc == RD_OK) {
                std::sort(t.begin(), t.end());
                ms = t[t.size() / 2];
            }
        }
        // a shape that cannot launch leaves no sticky error; anything else is fatal
        if ((e = cudaStreamSynchronize(S.st)) != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
        const rd_tune_entry ent = {sh.lanes, sh.block, sh.cps, sh.pw, ms};
        if (table && stored < table_cap) table[stored++] = ent;
        if (ms >= 0.0f) {
            if (best.ms < 0.0f || ms < best.ms) best = ent;
            if (sh.pw == 0 && (one.ms < 0.0f || ms < one.ms)) one = ent;
        }
    }
    if (table_len) *table_len = stored;
    if (best.ms < 0.0f) return rd_set_error(RD_ECUDA, "rd_autotune: no candidate shape could be launched");
    std::memset(out, 0, sizeof(*out));
    out->best = best;
    out->one_role = one;
    out->n_candidates = (int)cand.size();
    return RD_OK;
}

extern "C" int rd_alu_peak(int kind, int64_t iters, int ctas_per_sm, double *sink, uint64_t *flops, void *stream)
{
    if (kind != RD_PEAK_FP32 && kind != RD_PEAK_FP64) return rd_set_error(RD_EINVAL, "kind must be RD_PEAK_FP32 or RD_PEAK_FP64");
    if (iters < 1 || iters > ((int64_t)1 << 24)) return rd_set_error(RD_EINVAL, "iters must be in [1, 2^24]");
    if (ctas_per_sm < 1 || ctas_per_sm > 32) return rd_set_error(RD_EINVAL, "ctas_per_sm must be in [1, 32]");
    if (!sink || ((uintptr_t)sink & 7)) return rd_set_error(RD_EINVAL, "sink null or misaligned");
    const int grid = ctas_per_sm * rd_sm_count_cached(), block = 256;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (kind == RD_PEAK_FP32)
        rd::alu_peak_f32_kernel<<<grid, block, 0, st>>>((int)iters, 0.999999f, 1e-7f, -1.2345e-33f, sink);
    else
        rd::alu_peak_f64_kernel<<<grid, block, 0, st>>>((int)iters, 0.999999999, 1e-12, -1.2345e-300, sink);
    int rc = rd_check_launch("alu_peak_kernel");
    if (rc) return rc;
    const uint64_t fma_per_iter = (uint64_t)rd::PEAK_STEPS * rd::PEAK_CHAINS * (kind == RD_PEAK_FP32 ? 2u : 1u);
    if (flops) *flops = (uint64_t)grid * block * (uint64_t)iters * fma_per_iter * 2ull;
    return RD_OK;
}
