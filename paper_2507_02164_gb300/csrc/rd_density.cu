// rd_density.cu -- standalone root-density binning and buffer clearing.
//
// Paper: Tang & Quan, arXiv 2507.02164, Sec. III: solved roots are converted
// to pixel coordinates and written to video memory ("Roots to Pixels", "Video
// Memory", Table I). Here the frame is a uint32 [H][W] histogram in device
// memory; at 1920 x 1080 it is 8.3 MB and stays resident in the 129 MB L2, so
// the atomics never leave the chip.
#include "rd_common.cuh"

namespace rd {

// Standalone binning of n roots. With D.n_polys > 0 the roots are grouped
// like a solve's output ([d][n_polys], root r belongs to polynomial
// r mod n_polys), which the status mask and the tile clip need: a root of a
// polynomial whose status is not RD_STATUS_OK is dropped (D.status); with
// D.clip_on the root, a point w of its polynomial's unit disk, is mapped to
// z = centre + radius w and dropped unless it falls in that polynomial's own
// tile (Sec. II: each subregion D_i counts the zeros inside it). Dropped roots
// are counted in rd_stats.clipped; the others are binned as by the fused
// solve (same FP64 operations, no contraction).

__global__ void __launch_bounds__(256) density_kernel(const double2 *__restrict__ roots, int64_t n,
                                                      DensityArgs D, uint32_t *hist, rd_stats *stats)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, stats);
    unsigned binned = 0, oow = 0, dropped = 0;
    for (int64_t base = warp_id * 32; base < n; base += warps_total * 32) {
        int64_t i = base + lane;
        int pix = -1;
        if (i < n) {
            double2 z = __ldg(roots + i);
            double x = z.x, y = z.y;
            bool keep = true;
            if (D.n_polys > 0) {
                const int64_t p = i % D.n_polys;
                if (D.status) keep = __ldg(D.status + p) == RD_STATUS_OK;
                if (D.clip_on && keep) {
                    const double2 c = __ldg(reinterpret_cast<const double2 *>(D.centres) + p);
                    x = __dadd_rn(__dmul_rn(D.radius, x), c.x);  // z = c + rho w, no contraction
                    y = __dadd_rn(__dmul_rn(D.radius, y), c.y);
                    const int64_t own = D.tile_index ? __ldg(D.tile_index + p) : p;
                    const int t = pixel_of(D.tiles, x, y);
                    keep = (t >= 0) && ((int64_t)t == own);
                }
            }
            dropped += keep ? 0u : 1u;
            pix = keep ? pixel_of(D.bin, x, y) : -1;
            binned += pix >= 0 ? 1u : 0u;
            oow += (keep && pix < 0) ? 1u : 0u;
        }
        hist_add(hist, pix);
    }
    S.add(ST_BINNED, binned);
    S.add(ST_OOW, oow);
    S.add(ST_CLIPPED, dropped);
    stats_end(S, stats);
}

__global__ void __launch_bounds__(256) clear_kernel(uint32_t *p, int64_t words)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // 16-byte stores over the aligned body, then the tail word by word
    int64_t head = ((16 - ((uintptr_t)p & 15)) & 15) / 4;
    if (head > words) head = words;
    for (int64_t k = t; k < head; k += stride) p[k] = 0;
    uint4 *body = reinterpret_cast<uint4 *>(p + head);
    int64_t nvec = (words - head) / 4;
    for (int64_t k = t; k < nvec; k += stride) body[k] = make_uint4(0, 0, 0, 0);
    for (int64_t k = head + nvec * 4 + t; k < words; k += stride) p[k] = 0;
}

int launch_density(const double *roots, int64_t n, const DensityArgs &D, uint32_t *hist, rd_stats *stats,
                   cudaStream_t st)
{
    const int block = 256;
    int64_t ctas = (n + block - 1) / block;
    int64_t cap = (int64_t)rd_sm_count_cached() * 8;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    density_kernel<<<(unsigned)ctas, block, 0, st>>>(reinterpret_cast<const double2 *>(roots), n, D, hist, stats);
    return rd_check_launch("density_kernel");
}

int launch_clear(uint32_t *p, int64_t words, cudaStream_t st)
{
    const int block = 256;
    int64_t ctas = (words / 4 + block - 1) / block;
    int64_t cap = (int64_t)rd_sm_count_cached() * 4;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    clear_kernel<<<(unsigned)ctas, block, 0, st>>>(p, words);
    return rd_check_launch("clear_kernel");
}

}  // namespace rd
