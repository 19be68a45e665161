// rd_density.cu -- standalone root-density binning and buffer clearing.
//
// Paper: Tang & Quan, arXiv 2507.02164, Sec. III: solved roots are converted
// to pixel coordinates and written to video memory ("Roots to Pixels", "Video
// Memory", Table I). Here the frame is a uint32 [H][W] histogram in device
// memory; at 1920 x 1080 it is 8.3 MB and stays resident in the 129 MB L2, so
// the atomics never leave the chip.
#include "rd_common.cuh"

namespace rd {

__global__ void __launch_bounds__(256) density_kernel(const double2 *__restrict__ roots, int64_t n,
                                                      Binner bin, uint32_t *hist, rd_stats *stats)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    __shared__ unsigned long long acc[ST_WORDS];
    const CtaStats S = stats_begin(acc, stats);
    unsigned binned = 0, oow = 0;
    for (int64_t base = warp_id * 32; base < n; base += warps_total * 32) {
        int64_t i = base + lane;
        int pix = -1;
        if (i < n) {
            double2 z = __ldg(roots + i);
            pix = pixel_of(bin, z.x, z.y);
            binned += pix >= 0 ? 1u : 0u;
            oow += pix < 0 ? 1u : 0u;
        }
        hist_add(hist, pix);
    }
    S.add(ST_BINNED, binned);
    S.add(ST_OOW, oow);
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

int launch_density(const double *roots, int64_t n, const Binner &bin, uint32_t *hist, rd_stats *stats,
                   cudaStream_t st)
{
    const int block = 256;
    int64_t ctas = (n + block - 1) / block;
    int64_t cap = (int64_t)rd_sm_count_cached() * 8;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    density_kernel<<<(unsigned)ctas, block, 0, st>>>(reinterpret_cast<const double2 *>(roots), n, bin, hist, stats);
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
