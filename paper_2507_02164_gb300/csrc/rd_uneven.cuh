// rd_uneven.cuh -- workspace layout of the uneven-degree solve and the
// per-bin launcher that rd_uneven.cu calls once the batch is binned. The
// launcher is defined in rd_uneven_bins.cuh and instantiated once per
// storage type and precision mode, each in a translation unit of its own
// (rd_uneven_bins_*.cu), so that the 144 solve kernels compile in parallel.
#pragma once

#include "rd_solve.cuh"

namespace rd {

constexpr int UNEVEN_MAX_DEG = 12;

struct UnevenHeader {
    uint32_t count[16];      // polynomials per degree
    uint32_t cursor[16];     // pack cursors per degree
    uint32_t poly_base[16];  // first slot of each degree's bin in perm
    uint32_t head[16];       // task queue head of each degree's solve kernel
    uint32_t bad;            // polynomials whose offsets disagree with their degree
    uint32_t overflow;       // 1: the solvable polynomials overlap (sum of (d + 1) > n_coeffs)
    uint32_t pad[2];
    int64_t coef_base[16];   // first element of each degree's bin in the bins region
};
static_assert(sizeof(UnevenHeader) <= 512, "header must fit its 512-byte slot");

constexpr size_t UNEVEN_HEADER_BYTES = 512;

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct UnevenLayout {
    UnevenHeader *hdr;
    uint32_t *perm;
    char *bins;
};

// Largest batch the uneven path takes: n < 2^32 polynomials (32-bit slots)
// and n_coeffs <= 2^40 coefficients, so that no workspace size wraps.
constexpr int64_t UNEVEN_MAX_N = (int64_t)1 << 32;
constexpr int64_t UNEVEN_MAX_COEFFS = (int64_t)1 << 40;

inline bool uneven_sizes_ok(int64_t n, int64_t n_coeffs)
{
    return n >= 0 && n < UNEVEN_MAX_N && n_coeffs >= 0 && n_coeffs <= UNEVEN_MAX_COEFFS;
}

inline size_t uneven_bytes(int64_t n, int64_t n_coeffs, size_t elem)
{
    return UNEVEN_HEADER_BYTES + align256((size_t)n * 4) + align256((size_t)n_coeffs * elem);
}

inline UnevenLayout uneven_layout(void *ws, int64_t n)
{
    char *p = reinterpret_cast<char *>(ws);
    UnevenLayout L;
    L.hdr = reinterpret_cast<UnevenHeader *>(p);
    L.perm = reinterpret_cast<uint32_t *>(p + UNEVEN_HEADER_BYTES);
    L.bins = p + UNEVEN_HEADER_BYTES + align256((size_t)n * 4);
    return L;
}

// Fork: a helper stream of the calling host thread on the current device
// (created on its first use, non-blocking) made to wait for `st`; join:
// `st` made to wait for the helper. Both only record and wait on events, so
// they can be captured into a CUDA graph (as two parallel branches).
int uneven_fork(cudaStream_t st, cudaStream_t *side, cudaEvent_t *fork, cudaEvent_t *join, bool retry = false);
int uneven_join(cudaStream_t st, cudaStream_t side, cudaEvent_t join);

// Solve every degree bin of a packed batch (one persistent kernel per
// degree, largest degree first) with the per-degree launch shapes
// block[d], cps[d], lanes per polynomial lanes[d] and polish warps pw[d]
// (> 0: the warp-specialised form, mixed mode, degrees up to 8).
template <typename In, int MODE>
int launch_uneven_bins(const SolveArgs &a, const UnevenLayout &L, const int64_t *offsets, const int *block,
                       const int *cps, const int *lanes, const int *pw, bool fork, cudaStream_t st);

// rd_roots_uneven's argument checks and launch (rd_abi.cu); fork = false
// keeps every degree bin on `stream` and makes no helper stream.
int roots_uneven_common(const void *coeffs, rd_dtype dtype, const uint8_t *degrees, const int64_t *offsets, int64_t n,
                        int64_t n_coeffs, rd_mode mode, const rd_params *params, const rd_uneven_tuning *tuning,
                        const rd_window *window, int W, int H, uint32_t *hist, double *roots, uint8_t *status,
                        rd_stats *stats, void *ws, size_t ws_bytes, bool fork, void *stream);

}  // namespace rd
