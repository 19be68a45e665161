// rd_uneven_static.cu -- rd_roots_uneven without a caller-provided workspace.
//
// Some callers of this library cannot allocate device memory at the point
// where they want roots: code that runs under an allocator owned by another
// framework (a plugin inside a renderer or a simulation that hands out every
// byte of the GPU itself), latency-critical loops where cudaMalloc/cudaFree
// would synchronise the device, and deployments with a fixed device-memory
// budget decided up front. For them this file keeps the uneven-degree
// workspace in a fixed array of device memory that is part of the library
// image: it exists on every GPU that loads the library, for as long as the
// process lives, and no call here allocates or frees anything.
#include <cstring>
#include <mutex>

#include "rd_uneven.cuh"

// The shared scratch: 32 MiB, enough for the workspace of about 490,000
// complex64 polynomials of average degree 7. Device code could name it
// directly; host code must not pass `g_uneven_scratch` itself to a kernel
// (on the host it is only a stand-in symbol, not a device address) and looks
// up the real address with cudaGetSymbolAddress instead.
static __device__ __align__(256) unsigned char g_uneven_scratch[RD_STATIC_SCRATCH_BYTES];

namespace {

// Device address of g_uneven_scratch on the current device. A call whose
// stream is not being captured looks it up again with that device current
// (a cheap runtime query once the module is loaded), so the address follows
// a cudaDeviceReset, after which the library's module, and with it the
// array, is loaded anew; a call under stream capture takes the address the
// last call outside capture found on this device (capture forbids module
// loading), and fails if there was none.
int scratch_address(cudaStream_t st, void **out)
{
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rd_set_error(RD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return rd_set_error(RD_EUNSUPPORTED, "device index %d above 63", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return rd_set_error(RD_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_uneven_scratch);
        if (e != cudaSuccess || !p)
            return rd_set_error(RD_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        addr[dev] = p;
    } else if (!addr[dev]) {
        return rd_set_error(RD_EINVAL, "the first call on a device must come before any stream capture "
                                       "(it looks up the static scratch)");
    }
    *out = addr[dev];
    return RD_OK;
}

}  // namespace

extern "C" int rd_roots_uneven_static(const void *coeffs, rd_dtype dtype, const uint8_t *degrees,
                                      const int64_t *offsets, int64_t n, int64_t n_coeffs, rd_mode mode,
                                      const rd_params *params, const rd_uneven_tuning *tuning,
                                      const rd_window *window, int W, int H, uint32_t *hist, double *roots,
                                      uint8_t *status, rd_stats *stats, void *stream)
{
    if (n < 0 || n_coeffs < 0) return rd_set_error(RD_EINVAL, "n and n_coeffs must be >= 0");
    if (dtype != RD_C64 && dtype != RD_C128) return rd_set_error(RD_EINVAL, "dtype must be RD_C64 or RD_C128");
    size_t need = rd_uneven_workspace_bytes(n, n_coeffs, dtype);
    if (need == 0)
        return rd_set_error(RD_EINVAL, "batch too large for the uneven path (it takes n < 2^32 and n_coeffs <= 2^40), let alone the built-in scratch");
    if (need > (size_t)RD_STATIC_SCRATCH_BYTES)
        return rd_set_error(RD_EINVAL,
                            "batch needs %zu bytes of scratch; the built-in scratch holds %zu "
                            "(split the batch, or call rd_roots_uneven with your own workspace)",
                            need, (size_t)RD_STATIC_SCRATCH_BYTES);
    void *ws = nullptr;
    int rc = scratch_address(reinterpret_cast<cudaStream_t>(stream), &ws);
    if (rc) return rc;
    // the launch sequence of rd_roots_uneven, with every degree bin on the
    // caller's stream (no helper stream is made); its first launch clears the
    // scratch header, every other scratch byte is written before it is read
    return rd::roots_uneven_common(coeffs, dtype, degrees, offsets, n, n_coeffs, mode, params, tuning, window, W, H,
                                   hist, roots, status, stats, ws, (size_t)RD_STATIC_SCRATCH_BYTES, false, stream);
}
