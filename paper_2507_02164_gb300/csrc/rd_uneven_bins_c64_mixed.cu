// rd_uneven_bins_c64_mixed.cu -- uneven-degree bin solvers, complex64 coefficients,
// FP32 sweeps, FP64 polish.
#include "rd_uneven_bins.cuh"

RD_UNEVEN_BINS(float2, rd::MODE_MIXED_FP64)
