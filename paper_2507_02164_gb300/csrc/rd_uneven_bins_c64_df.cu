// rd_uneven_bins_c64_df.cu -- uneven-degree bin solvers, complex64 coefficients,
// FP32 sweeps, double-float polish.
#include "rd_uneven_bins.cuh"

RD_UNEVEN_BINS(float2, rd::MODE_MIXED_DF)
