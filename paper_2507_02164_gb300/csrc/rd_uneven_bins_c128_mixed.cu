// rd_uneven_bins_c128_mixed.cu -- uneven-degree bin solvers, complex128 coefficients,
// FP32 sweeps, FP64 polish.
#include "rd_uneven_bins.cuh"

RD_UNEVEN_BINS(double2, rd::MODE_MIXED_FP64)
