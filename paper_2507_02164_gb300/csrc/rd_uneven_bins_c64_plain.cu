// rd_uneven_bins_c64_plain.cu -- uneven-degree bin solvers, complex64 coefficients,
// FP64 sweeps.
#include "rd_uneven_bins.cuh"

RD_UNEVEN_BINS(float2, rd::MODE_PLAIN)
