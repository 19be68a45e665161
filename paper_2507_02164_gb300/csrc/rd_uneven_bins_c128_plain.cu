// rd_uneven_bins_c128_plain.cu -- uneven-degree bin solvers, complex128 coefficients,
// FP64 sweeps.
#include "rd_uneven_bins.cuh"

RD_UNEVEN_BINS(double2, rd::MODE_PLAIN)
