// Instantiates the push / locate / deposit kernels for NGeo = 4, fp64 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(5, true, fam_g5_fp64)
