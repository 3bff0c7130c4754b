// Instantiates the push / locate / deposit kernels for NGeo = 1, fp64 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(2, true, fam_g2_fp64)
