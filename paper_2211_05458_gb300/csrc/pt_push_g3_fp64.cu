// Instantiates the push / locate / deposit kernels for NGeo = 2, fp64 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(3, true, fam_g3_fp64)
