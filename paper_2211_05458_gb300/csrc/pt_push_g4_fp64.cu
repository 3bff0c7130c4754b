// Instantiates the push / locate / deposit kernels for NGeo = 3, fp64 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(4, true, fam_g4_fp64)
