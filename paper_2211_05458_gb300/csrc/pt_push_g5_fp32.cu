// Instantiates the push / locate / deposit kernels for NGeo = 4, fp32 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(5, false, fam_g5_fp32)
