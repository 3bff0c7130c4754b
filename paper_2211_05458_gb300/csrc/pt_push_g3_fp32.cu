// Instantiates the push / locate / deposit kernels for NGeo = 2, fp32 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(3, false, fam_g3_fp32)
