// Instantiates the push / locate / deposit kernels for NGeo = 3, fp32 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(4, false, fam_g4_fp32)
