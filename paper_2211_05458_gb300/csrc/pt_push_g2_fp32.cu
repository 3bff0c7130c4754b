// Instantiates the push / locate / deposit kernels for NGeo = 1, fp32 mode.
#include "pt_kernels.cuh"
PT_DEFINE_FAMILY(2, false, fam_g2_fp32)
