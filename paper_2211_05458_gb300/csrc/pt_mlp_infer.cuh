// pt_mlp_infer.cuh -- learned Newton start inside the push (no counterpart in
// the paper).  A 51-64-64-64-3 GELU network corrects the trilinear guess:
//   z1 = pre_e + W1x xi_tri          (element part of layer 1 precomputed per element)
//   h_l = GELU(z_l),  z2 = W2 h1 + b2,  z3 = W3 h2 + b3   (BF16 tensor cores, FP32 accumulate)
//   xi0 = xi_tri + oscale * (W4 h3 + b4)
// A warp evaluates its 32 particles together: layers 2 and 3 are
// [32 x 64] x [64 x 64] products on mma.sync.m16n8k16 (bf16 in, f32 out), the
// activations staged in shared memory in the fragment-friendly padded layout.
#pragma once
#include <cuda_bf16.h>

#include "pt_device.cuh"

namespace pt {

constexpr int MLP_LD = 72;  // padded row length (bf16) of activations and weights

struct MlpSmem {
  __nv_bfloat16 w2[64 * MLP_LD];
  __nv_bfloat16 w3[64 * MLP_LD];
  __nv_bfloat16 act[4][32 * MLP_LD];  // one [32][72] tile per warp (blocks <= 128 threads)
};

// GELU for inference in its tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
// (Hendrycks & Gimpel 2016), with the hardware tanh approximation: within about
// 1e-3 of the erf form the network was trained with, below the BF16 rounding of
// weights and activations.
__device__ __forceinline__ float gelu_f(float z) {
  float u = 0.7978845608028654f * fmaf(0.044715f * z, z * z, z), t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return 0.5f * z * (1.f + t);
}

// Fills the block's weight copy (call by every thread, followed by __syncthreads).
__device__ __forceinline__ void mlp_load(MlpSmem& s, const DevMLP& p) {
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int o = i >> 6, c = i & 63;
    s.w2[o * MLP_LD + c] = __ushort_as_bfloat16(p.w2[i]);
    s.w3[o * MLP_LD + c] = __ushort_as_bfloat16(p.w3[i]);
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// act <- GELU(act W^T + b) for the warp's [32][64] tile (in place).  The 64
// output columns are produced in two halves so that only 32 accumulators are
// live; all results stay in registers until both halves are done.
__device__ __forceinline__ void mlp_layer(__nv_bfloat16* act, const __nv_bfloat16* W,
                                          const float* bias) {
  const int lane = threadIdx.x & 31;
  const int r = lane >> 2, cq = (lane & 3) * 2;
  uint32_t outp[2][8][2];  // packed bf16 results: [m-tile][n-tile][row, row+8]
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int k0 = ks * 16;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const __nv_bfloat16* A = act + (mt * 16 + r) * MLP_LD + k0 + cq;
        a[mt][0] = *reinterpret_cast<const uint32_t*>(A);
        a[mt][1] = *reinterpret_cast<const uint32_t*>(A + 8 * MLP_LD);
        a[mt][2] = *reinterpret_cast<const uint32_t*>(A + 8);
        a[mt][3] = *reinterpret_cast<const uint32_t*>(A + 8 * MLP_LD + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* B = W + ((half * 4 + nt) * 8 + r) * MLP_LD + k0 + cq;
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(B);
        b[1] = *reinterpret_cast<const uint32_t*>(B + 8);
        mma_bf16_16816(acc[0][nt], a[0], b);
        mma_bf16_16816(acc[1][nt], a[1], b);
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = (half * 4 + nt) * 8 + cq;
        const float b0 = bias[col], b1 = bias[col + 1];
        __nv_bfloat162 lo = __floats2bfloat162_rn(gelu_f(acc[mt][nt][0] + b0),
                                                  gelu_f(acc[mt][nt][1] + b1));
        __nv_bfloat162 hi = __floats2bfloat162_rn(gelu_f(acc[mt][nt][2] + b0),
                                                  gelu_f(acc[mt][nt][3] + b1));
        outp[mt][half * 4 + nt][0] = *reinterpret_cast<uint32_t*>(&lo);
        outp[mt][half * 4 + nt][1] = *reinterpret_cast<uint32_t*>(&hi);
      }
  }
  __syncwarp();
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + cq;
      *reinterpret_cast<uint32_t*>(act + (mt * 16 + r) * MLP_LD + col) = outp[mt][nt][0];
      *reinterpret_cast<uint32_t*>(act + (mt * 16 + r + 8) * MLP_LD + col) = outp[mt][nt][1];
    }
  __syncwarp();
}

// Corrects guess[3] (the trilinear start) of this lane's particle.  Warp-
// collective: all 32 lanes call it together; a lane with live == false uses
// its own inputs and keeps its guess.
__device__ __forceinline__ void mlp_correct_smem(MlpSmem& s, const DevMLP& p, const DevMesh& m,
                                                 int e, bool live, float* guess) {
  __syncwarp();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __nv_bfloat16* act = s.act[w];
  const float* pre = m.mlp_pre + 64 * (size_t)e;
  // layer 1: element part + xi_tri columns, GELU, into this lane's row
#pragma unroll 8
  for (int o = 0; o < 64; o += 2) {
    float z0 = __ldg(pre + o) + p.w1x[3 * o] * guess[0] + p.w1x[3 * o + 1] * guess[1] +
               p.w1x[3 * o + 2] * guess[2];
    float z1 = __ldg(pre + o + 1) + p.w1x[3 * o + 3] * guess[0] + p.w1x[3 * o + 4] * guess[1] +
               p.w1x[3 * o + 5] * guess[2];
    *reinterpret_cast<__nv_bfloat162*>(act + lane * MLP_LD + o) =
        __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
  }
  __syncwarp();
  mlp_layer(act, s.w2, p.b2);
  mlp_layer(act, s.w3, p.b3);
  // output layer (FP32) on this lane's row
  float y[3] = {p.b4[0], p.b4[1], p.b4[2]};
#pragma unroll 8
  for (int i = 0; i < 64; i += 2) {
    float2 h = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(act + lane * MLP_LD + i));
#pragma unroll
    for (int q = 0; q < 3; ++q) y[q] += p.w4[64 * q + i] * h.x + p.w4[64 * q + i + 1] * h.y;
  }
  __syncwarp();
  if (live) {
#pragma unroll
    for (int q = 0; q < 3; ++q) guess[q] += y[q];
  }
}

}  // namespace pt
