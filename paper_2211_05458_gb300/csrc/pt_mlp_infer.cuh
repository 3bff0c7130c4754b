// pt_mlp_infer.cuh -- learned Newton start inside the push (no counterpart in
// the paper).  A 51-64-64-64-3 GELU network corrects the trilinear guess:
//   z1 = pre_e + W1x xi_tri          (element part of layer 1 precomputed per element)
//   h_l = GELU(z_l),  z2 = W2 h1 + b2,  z3 = W3 h2 + b3   (BF16 tensor cores, FP32 accumulate)
//   xi0 = xi_tri + oscale * (W4 h3 + b4)
// A warp evaluates its 32 particles together and keeps the activations in
// registers: layers 2 and 3 are [32 x 64] x [64 x 64] products on
// mma.sync.m16n8k16 (bf16 in, f32 out), and the accumulator layout of one
// product is the operand layout of the next, so activations never go through
// shared memory.  Layer 1 is evaluated directly in that operand layout.
#pragma once
#include <cuda_bf16.h>

#include "pt_device.cuh"

namespace pt {

constexpr int MLP_LD = 72;  // padded row length (bf16) of the weight tiles

struct MlpSmem {
  __nv_bfloat16 w[2][64 * MLP_LD];  // layers 2 and 3, [out][in], padded rows
  float b[2][64];                   // their biases
  float w1x[3][64];                 // first-layer columns of xi_tri
  float w4[3][64];                  // output layer (scaled)
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

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Fills the block's weight copy (call by every thread, followed by __syncthreads).
__device__ __forceinline__ void mlp_load(MlpSmem& s, const DevMLP& p) {
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int o = i >> 6, c = i & 63;
    s.w[0][o * MLP_LD + c] = __ushort_as_bfloat16(p.w2[i]);
    s.w[1][o * MLP_LD + c] = __ushort_as_bfloat16(p.w3[i]);
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s.b[0][i] = p.b2[i];
    s.b[1][i] = p.b3[i];
  }
  for (int i = threadIdx.x; i < 3 * 64; i += blockDim.x) {
    const int q = i >> 6, o = i & 63;
    s.w1x[q][o] = p.w1x[3 * o + q];
    s.w4[q][o] = p.w4[i];
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Operand fragments of a warp's [32 x 64] activation: A[mt][kt][4] holds, for
// lane (g = lane/4, t = lane%4), rows 16mt+g and 16mt+g+8 at columns
// 16kt+2t, +1 (regs 0 and 1) and 16kt+2t+8, +9 (regs 2 and 3), as bf16 pairs.
// One hidden layer: A <- pack(GELU(A W^T + b)), computed in two halves of 32
// outputs; accumulator columns 8n+2t (n-tile n) are operand tile n/2, regs
// {0,1} for even n and {2,3} for odd n.
__device__ __forceinline__ void mlp_hidden(uint32_t (&A)[2][4][4], const __nv_bfloat16* W,
                                           const float* bias) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t2 = (lane & 3) * 2;
  uint32_t out[2][4][4];
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
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* B = W + ((half * 4 + nt) * 8 + g) * MLP_LD + kt * 16 + t2;
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(B);
        b[1] = *reinterpret_cast<const uint32_t*>(B + 8);
        mma_bf16_16816(acc[0][nt], A[0][kt], b);
        mma_bf16_16816(acc[1][nt], A[1][kt], b);
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = (half * 4 + nt) * 8 + t2;
        const float b0 = bias[col], b1 = bias[col + 1];
        acc[mt][nt][0] = gelu_f(acc[mt][nt][0] + b0);
        acc[mt][nt][1] = gelu_f(acc[mt][nt][1] + b1);
        acc[mt][nt][2] = gelu_f(acc[mt][nt][2] + b0);
        acc[mt][nt][3] = gelu_f(acc[mt][nt][3] + b1);
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int kt = half * 2 + j;
        out[mt][kt][0] = pack_bf16(acc[mt][2 * j][0], acc[mt][2 * j][1]);
        out[mt][kt][1] = pack_bf16(acc[mt][2 * j][2], acc[mt][2 * j][3]);
        out[mt][kt][2] = pack_bf16(acc[mt][2 * j + 1][0], acc[mt][2 * j + 1][1]);
        out[mt][kt][3] = pack_bf16(acc[mt][2 * j + 1][2], acc[mt][2 * j + 1][3]);
      }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int q = 0; q < 4; ++q) A[mt][kt][q] = out[mt][kt][q];
}

// Corrects guess[3] (the trilinear start) of this lane's particle.  Warp-
// collective: all 32 lanes call it together; a lane with live == false uses
// its own inputs and keeps its guess.
__device__ __forceinline__ void mlp_correct_smem(MlpSmem& s, const DevMLP& p, const DevMesh& m,
                                                 int e, bool live, float* guess) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t2 = (lane & 3) * 2;
  // layer 1 for the four particles (rows 16mt+g+8hr) this lane holds
  uint32_t A[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int src = 16 * mt + g + 8 * hr;
      const float x0 = __shfl_sync(0xffffffffu, guess[0], src);
      const float x1 = __shfl_sync(0xffffffffu, guess[1], src);
      const float x2 = __shfl_sync(0xffffffffu, guess[2], src);
      const int es = __shfl_sync(0xffffffffu, e, src);
      const float* pre = m.mlp_pre + 64 * (size_t)es;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const int col = kt * 16 + t2 + 8 * hc;
          const float2 pr = __ldg(reinterpret_cast<const float2*>(pre + col));
          const float z0 = pr.x + s.w1x[0][col] * x0 + s.w1x[1][col] * x1 + s.w1x[2][col] * x2;
          const float z1 = pr.y + s.w1x[0][col + 1] * x0 + s.w1x[1][col + 1] * x1 +
                           s.w1x[2][col + 1] * x2;
          A[mt][kt][hr + 2 * hc] = pack_bf16(gelu_f(z0), gelu_f(z1));
        }
    }
  // layers 2 and 3 (one copy of the code)
#pragma unroll 1
  for (int l = 0; l < 2; ++l) mlp_hidden(A, s.w[l], s.b[l]);
  // output layer: partial sums over this lane's 16 columns for its 4 rows,
  // then summed over the 4 lanes of the row group
  float y[4][3];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const int col = kt * 16 + t2 + 8 * hc;
          uint32_t v = A[mt][kt][hr + 2 * hc];
          const float2 h = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&v));
          a0 = fmaf(s.w4[0][col], h.x, fmaf(s.w4[0][col + 1], h.y, a0));
          a1 = fmaf(s.w4[1][col], h.x, fmaf(s.w4[1][col + 1], h.y, a1));
          a2 = fmaf(s.w4[2][col], h.x, fmaf(s.w4[2][col + 1], h.y, a2));
        }
      y[2 * mt + hr][0] = a0;
      y[2 * mt + hr][1] = a1;
      y[2 * mt + hr][2] = a2;
    }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      y[j][q] += __shfl_xor_sync(0xffffffffu, y[j][q], 1);
      y[j][q] += __shfl_xor_sync(0xffffffffu, y[j][q], 2);
    }
  // row r = 8 j + g sits in slot j of row group g: this lane's particle is
  // row = lane, i.e. group lane % 8, slot lane / 8
  const int srcl = 4 * (lane & 7), slot = lane >> 3;
  float out[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float v0 = __shfl_sync(0xffffffffu, y[0][q], srcl);
    const float v1 = __shfl_sync(0xffffffffu, y[1][q], srcl);
    const float v2 = __shfl_sync(0xffffffffu, y[2][q], srcl);
    const float v3 = __shfl_sync(0xffffffffu, y[3][q], srcl);
    out[q] = slot == 0 ? v0 : slot == 1 ? v1 : slot == 2 ? v2 : v3;
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < 3; ++q) guess[q] += out[q] + p.b4[q];
  }
}

}  // namespace pt
