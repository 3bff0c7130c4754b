// pt_mlp_infer.cuh -- learned Newton start inside the push (no counterpart in
// the paper).  A 51-64-64-64-3 GELU network corrects the trilinear guess:
//   z1 = pre_e + W1x xi_tri          (element part of layer 1 precomputed per element)
//   h_l = GELU(z_l),  z2 = W2 h1 + b2,  z3 = W3 h2 + b3
//   xi0 = xi_tri + oscale * (W4 h3 + b4)
// A warp evaluates its 32 particles together and keeps the activations in
// registers; all four layers are mma.sync.m16n8k16 products (BF16 operands,
// FP32 accumulate) whose accumulator layout is the operand layout of the next
// layer, so activations never go through shared memory:
//   layer 1: [32 x 16] x [16 x 64], the k columns holding xi_tri split into a
//            high and a low BF16 part (so xi_tri enters with ~16 significant
//            bits), accumulators initialised with pre_e;
//   layers 2, 3: [32 x 64] x [64 x 64], accumulators initialised with the bias;
//   output: [32 x 64] x [64 x 8] (3 columns used).
// GELU runs on packed BF16 pairs -- its result is rounded to BF16 for the next
// product anyway.  Its factor 1/2 is moved into the weights of the layer that
// consumes it (layers 2, 3 and the output), which is exact in BF16: the
// hidden activations are 2 GELU(z).
#pragma once
#include <cuda_bf16.h>

#include "pt_device.cuh"

namespace pt {

constexpr int MLP_LD = 72;   // padded row length (bf16) of the 64-wide weight tiles
constexpr int MLP_LD1 = 24;  // padded row length (bf16) of the layer-1 tile

struct __align__(16) MlpSmem {
  __nv_bfloat16 w[2][64 * MLP_LD];  // layers 2 and 3, [out][in], padded rows
  __nv_bfloat16 w1[64 * MLP_LD1];   // layer 1, [out][k]: k = 2q, 2q+1 both W1x[out][q]
  __nv_bfloat16 w4[8 * MLP_LD];     // output layer (scaled), rows 3..7 zero
  float b[2][64];                   // biases of layers 2 and 3
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Twice the GELU in its tanh form, z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
// (Hendrycks & Gimpel 2016), on a packed pair, in BF16 arithmetic with the
// hardware tanh approximation: within a few BF16 ulps of the erf form the
// network was trained with.
__device__ __forceinline__ uint32_t gelu2_bf16x2(float z0, float z1) {
  const uint32_t z = pack_bf16(z0, z1);
  // sqrt(2/pi) * 0.044715 and sqrt(2/pi), as bf16 pairs
  const uint32_t ka = 0x3D123D12u, kc = 0x3F4C3F4Cu;
  uint32_t z2, p, u, t, out;
  asm("mul.rn.bf16x2 %0, %1, %1;" : "=r"(z2) : "r"(z));
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(p) : "r"(z2), "r"(ka), "r"(kc));
  asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(u) : "r"(z), "r"(p));
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(u));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(out) : "r"(z), "r"(t));
  return out;
}

// Fills the block's weight copy (call by every thread, followed by __syncthreads).
__device__ __forceinline__ void mlp_load(MlpSmem& s, const DevMLP& p) {
  // layers that consume a hidden activation carry GELU's factor 1/2
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int o = i >> 6, c = i & 63;
    s.w[0][o * MLP_LD + c] = __float2bfloat16_rn(0.5f * __bfloat162float(__ushort_as_bfloat16(p.w2[i])));
    s.w[1][o * MLP_LD + c] = __float2bfloat16_rn(0.5f * __bfloat162float(__ushort_as_bfloat16(p.w3[i])));
  }
  for (int i = threadIdx.x; i < 64 * MLP_LD1; i += blockDim.x) {
    const int o = i / MLP_LD1, k = i - o * MLP_LD1;
    s.w1[i] = __float2bfloat16_rn(k < 6 ? p.w1x[3 * o + (k >> 1)] : 0.f);
  }
  for (int i = threadIdx.x; i < 8 * MLP_LD; i += blockDim.x) {
    const int q = i / MLP_LD, c = i - q * MLP_LD;
    s.w4[i] = __float2bfloat16_rn(q < 3 && c < 64 ? 0.5f * p.w4[q * 64 + c] : 0.f);
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s.b[0][i] = p.b2[i];
    s.b[1][i] = p.b3[i];
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragments of two adjacent 8-column tiles (n-tiles nt, nt+1) for k-tile kt
// of a [out][in] weight tile with row length MLP_LD: b[0..1] for nt, b[2..3]
// for nt + 1.  Lane l addresses row 8 (nt + l/16) + l%8, columns 16 kt + 8 ((l/8)%2).
__device__ __forceinline__ void ldsm_b2(uint32_t* b, const __nv_bfloat16* W, int nt, int kt) {
  const int lane = threadIdx.x & 31;
  const __nv_bfloat16* row =
      W + (8 * (nt + (lane >> 4)) + (lane & 7)) * MLP_LD + 16 * kt + 8 * ((lane >> 3) & 1);
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
               : "r"(addr));
}

// Operand fragments of a warp's [32 x 64] activation: A[mt][kt][4] holds, for
// lane (g = lane/4, t = lane%4), rows 16mt+g and 16mt+g+8 at columns
// 16kt+2t, +1 (regs 0 and 1) and 16kt+2t+8, +9 (regs 2 and 3), as bf16 pairs.
// The accumulator of n-tile nt (columns 8nt+2t, +1; rows g and g+8) becomes
// operand tile nt/2, regs {0,1} for even nt and {2,3} for odd nt.
__device__ __forceinline__ void acc_to_operand(uint32_t (&A)[2][4][4], const float (&acc)[2][4][4],
                                               int half) {
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int kt = half * 2 + j;
      A[mt][kt][0] = gelu2_bf16x2(acc[mt][2 * j][0], acc[mt][2 * j][1]);
      A[mt][kt][1] = gelu2_bf16x2(acc[mt][2 * j][2], acc[mt][2 * j][3]);
      A[mt][kt][2] = gelu2_bf16x2(acc[mt][2 * j + 1][0], acc[mt][2 * j + 1][1]);
      A[mt][kt][3] = gelu2_bf16x2(acc[mt][2 * j + 1][2], acc[mt][2 * j + 1][3]);
    }
}

// One hidden layer: A <- GELU(A W^T + b), in two halves of 32 outputs.
__device__ __forceinline__ void mlp_hidden(uint32_t (&A)[2][4][4], const __nv_bfloat16* W,
                                           const float* bias) {
  const int lane = threadIdx.x & 31;
  const int t2 = (lane & 3) * 2;
  uint32_t out[2][4][4];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[2][4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float2 bb = *reinterpret_cast<const float2*>(bias + (half * 4 + nt) * 8 + t2);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        acc[mt][nt][0] = bb.x;
        acc[mt][nt][1] = bb.y;
        acc[mt][nt][2] = bb.x;
        acc[mt][nt][3] = bb.y;
      }
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        uint32_t b[4];
        ldsm_b2(b, W, half * 4 + 2 * np, kt);
        mma_bf16_16816(acc[0][2 * np], A[0][kt], b);
        mma_bf16_16816(acc[1][2 * np], A[1][kt], b);
        mma_bf16_16816(acc[0][2 * np + 1], A[0][kt], b + 2);
        mma_bf16_16816(acc[1][2 * np + 1], A[1][kt], b + 2);
      }
    acc_to_operand(out, acc, half);
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
  const int g = lane >> 2, t = lane & 3, t2 = 2 * t;
  // layer-1 operand: lane (g, t) holds component t (t < 3) of rows 16mt+g and
  // 16mt+g+8 as (hi, lo) at k = 2t, 2t+1; k >= 8 is zero
  uint32_t A1[2][4];
  int es[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int src = 16 * mt + g + 8 * hr;
      const float x0 = __shfl_sync(0xffffffffu, guess[0], src);
      const float x1 = __shfl_sync(0xffffffffu, guess[1], src);
      const float x2 = __shfl_sync(0xffffffffu, guess[2], src);
      es[mt][hr] = __shfl_sync(0xffffffffu, e, src);
      const float xv = t == 0 ? x0 : t == 1 ? x1 : t == 2 ? x2 : 0.f;
      const float hi = __bfloat162float(__float2bfloat16_rn(xv));
      A1[mt][hr] = pack_bf16(hi, xv - hi);
      A1[mt][2 + hr] = 0u;
    }
  uint32_t A[2][4][4];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const float* pre = m.mlp_pre + 64 * (size_t)es[mt][hr];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float2 pr = __ldg(reinterpret_cast<const float2*>(pre + (half * 4 + nt) * 8 + t2));
          acc[mt][nt][2 * hr] = pr.x;
          acc[mt][nt][2 * hr + 1] = pr.y;
        }
      }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      uint32_t b[2];
      b[0] = *reinterpret_cast<const uint32_t*>(s.w1 + ((half * 4 + nt) * 8 + g) * MLP_LD1 + t2);
      b[1] = 0u;
      mma_bf16_16816(acc[0][nt], A1[0], b);
      mma_bf16_16816(acc[1][nt], A1[1], b);
    }
    acc_to_operand(A, acc, half);
  }
  // layers 2 and 3 (one copy of the code)
#pragma unroll 1
  for (int l = 0; l < 2; ++l) mlp_hidden(A, s.w[l], s.b[l]);
  // output layer: one n-tile (columns 0..2 used)
  float y[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int q = 0; q < 4; ++q) y[mt][q] = 0.f;
#pragma unroll
  for (int kt = 0; kt < 4; kt += 2) {
    uint32_t b[4];  // k-tiles kt and kt + 1 of the single n-tile
    {
      const __nv_bfloat16* row = s.w4 + (lane & 7) * MLP_LD + 16 * kt + 8 * (lane >> 3);
      const uint32_t addr = (uint32_t)__cvta_generic_to_shared(row);
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                   : "r"(addr));
    }
    mma_bf16_16816(y[0], A[0][kt], b);
    mma_bf16_16816(y[1], A[1][kt], b);
    mma_bf16_16816(y[0], A[0][kt + 1], b + 2);
    mma_bf16_16816(y[1], A[1][kt + 1], b + 2);
  }
  // row r = lane of this lane's particle: mt = r/16, row group g' = r%8,
  // hr = (r/8)%2; columns 0, 1 sit in lane 4g' (regs 2hr, 2hr+1), column 2 in
  // lane 4g'+1 (reg 2hr)
  const int gs = lane & 7, mts = lane >> 4, hrs = (lane >> 3) & 1;
  float o[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int srcl = 4 * gs + (c >> 1), r0 = c & 1;
    const float v00 = __shfl_sync(0xffffffffu, y[0][r0], srcl);
    const float v01 = __shfl_sync(0xffffffffu, y[0][2 + r0], srcl);
    const float v10 = __shfl_sync(0xffffffffu, y[1][r0], srcl);
    const float v11 = __shfl_sync(0xffffffffu, y[1][2 + r0], srcl);
    o[c] = mts ? (hrs ? v11 : v10) : (hrs ? v01 : v00);
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < 3; ++q) guess[q] += o[q] + p.b4[q];
  }
}

}  // namespace pt
