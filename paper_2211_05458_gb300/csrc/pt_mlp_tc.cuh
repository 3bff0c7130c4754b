// pt_mlp_tc.cuh -- the learned Newton start on the 5th-generation tensor cores
// (no counterpart in the paper).  The same 51-64-64-64-3 GELU network as
// pt_mlp_infer.cuh, evaluated for a tile of 128 particles per CTA with
// tcgen05.mma (BF16 operands in shared memory, FP32 accumulators in tensor
// memory):
//   layer 1: D[128 x 64] = pre_e (per-particle element part, written into
//            TMEM with tcgen05.st) + A1[128 x 16] B1[16 x 64], A1 holding
//            xi_tri as a high and a low BF16 part per component;
//   layers 2, 3: D = 1 b^T + A[128 x 64] (W/2)^T, A = 2 GELU(z) of the
//            previous layer (GELU on packed BF16 pairs, the factor 1/2 in the
//            weights, as in the warp-level form); the bias enters as one more
//            K = 16 MMA of a constant operand (columns 0, 1 = 1) with the
//            bias's high and low BF16 parts, so no thread handles it;
//   output: D[128 x 16] = A (W4/2)^T (rows 3..15 of W4 zero), + b4 in FP32.
// One elected thread issues the MMAs and commits them to an mbarrier; every
// thread reads its own row (TMEM lane = particle) with tcgen05.ld, applies
// GELU and writes the next operand row into shared memory.
//
// Operand tiles use the no-swizzle K-major layout of 8-row x 16-byte core
// matrices: row r, k-group g (8 BF16) at byte (r/8) SBO + g LBO + (r%8) 16,
// with LBO = 128 and SBO = 128 x (K/8).
#pragma once
#include <cuda_bf16.h>

#include "pt_mlp_infer.cuh"

namespace pt {

struct __align__(1024) MlpTcSmem {
  uint16_t ah[128 * 64];  // hidden operand, K = 64
  uint16_t b2[64 * 64];   // W2 / 2, N = 64 rows, K = 64
  uint16_t b3[64 * 64];   // W3 / 2
  uint16_t a1[128 * 16];  // layer-1 operand, K = 16
  uint16_t b1[64 * 16];   // layer-1 weights, K = 16 (columns 2q, 2q+1 = W1x[.][q])
  uint16_t b4[16 * 64];   // W4 / 2, rows 3..15 zero
  uint16_t ones[128 * 16];  // bias operand: k = 0, 1 equal to 1, K = 16
  uint16_t bb[2][64 * 16];  // b2, b3 as high (k = 0) and low (k = 1) BF16 parts
  unsigned long long mbar;
  uint32_t tmem;
};
// dynamic shared memory of k_guess_tc (the struct plus room to align it to
// 1024 bytes): at most 4 CTAs per SM (4 x 128 TMEM columns = the SM's 512)
constexpr int kMlpTcSmem = (int)sizeof(MlpTcSmem) + 1024;
static_assert(4 * (kMlpTcSmem + 1024) <= 228 * 1024, "4 CTAs per SM");
constexpr uint32_t kMlpTcCols = 128;

__device__ __forceinline__ uint32_t cm_off(int row, int kg, int sbo) {
  return (uint32_t)((row >> 3) * sbo + kg * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (M/N) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd,
                                          uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          mbar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Waits for phase `parity` of the mbarrier to complete, for at most ~0.2 s of
// device time; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (t1 - t0 > 200000000ull) return false;
  }
}

// Fills the CTA's weight tiles (every thread; followed by a barrier).
__device__ __forceinline__ void mlp_tc_load(MlpTcSmem& s, const DevMLP& p) {
  // hidden layers: 64 rows x 8 k-groups of 8 BF16, W/2
  for (int i = threadIdx.x; i < 2 * 64 * 8; i += blockDim.x) {
    const int l = i >> 9, row = (i >> 3) & 63, kg = i & 7;
    const uint16_t* src = (l ? p.w3 : p.w2) + row * 64 + kg * 8;
    uint16_t* dst = (l ? s.b3 : s.b2) + cm_off(row, kg, 1024) / 2;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      dst[j] = __bfloat16_as_ushort(
          __float2bfloat16_rn(0.5f * __bfloat162float(__ushort_as_bfloat16(src[j]))));
  }
  // layer 1: 64 rows x 2 k-groups, columns 2q, 2q+1 = W1x[row][q] (q < 3)
  for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
    const int row = i >> 4, k = i & 15;
    s.b1[cm_off(row, k >> 3, 256) / 2 + (k & 7)] =
        __bfloat16_as_ushort(__float2bfloat16_rn(k < 6 ? p.w1x[3 * row + (k >> 1)] : 0.f));
  }
  // output layer: 16 rows x 8 k-groups, W4 / 2 in rows 0..2
  for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
    const int row = i >> 6, c = i & 63;
    s.b4[cm_off(row, c >> 3, 1024) / 2 + (c & 7)] =
        __bfloat16_as_ushort(__float2bfloat16_rn(row < 3 ? 0.5f * p.w4[row * 64 + c] : 0.f));
  }
  for (int i = threadIdx.x; i < 128 * 16; i += blockDim.x) {
    const int row = i >> 4, k = i & 15;
    s.ones[cm_off(row, k >> 3, 256) / 2 + (k & 7)] =
        __bfloat16_as_ushort(__float2bfloat16_rn(k < 2 ? 1.f : 0.f));
  }
  for (int i = threadIdx.x; i < 2 * 64 * 16; i += blockDim.x) {
    const int l = i >> 10, row = (i >> 4) & 63, k = i & 15;
    const float b = l ? p.b3[row] : p.b2[row];
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
    s.bb[l][cm_off(row, k >> 3, 256) / 2 + (k & 7)] =
        __bfloat16_as_ushort(__float2bfloat16_rn(k == 0 ? hi : (k == 1 ? b - hi : 0.f)));
  }
}

// One network evaluation for the CTA's 128 rows: xi_tri of this thread's row
// in, the corrected start out (guess = xi_tri + network).  Every thread of the
// CTA calls it; returns false (for every thread) if an MMA did not complete in
// time.  phase: the mbarrier's current parity, advanced here.
__device__ __forceinline__ bool mlp_tc_tile(MlpTcSmem& s, const DevMLP& p, const DevMesh& m,
                                            uint32_t tmem, int e, const float* xi_tri,
                                            float* guess, uint32_t& phase) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t mbar = smem_u32(&s.mbar);
  // accumulator of layer 1 starts at the element part pre_e
  {
    const float4* pre = reinterpret_cast<const float4*>(m.mlp_pre + 64 * (size_t)e);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 q = __ldg(pre + 4 * c + j);
        v[4 * j] = q.x;
        v[4 * j + 1] = q.y;
        v[4 * j + 2] = q.z;
        v[4 * j + 3] = q.w;
      }
      tmem_st16(lane_base + 16 * c, v);
    }
    tmem_wait_st();
  }
  // layer-1 operand row: (hi, lo) BF16 parts of xi_tri at k = 2q, 2q+1
  {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float hi = __bfloat162float(__float2bfloat16_rn(xi_tri[q]));
      w[q] = pack_bf16(hi, xi_tri[q] - hi);
    }
#pragma unroll
    for (int q = 3; q < 8; ++q) w[q] = 0u;
    const uint32_t a = smem_u32(s.a1) + cm_off(tid, 0, 256);
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(a), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(a + 128), "r"(w[4]), "r"(w[5]),
                 "r"(w[6]), "r"(w[7])
                 : "memory");
  }
  bool ok = true;
#pragma unroll 1
  for (int layer = 0; layer < 4; ++layer) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      if (layer == 0) {
        umma_bf16(tmem, umma_desc(smem_u32(s.a1), 128, 256), umma_desc(smem_u32(s.b1), 128, 256),
                  umma_idesc(128, 64), 1u);
      } else {
        const uint16_t* B = layer == 1 ? s.b2 : layer == 2 ? s.b3 : s.b4;
        const uint32_t dcol = layer == 3 ? 64u : 0u;
        const int N = layer == 3 ? 16 : 64;
        if (layer < 3)  // the accumulator starts at the bias
          umma_bf16(tmem, umma_desc(smem_u32(s.ones), 128, 256),
                    umma_desc(smem_u32(s.bb[layer - 1]), 128, 256), umma_idesc(128, 64), 0u);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          umma_bf16(tmem + dcol, umma_desc(smem_u32(s.ah) + 256 * kk, 128, 1024),
                    umma_desc(smem_u32(B) + 256 * kk, 128, 1024), umma_idesc(128, N),
                    (layer == 3 && kk == 0) ? 0u : 1u);
      }
      umma_commit(mbar);
    }
    const bool done = mbar_wait(mbar, phase);
    if (__syncthreads_or(!done)) {
      // one more bounded wait for the MMA in flight before the caller frees TMEM
      if (!done) mbar_wait(mbar, phase);
      ok = false;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    if (layer == 3) {
      float o[4];
      tmem_ld4(lane_base + 64, o);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 3; ++q) guess[q] = xi_tri[q] + o[q] + p.b4[q];
      break;
    }
    // epilogue: 2 GELU(z) of this row as the next layer's operand row
    float z[64];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld16(lane_base + 16 * c, z + 16 * c);
    tmem_wait_ld();
    const uint32_t arow = smem_u32(s.ah) + cm_off(tid, 0, 1024);
#pragma unroll
    for (int kg = 0; kg < 8; ++kg) {
      const uint32_t w0 = gelu2_bf16x2(z[8 * kg], z[8 * kg + 1]);
      const uint32_t w1 = gelu2_bf16x2(z[8 * kg + 2], z[8 * kg + 3]);
      const uint32_t w2 = gelu2_bf16x2(z[8 * kg + 4], z[8 * kg + 5]);
      const uint32_t w3 = gelu2_bf16x2(z[8 * kg + 6], z[8 * kg + 7]);
      asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(arow + 128 * kg), "r"(w0),
                   "r"(w1), "r"(w2), "r"(w3)
                   : "memory");
    }
  }
  return ok;
}

}  // namespace pt
