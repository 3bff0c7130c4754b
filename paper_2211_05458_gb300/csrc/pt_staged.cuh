// pt_staged.cuh -- the push as one kernel per RK stage (the "staged" schedule).
//
// The resident push (k_push) keeps every particle in registers for all
// nsteps x 5 stages of a call; its one kernel carries the inverse map, the
// interpolation, the drag, the RK update, the exact face intersection, the
// walk and (optionally) the learned start, so that its register budget and
// instruction footprint are those of the largest path, and a warp in which one
// lane intersects faces stalls the other 31.  The staged schedule splits a
// stage into
//   k_stage_*   every live particle: start guess, inverse map, interpolation,
//               drag, RK update and the FP32 slab test; a particle whose stage
//               segment may touch a face (~0.5 % at the 64^3 workload) is
//               appended to a compacted list instead of being intersected;
//   k_track_*   the listed particles on full warps: exact tracking through
//               the faces (Secs. 3.2.3, 3.2.4, 2.4) and the walk that checks
//               the new owner (the missed-crossing repair of the resident
//               push, run at once instead of at the next stage's start);
// and, with the learned start, k_guess_mlp before k_stage_*.  Between stages
// the particle state goes through HBM in element-sorted order: k_gather
// copies it from the caller's arrays into library-owned structure-of-arrays
// buffers (coalesced in the visiting order), k_scatter copies it back.  Every
// arithmetic step is the resident push's own device code, in the same order.
#pragma once
#include "pt_kernels.cuh"
#include "pt_mlp_tc.cuh"

#ifndef PT_STAGE_MINB
#define PT_STAGE_MINB 3
#endif
// 1: k_stage_f32 stages the nodal state (rho, rho u) of each element its tile
// of 128 sorted particles needs in shared memory, one bulk copy per element
// (cp.async.bulk, completion on an mbarrier), and interpolates from there;
// 0: interpolation reads the state through L1
#ifndef PT_STAGE_U
#define PT_STAGE_U 0
#endif
// 1: the FP32 stage runs as two kernels, k_locate_f32 (inverse map) and
// k_advance_f32 (interpolation, drag, RK update, slab test); 0: one kernel,
// k_stage_f32
#ifndef PT_STAGE_SPLIT
#define PT_STAGE_SPLIT 0
#endif
#ifndef PT_LOCATE_MINB
#define PT_LOCATE_MINB 3
#endif
#ifndef PT_ADVANCE_MINB
#define PT_ADVANCE_MINB 3
#endif

namespace pt {

// list entry: position t in the sorted state; the high bit marks a stage end
// that needs only the walk (reference-space localisation without a wall)
constexpr unsigned kSettleOnly = 0x80000000u;

// Appends t (| flag) for every lane with want != 0; warp-collective (all 32
// lanes must call it).
__device__ __forceinline__ void list_append(const StageArgs& a, int64_t t, unsigned want) {
  const unsigned m = __ballot_sync(0xffffffffu, want != 0u);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0u;
  if (lane == leader) base = atomicAdd(a.count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) a.list[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)t | (want == 2u ? kSettleOnly : 0u);
}

// Per-thread histogram of small counts: four 16-bit bins per word (a thread
// sees far fewer than 65536 particles per launch).
struct Hist8 {
  unsigned long long w[2] = {0ull, 0ull};
  __device__ __forceinline__ void add(int v) {
    const int b = v < 7 ? (v > 0 ? v : 0) : 7;
    w[b >> 2] += 1ull << (16 * (b & 3));
  }
  __device__ __forceinline__ void flush(unsigned long long* stats, int slot, int nbins) const {
    for (int b = 0; b < nbins; ++b)
      count_add(stats, slot + b, (w[b >> 2] >> (16 * (b & 3))) & 0xFFFFull);
  }
};

__device__ __forceinline__ void stage_counters(const StageArgs& a, const PushCounters& c) {
  count_add(a.stats, PT_C_STEPS, c.steps);
  count_add(a.stats, PT_C_IT32, c.it32);
  count_add(a.stats, PT_C_IT64, c.it64);
  count_add(a.stats, PT_C_CROSS, (unsigned long long)c.tc.cross);
  count_add(a.stats, PT_C_HITS, (unsigned long long)c.tc.hits);
  count_add(a.stats, PT_C_SLOW, (unsigned long long)c.tc.slow);
}

// ---------------------------------------------------------------------------
// FP32 mode: position as a double-float offset from the owner's centre
// ---------------------------------------------------------------------------

// Returns 0 (stage end committed), 1 (listed for exact tracking) or 2 (listed
// for the walk only).
// interp4 from a shared-memory copy of the element's first four variables
template <int NP>
__device__ __forceinline__ void interp4_sh(const float* Ue, const float* l1, const float* l2,
                                           const float* l3, float* out) {
  constexpr int N3 = NP * NP * NP;
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    const float* Uv = Ue + v * N3;
    float acc = 0.f;
#pragma unroll 1
    for (int kk = 0; kk < NP; ++kk) {
      float t2 = 0.f;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const float* row = Uv + NP * (j + NP * kk);
        float t1 = 0.f;
#pragma unroll
        for (int i = 0; i < NP; i += 2) {
          const float2 q = *reinterpret_cast<const float2*>(row + i);
          t1 = fmaf(q.x, l1[i], t1);
          t1 = fmaf(q.y, l1[i + 1], t1);
        }
        t2 = fmaf(t1, l2[j], t2);
      }
      acc = fmaf(t2, l3[kk], acc);
    }
    out[v] = acc;
  }
}

// Element data requested up front: the element's FP32 geometry (high and low
// parts, 12 G^3 bytes each) and rho, rho u (16 NP^3 bytes) are read through
// rolled loops, one 64-byte piece per iteration, so without a prefetch their
// cache misses follow one another.  Issued when the owner is known, the
// misses overlap.  0: no prefetch; 1: one prefetch.global.L2 per 128-byte
// line, every thread for its own element (equal addresses of a warp merge);
// 2: the same with prefetch.global.L1; 3: one cp.async.bulk.prefetch.L2 per
// array, issued by the first lane of each run of equal owners in the warp.
// Measured on the 64^3 channel (10^7 particles): mode 3 gains 2-3 % with the
// trilinear start (whose table read, a load that depends on the owner, comes
// before the first node loads and leaves the copies time to land) and loses
// 2-3 % with the learned start; modes 1 and 2 lose 10 % with the learned
// start.  Default: mode 3, trilinear start only (PT_PREFETCH_CUR).
#ifndef PT_PREFETCH_ELEM
#define PT_PREFETCH_ELEM 3
#endif
// parts of the element data prefetched: 1 nodes (high), 2 nodes (low), 4 rho, rho u
#ifndef PT_PREFETCH_PARTS
#define PT_PREFETCH_PARTS 6
#endif
// 1: the current particle's element data is prefetched (mode PT_PREFETCH_ELEM);
// 2: only with the trilinear start
#ifndef PT_PREFETCH_CUR
#define PT_PREFETCH_CUR 2
#endif
// 1: the particle state of the thread's next grid-stride position is
// prefetched into L2 at the start of the current one; 2: in addition, that
// position's owner is read at the start and its element data prefetched
// after the current particle's inverse map
#ifndef PT_PREFETCH_NEXT
#define PT_PREFETCH_NEXT 0
#endif

__device__ __forceinline__ void prefetch_line(const void* p) {
#if PT_PREFETCH_ELEM == 2
  asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
#else
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
#endif
}

template <int BYTES>
__device__ __forceinline__ void prefetch_range(const void* p) {
  const uintptr_t b0 = (uintptr_t)p & ~(uintptr_t)127, b1 = (uintptr_t)p + BYTES;
#pragma unroll
  for (int i = 0; i < BYTES / 128 + 2; ++i)
    if (b0 + 128u * i < b1) prefetch_line(reinterpret_cast<const void*>(b0 + 128u * i));
}

template <int G, int NP>
__device__ __forceinline__ void prefetch_element(const StageArgs& a, int e, bool tri) {
  constexpr int G3 = G * G * G, N3 = NP * NP * NP;
  const float* xh = a.m.xg32 + (size_t)e * 3 * G3;
  const float* xl = a.m.xg32lo + (size_t)e * 3 * G3;
  const float* U = reinterpret_cast<const float*>(a.U) + (size_t)e * 5 * N3;
#if PT_PREFETCH_ELEM == 3
  // a bulk prefetch needs a 16-byte aligned start and size: element blocks are
  // 12 G^3 and 20 NP^3 bytes apart from aligned bases
  // (called by the warp's live lanes only)
  const int lane = threadIdx.x & 31;
  const unsigned live = __activemask();
  const int prev = __shfl_up_sync(live, e, 1);
  if (lane == 0 || !((live >> (lane - 1)) & 1u) || prev != e) {
    if constexpr ((12 * G3) % 16 == 0) {
      if (PT_PREFETCH_PARTS & 1)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(xh), "r"(12 * G3));
      if (PT_PREFETCH_PARTS & 2)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(xl), "r"(12 * G3));
    }
    if constexpr ((20 * N3) % 16 == 0) {
      if (PT_PREFETCH_PARTS & 4)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(U), "r"(16 * N3));
    }
  }
#elif PT_PREFETCH_ELEM
  if (PT_PREFETCH_PARTS & 1) prefetch_range<12 * G3>(xh);
  if (PT_PREFETCH_PARTS & 2) prefetch_range<12 * G3>(xl);
  if (PT_PREFETCH_PARTS & 4) prefetch_range<16 * N3>(U);
  if (tri) prefetch_line(a.m.tri + 12 * (size_t)e);
#endif
}

// L2 prefetch of the state that stage_one_f32 reads at position t
__device__ __forceinline__ void prefetch_state(const StageArgs& a, int64_t t, bool guess) {
  const int64_t n = a.n;
  const float* v = reinterpret_cast<const float*>(a.v);
  const float* kx = reinterpret_cast<const float*>(a.kx);
  const float* kv = reinterpret_cast<const float*>(a.kv);
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.st + t));
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.e + t));
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(reinterpret_cast<const float*>(a.d) + t));
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.xh + r * n + t));
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.xl + r * n + t));
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(v + r * n + t));
    if (a.stage > 0) {
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(kx + r * n + t));
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(kv + r * n + t));
    }
    if (guess) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.guess + r * n + t));
  }
}

// Warp slots: per warp, K copies of an element's data in shared memory (the
// FP32 nodes, high then low parts, 6 G^3 floats; rho, rho u, 4 NP^3 floats),
// one per run of equal owners among the warp's 32 sorted particles (one or
// two runs at ~30 particles per element).  The warp's lanes copy each slot
// together, all loads in flight at once, so that the element's cache misses
// overlap instead of following one another through the rolled loops of the
// inverse map and the interpolation; particles of further runs read global
// memory.  PT_STAGE_WSLOT: slots per warp (0: none; at most 40 KB per block).
// Measured slower than reading through L1 at every size (the slots leave L1 a
// third of its room, and the kernel's local memory then misses): off.
#ifndef PT_STAGE_WSLOT
#define PT_STAGE_WSLOT 0
#endif
template <int G, int NP>
struct WSlot {
  static constexpr int G3 = G * G * G, N3 = NP * NP * NP;
  // parts start on 16-byte boundaries: nodes high at 0, low at XS, state at UO
  static constexpr int XS = (3 * G3 + 3) & ~3;
  static constexpr int UO = 2 * XS;
  static constexpr int F = UO + 4 * N3;  // floats per slot (a multiple of 4)
  // float4 copies: element blocks of the nodes (3 G^3 floats) and of the
  // state (5 NP^3 floats) and the slot parts are multiples of 16 bytes
  static constexpr bool vec = (3 * G3) % 4 == 0 && N3 % 4 == 0;
  static constexpr int K = (PT_STAGE_WSLOT >= 2 && 8 * F * 4 <= 40960)
                               ? 2
                               : ((PT_STAGE_WSLOT >= 1 && 4 * F * 4 <= 40960) ? 1 : 0);
  static constexpr int bytes = 4 * K * F * 4;  // dynamic shared memory, 4 warps per block
};

// rows of the per-thread shared-memory scratch: the inverse map's bases (6 G
// floats) and the rolled loops' results (kScratchOut on)
#ifndef PT_SMEM_BASIS
#define PT_SMEM_BASIS 1
#endif
constexpr int kBasisRows = kScratchRows;

// The particle state one FP32 stage reads, loaded at once and before anything
// that depends on it (the status test included), so that its HBM latency is
// paid once per particle rather than once for the status and again for the
// rest.
struct StageIn {
  unsigned st;
  int e;
  float d;
  df xd[3];
  float v[3], kx[3], kv[3], g[3];
};

template <bool MLP>
__device__ __forceinline__ void stage_load(const StageArgs& a, int64_t t, StageIn& in) {
  const int64_t n = a.n;
  const float* vg = reinterpret_cast<const float*>(a.v);
  const float* kxg = reinterpret_cast<const float*>(a.kx);
  const float* kvg = reinterpret_cast<const float*>(a.kv);
  in.st = a.st[t];
  in.e = a.e[t];
  in.d = reinterpret_cast<const float*>(a.d)[t];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    in.xd[r] = df{a.xh[r * n + t], a.xl[r * n + t]};
    in.v[r] = vg[r * n + t];
    in.kx[r] = a.stage > 0 ? kxg[r * n + t] : 0.f;
    in.kv[r] = a.stage > 0 ? kvg[r * n + t] : 0.f;
    if constexpr (MLP) in.g[r] = a.guess[r * n + t];
  }
}

// ES: the element's data may come from a warp slot Es (WSlot layout: FP32
// nodes, high then low parts, then rho, rho u), read with generic loads;
// Es == nullptr reads global memory the same way.
template <int G, int NP, bool MLP, bool ES = false>
__device__ __forceinline__ unsigned stage_one_f32(const StageArgs& a, int64_t t,
                                                  const StageIn& in,
                                                  PushCounters& c, Hist8& h32, Hist8& h64,
                                                  const float* Us = nullptr,
                                                  float* sb = nullptr, int e_next = -1,
                                                  const float* Es = nullptr) {
  constexpr int N3 = NP * NP * NP;
  const int64_t n = a.n;
  const int s = a.stage;
  unsigned st = in.st;
  if (st & PT_ST_FROZEN) return 0u;
  const int e = in.e;
  if (PT_PREFETCH_CUR == 1 || (PT_PREFETCH_CUR == 2 && !MLP)) prefetch_element<G, NP>(a, e, !MLP);
  float* vg = reinterpret_cast<float*>(a.v);
  float* kxg = reinterpret_cast<float*>(a.kx);
  float* kvg = reinterpret_cast<float*>(a.kv);
  const float d = in.d;
  df xd[3];
  float v[3], kx[3], kv[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    xd[r] = in.xd[r];
    v[r] = in.v[r];
    kx[r] = in.kx[r];
    kv[r] = in.kv[r];
  }
  const float mu = (float)a.k.mu;
  const float tau = (float)a.k.rho_p * d * d / (18.f * mu);
  float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
  float guess[3];
  if constexpr (MLP) {
#pragma unroll
    for (int r = 0; r < 3; ++r) guess[r] = in.g[r];
  } else {
    trilinear_guess(a.m, e, xf, guess);
  }
  df zd[3];
  int i32 = 0, i64 = 0;
  bool ok;
  if constexpr (ES)
    ok = newton_df<G, 128, true>(a.m, a.k, e, xd, guess, zd, i32, i64, sb, Es);
  else
    ok = (PT_SMEM_BASIS && sb) ? newton_df<G, 128>(a.m, a.k, e, xd, guess, zd, i32, i64, sb)
                               : newton_df<G>(a.m, a.k, e, xd, guess, zd, i32, i64);
  if (e_next >= 0) prefetch_element<G, NP>(a, e_next, !MLP);
  c.it32 += i32;
  c.it64 += i64;
  h32.add(i32);
  h64.add(i64);
  if (!ok) {
    a.st[t] = st | PT_ST_NEWTON_FAIL;
    return 0u;
  }
  const float xi[3] = {zd[0].hi + zd[0].lo, zd[1].hi + zd[1].lo, zd[2].hi + zd[2].lo};
  const float mx = tmax3(xi[0], xi[1], xi[2]);
  if (mx > 1.f - fmaxf(1e-5f, (float)a.k.band_ref)) {  // decide the bands exactly (rare)
    const double z[3] = {df_to_double(zd[0]), df_to_double(zd[1]), df_to_double(zd[2])};
    const double md = tmax3(z[0], z[1], z[2]);
    if (md > 1.0 + a.k.lost_tol) {  // outside: the walk after the last crossing ran already
      a.st[t] = st | PT_ST_LOST;
      return 0u;
    }
    if (md > 1.0 - a.k.band_ref) st |= near_bits(a.m, e, z, a.k.band_ref);
  }
  // interpolation of rho, rho u at xi, drag + gravity
  const float* Ue = reinterpret_cast<const float*>(a.U) + (size_t)e * 5 * N3;
  float l1[NP], l2[NP], l3[NP], Uv[4], acc[3];
  lagr<NP, float>(xi[0], a.k.sn32, a.k.sw32, l1);
  lagr<NP, float>(xi[1], a.k.sn32, a.k.sw32, l2);
  lagr<NP, float>(xi[2], a.k.sn32, a.k.sw32, l3);
  if constexpr (ES)
    interp4<NP, float, true, 128>(Es ? Es + WSlot<G, NP>::UO : Ue, l1, l2, l3, Uv, sb);
  else if (Us)
    interp4_sh<NP>(Us, l1, l2, l3, Uv);
  else if (PT_SMEM_BASIS && sb)
    interp4<NP, float, false, 128>(Ue, l1, l2, l3, Uv, sb);
  else
    interp4<NP, float>(Ue, l1, l2, l3, Uv);
  particle_accel_f32<G, NP>(a.m, a.k, Ue, e, zd, Uv, v, d, tau, st, acc);
  const float As = a.k.A32[s], Bs = a.k.B32[s], dt = (float)a.dt;
  df xe[3];
  float bf[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    kx[r] = As * kx[r] + dt * v[r];
    kv[r] = As * kv[r] + dt * acc[r];
    xe[r] = df_add(xd[r], df_from(Bs * kx[r]));
    bf[r] = xe[r].hi;
    v[r] = v[r] + Bs * kv[r];
  }
  const int touch = slab_touch(a.m, e, xf, bf);
  unsigned list = 0u;
  if (!(touch & (a.k.track == PT_TRACK_REFERENCE ? 2 : 1))) {
    // no face reachable, or (localisation) no wall or open face: with a touch
    // the end point's owner is checked by the walk
#pragma unroll
    for (int r = 0; r < 3; ++r) xd[r] = xe[r];
    if (touch) list = 2u;
  } else {
    float* xeg = reinterpret_cast<float*>(a.xe);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      xeg[r * n + t] = xe[r].hi;
      xeg[(3 + r) * n + t] = xe[r].lo;
    }
    list = 1u;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    a.xh[r * n + t] = xd[r].hi;
    a.xl[r * n + t] = xd[r].lo;
    vg[r * n + t] = v[r];
    if (s < 4) {
      kxg[r * n + t] = kx[r];
      kvg[r * n + t] = kv[r];
    }
  }
  a.st[t] = st;
  if (s == 4 && !list) ++c.steps;
  return list;
}

// ---------------------------------------------------------------------------
// FP32 mode, split stage: the inverse map and the rest of the stage in two
// kernels, each with fewer live registers than the whole stage (the
// converged xi goes through HBM as a double-float, 24 bytes)
// ---------------------------------------------------------------------------

template <int G, bool MLP>
__global__ void __launch_bounds__(128, PT_LOCATE_MINB) k_locate_f32(const __grid_constant__ StageArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count_next = 0u;
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  Hist8 h32, h64;
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    unsigned st = a.st[t];
    if (st & PT_ST_FROZEN) continue;
    const int e = a.e[t];
    df xd[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) xd[r] = df{a.xh[r * n + t], a.xl[r * n + t]};
    float guess[3];
    if constexpr (MLP) {
#pragma unroll
      for (int r = 0; r < 3; ++r) guess[r] = a.guess[r * n + t];
    } else {
      const float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
      trilinear_guess(a.m, e, xf, guess);
    }
    df zd[3];
    int i32 = 0, i64 = 0;
    const bool ok = newton_df<G>(a.m, a.k, e, xd, guess, zd, i32, i64);
    c.it32 += i32;
    c.it64 += i64;
    h32.add(i32);
    h64.add(i64);
    if (!ok) {
      a.st[t] = st | PT_ST_NEWTON_FAIL;
      continue;
    }
    const float mx = tmax3(zd[0].hi + zd[0].lo, zd[1].hi + zd[1].lo, zd[2].hi + zd[2].lo);
    if (mx > 1.f - fmaxf(1e-5f, (float)a.k.band_ref)) {  // decide the bands exactly (rare)
      const double z[3] = {df_to_double(zd[0]), df_to_double(zd[1]), df_to_double(zd[2])};
      const double md = tmax3(z[0], z[1], z[2]);
      if (md > 1.0 + a.k.lost_tol) {  // outside: the walk after the last crossing ran already
        a.st[t] = st | PT_ST_LOST;
        continue;
      }
      if (md > 1.0 - a.k.band_ref) a.st[t] = st | near_bits(a.m, e, z, a.k.band_ref);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.xih[r * n + t] = zd[r].hi;
      a.xil[r * n + t] = zd[r].lo;
    }
  }
  stage_counters(a, c);
  h32.flush(a.stats, PT_C_H32, 8);
  h64.flush(a.stats, PT_C_H64, 8);
}

// Interpolation, drag, RK update and slab test of every live particle from
// the xi of k_locate_f32; returns 0, 1 (listed for exact tracking) or 2
// (listed for the walk), as stage_one_f32.
template <int G, int NP>
__device__ __forceinline__ unsigned advance_one_f32(const StageArgs& a, int64_t t,
                                                    PushCounters& c) {
  constexpr int N3 = NP * NP * NP;
  const int64_t n = a.n;
  const int s = a.stage;
  unsigned st = a.st[t];
  if (st & PT_ST_FROZEN) return 0u;
  const int e = a.e[t];
  float* vg = reinterpret_cast<float*>(a.v);
  float* kxg = reinterpret_cast<float*>(a.kx);
  float* kvg = reinterpret_cast<float*>(a.kv);
  const float d = reinterpret_cast<const float*>(a.d)[t];
  df xd[3], zd[3];
  float v[3], kx[3] = {0.f, 0.f, 0.f}, kv[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    xd[r] = df{a.xh[r * n + t], a.xl[r * n + t]};
    zd[r] = df{a.xih[r * n + t], a.xil[r * n + t]};
    v[r] = vg[r * n + t];
    if (s > 0) {
      kx[r] = kxg[r * n + t];
      kv[r] = kvg[r * n + t];
    }
  }
  const float mu = (float)a.k.mu;
  const float tau = (float)a.k.rho_p * d * d / (18.f * mu);
  const float xi[3] = {zd[0].hi + zd[0].lo, zd[1].hi + zd[1].lo, zd[2].hi + zd[2].lo};
  const float* Ue = reinterpret_cast<const float*>(a.U) + (size_t)e * 5 * N3;
  float l1[NP], l2[NP], l3[NP], Uv[4], acc[3];
  lagr<NP, float>(xi[0], a.k.sn32, a.k.sw32, l1);
  lagr<NP, float>(xi[1], a.k.sn32, a.k.sw32, l2);
  lagr<NP, float>(xi[2], a.k.sn32, a.k.sw32, l3);
  interp4<NP, float>(Ue, l1, l2, l3, Uv);
  particle_accel_f32<G, NP>(a.m, a.k, Ue, e, zd, Uv, v, d, tau, st, acc);
  const float As = a.k.A32[s], Bs = a.k.B32[s], dt = (float)a.dt;
  const float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
  df xe[3];
  float bf[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    kx[r] = As * kx[r] + dt * v[r];
    kv[r] = As * kv[r] + dt * acc[r];
    xe[r] = df_add(xd[r], df_from(Bs * kx[r]));
    bf[r] = xe[r].hi;
    v[r] = v[r] + Bs * kv[r];
  }
  const int touch = slab_touch(a.m, e, xf, bf);
  unsigned list = 0u;
  if (!(touch & (a.k.track == PT_TRACK_REFERENCE ? 2 : 1))) {
#pragma unroll
    for (int r = 0; r < 3; ++r) xd[r] = xe[r];
    if (touch) list = 2u;
  } else {
    float* xeg = reinterpret_cast<float*>(a.xe);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      xeg[r * n + t] = xe[r].hi;
      xeg[(3 + r) * n + t] = xe[r].lo;
    }
    list = 1u;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    a.xh[r * n + t] = xd[r].hi;
    a.xl[r * n + t] = xd[r].lo;
    vg[r * n + t] = v[r];
    if (s < 4) {
      kxg[r * n + t] = kx[r];
      kvg[r * n + t] = kv[r];
    }
  }
  a.st[t] = st;
  if (s == 4 && !list) ++c.steps;
  return list;
}

template <int G, int NP>
__global__ void __launch_bounds__(128, PT_ADVANCE_MINB) k_advance_f32(const __grid_constant__ StageArgs a) {
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;  // uniform trip count per warp
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
    const unsigned want = t < n ? advance_one_f32<G, NP>(a, t, c) : 0u;
    list_append(a, t, want);
  }
  stage_counters(a, c);
}

// shared-memory slots of the element staging (at most 40 KB per block)
template <int NP>
struct UStage {
  static constexpr int bytes = 16 * NP * NP * NP;  // rho, rho u1..u3 of one element
  static constexpr int slots = (40960 / bytes) < 8 ? (40960 / bytes) : 8;
  // a bulk copy needs 16-byte aligned element blocks: 20 NP^3 bytes apart
  static constexpr bool ok = PT_STAGE_U && (NP % 2 == 0);
};

// Fills the warp's slots for the lanes' owners e0 (-1: no particle, or a
// frozen one; every lane of the warp calls it) and returns this lane's slot,
// or nullptr.
template <int G, int NP>
__device__ __forceinline__ const float* wslot_fill(const StageArgs& a, int e0, float* slots) {
  using W = WSlot<G, NP>;
  constexpr int G3 = W::G3, N3 = W::N3, F = W::F;
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xffffffffu, e0, 1);
  const bool start = e0 >= 0 && (lane == 0 || prev != e0);
  const unsigned bm = __ballot_sync(0xffffffffu, start);
  const int run = __popc(bm & ((2u << lane) - 1u)) - 1;  // this lane's run
  __syncwarp();  // the warp's reads of the previous contents are complete
  unsigned rest = bm;
#pragma unroll
  for (int q = 0; q < W::K; ++q) {
    if (!rest) break;
    const int es = __shfl_sync(0xffffffffu, e0, __ffs(rest) - 1);
    rest &= rest - 1u;
    float* dst = slots + q * F;
    const float* xh = a.m.xg32 + (size_t)es * 3 * G3;
    const float* xl = a.m.xg32lo + (size_t)es * 3 * G3;
    const float* U = reinterpret_cast<const float*>(a.U) + (size_t)es * 5 * N3;
    if constexpr (W::vec) {
      // float4 pieces: nodes high, nodes low, state; CH loads in flight per lane
      constexpr int nx = 3 * G3 / 4, nt = F / 4, per = (nt + 31) / 32, CH = 12;
#pragma unroll
      for (int j0 = 0; j0 < per; j0 += CH) {
        float4 r[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int i = lane + 32 * (j0 + j);
          if (j0 + j < per && i < nt) {
            const float* src =
                i < nx ? xh + 4 * i : (i < 2 * nx ? xl + 4 * (i - nx) : U + 4 * (i - 2 * nx));
            r[j] = __ldg(reinterpret_cast<const float4*>(src));
          }
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int i = lane + 32 * (j0 + j);
          if (j0 + j < per && i < nt) reinterpret_cast<float4*>(dst)[i] = r[j];
        }
      }
    } else {
      // slot index i: nodes high below XS, low below UO (the padding after
      // 3 G^3 floats of each is left unwritten), state above
      constexpr int nx = 3 * G3, XS = W::XS, UO = W::UO, per = (F + 31) / 32, CH = 32;
#pragma unroll
      for (int j0 = 0; j0 < per; j0 += CH) {
        float r[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int i = lane + 32 * (j0 + j);
          const int o = i < XS ? i : (i < UO ? i - XS : i - UO);
          if (j0 + j < per && i < F && (i >= UO || o < nx))
            r[j] = __ldg(i < XS ? xh + o : (i < UO ? xl + o : U + o));
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int i = lane + 32 * (j0 + j);
          const int o = i < XS ? i : (i < UO ? i - XS : i - UO);
          if (j0 + j < per && i < F && (i >= UO || o < nx)) dst[i] = r[j];
        }
      }
    }
  }
  __syncwarp();
  return (e0 >= 0 && run < W::K) ? slots + run * F : nullptr;
}

template <int G, int NP, bool MLP>
__global__ void __launch_bounds__(128, PT_STAGE_MINB) k_stage_f32(const __grid_constant__ StageArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count_next = 0u;
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  Hist8 h32, h64;
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;  // uniform trip count per warp
  if constexpr (!UStage<NP>::ok) {
    // this thread's column of the basis scratch (blocks of 128 threads)
    __shared__ float s_basis[PT_SMEM_BASIS ? kBasisRows * 128 : 1];
    float* sb = PT_SMEM_BASIS ? s_basis + threadIdx.x : nullptr;
    if constexpr (WSlot<G, NP>::K > 0) {
      extern __shared__ __align__(16) float s_wslot[];
      float* slots = s_wslot + (threadIdx.x >> 5) * WSlot<G, NP>::K * WSlot<G, NP>::F;
      for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
        StageIn in;
        if (t < n) stage_load<MLP>(a, t, in);
        const int e0 = (t < n && !(in.st & PT_ST_FROZEN)) ? in.e : -1;
        const float* Es = wslot_fill<G, NP>(a, e0, slots);
        const unsigned want =
            t < n ? stage_one_f32<G, NP, MLP, true>(a, t, in, c, h32, h64, nullptr, sb, -1, Es)
                  : 0u;
        list_append(a, t, want);
      }
    } else
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
      int e_next = -1;
      if (PT_PREFETCH_NEXT && t + stride < n) {
        prefetch_state(a, t + stride, MLP);
        if (PT_PREFETCH_NEXT == 2) {
          e_next = a.e[t + stride];
          if ((unsigned)e_next >= (unsigned)a.m.nelem) e_next = -1;
        }
      }
      StageIn in;
      if (t < n) stage_load<MLP>(a, t, in);
      const unsigned want =
          t < n ? stage_one_f32<G, NP, MLP>(a, t, in, c, h32, h64, nullptr, sb, e_next) : 0u;
      list_append(a, t, want);
    }
  } else {
    // Per tile of 128 consecutive sorted particles: every run of equal owners
    // gets a slot (the first UStage::slots runs), filled by one bulk copy of
    // that element's rho, rho u; the tile's particles interpolate from the
    // slot (from global memory beyond the slots).
    constexpr int N3 = NP * NP * NP;
    constexpr int SL = UStage<NP>::slots;
    __shared__ __align__(128) float sU[SL][4 * N3];
    __shared__ int se[128];
    __shared__ int wcnt[4];
    __shared__ unsigned long long mbar;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t mb = smem_u32(&mbar);
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0u;
    const float* Ug = reinterpret_cast<const float*>(a.U);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + tid; t < nround; t += stride) {
      const bool inr = t < n;
      const unsigned st0 = inr ? a.st[t] : (unsigned)PT_ST_FROZEN;
      const int e0 = (inr && !(st0 & PT_ST_FROZEN)) ? a.e[t] : -1;
      fence_async_smem();  // this thread's reads of the previous tile's slots come first
      se[tid] = e0;
      __syncthreads();
      const bool start = e0 >= 0 && (tid == 0 || se[tid - 1] != e0);
      const unsigned bm = __ballot_sync(0xffffffffu, start);
      if (lane == 0) wcnt[w] = __popc(bm);
      __syncthreads();
      int off = 0, total = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        off += j < w ? wcnt[j] : 0;
        total += wcnt[j];
      }
      const int run = off + __popc(bm & ((2u << lane) - 1u)) - 1;  // run index of e0
      const int nslot = total < SL ? total : SL;
      if (tid == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb),
                     "r"(nslot * UStage<NP>::bytes)
                     : "memory");
      if (start && run < SL)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];\n" ::"r"(smem_u32(sU[run])),
            "l"(Ug + (size_t)e0 * 5 * N3), "r"(UStage<NP>::bytes), "r"(mb)
            : "memory");
      const bool done = mbar_wait(mb, phase);
      if (__syncthreads_or(!done)) {
        if (!done) mbar_wait(mb, phase);
        if (tid == 0) atomicAdd(a.stats + PT_C_TIMEOUT, 1ull);
        break;
      }
      phase ^= 1u;
      const float* Us = (e0 >= 0 && run < SL) ? sU[run] : nullptr;
      StageIn in;
      if (inr) stage_load<MLP>(a, t, in);
      const unsigned want = inr ? stage_one_f32<G, NP, MLP>(a, t, in, c, h32, h64, Us) : 0u;
      list_append(a, t, want);
    }
  }
  stage_counters(a, c);
  h32.flush(a.stats, PT_C_H32, 8);
  h64.flush(a.stats, PT_C_H64, 8);
}

// Exact tracking of the listed stage segments, then the walk that checks the
// new owner; FP64 on global positions, back to the double-float offset.
#ifndef PT_TRACK_MINB
#define PT_TRACK_MINB 1
#endif
template <int G, bool CLIP>
__global__ void __launch_bounds__(128, PT_TRACK_MINB) k_track_f32(const __grid_constant__ StageArgs a) {
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  Hist8 hcr;
  const int64_t n = a.n;
  const int s = a.stage;
  const unsigned cnt = *a.count;
  float* vg = reinterpret_cast<float*>(a.v);
  float* kxg = reinterpret_cast<float*>(a.kx);
  float* kvg = reinterpret_cast<float*>(a.kv);
  const float* xeg = reinterpret_cast<const float*>(a.xe);
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned cround = (cnt + stride - 1) / stride * stride;
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < cround; j += stride) {
    if (j >= cnt) continue;
    const unsigned ent = a.list[j];
    const int64_t t = ent & ~kSettleOnly;
    unsigned st = a.st[t];
    int e = a.e[t], hits = a.hits[t];
    df xd[3];
    float v[3], kx[3], kv[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      xd[r] = df{a.xh[r * n + t], a.xl[r * n + t]};
      v[r] = vg[r * n + t];
      kx[r] = kxg[r * n + t];  // stale at the last stage of a step: not used after it
      kv[r] = kvg[r * n + t];
    }
    bool frozen = false;
    if (!(ent & kSettleOnly)) {
      const double* ce = a.m.ce + 3 * (size_t)e;
      double xs[3], xg[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double cr = __ldg(ce + r);
        xs[r] = cr + df_to_double(xd[r]);
        xg[r] = cr + df_to_double(df{xeg[r * n + t], xeg[(3 + r) * n + t]});
      }
      const int cr0 = c.tc.cross;
      track_slow<G, float, CLIP>(a.m, a.k, e, xs, xg, v, kx, kv, hits, st, c.tc);
      hcr.add(c.tc.cross - cr0);
      const double* cn = a.m.ce + 3 * (size_t)e;
#pragma unroll
      for (int r = 0; r < 3; ++r) xd[r] = df_from_double(xs[r] - __ldg(cn + r));
      frozen = (st & PT_ST_FROZEN) != 0;
    }
    if (!frozen) {
      df zd[3];
      int cr = 0, j32 = 0, j64 = 0;
      const int rc = settle_f32<G>(a.m, a.k, e, xd, zd, false, j32, j64, cr);
      c.it32 += j32;
      c.it64 += j64;
      c.tc.cross += cr;
      if (rc) st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.xh[r * n + t] = xd[r].hi;
      a.xl[r * n + t] = xd[r].lo;
      vg[r * n + t] = v[r];
      if (s < 4) {
        kxg[r * n + t] = kx[r];
        kvg[r * n + t] = kv[r];
      }
    }
    a.e[t] = e;
    a.hits[t] = hits;
    a.st[t] = st;
    if (s == 4 && !(st & PT_ST_FROZEN)) ++c.steps;
  }
  stage_counters(a, c);
  hcr.flush(a.stats, PT_C_HCR, 4);
}

// Position of particle t relative to its owner's centre, in FP32: from the
// sorted state (the high part of the double-float offset), or (FROM_X) from
// global FP64 positions a.x.
template <bool FROM_X>
__device__ __forceinline__ void start_pos(const StageArgs& a, int64_t t, int e, float* xf) {
  const int64_t n = a.n;
  if constexpr (FROM_X) {
    const double* ce = a.m.ce + 3 * (size_t)e;
#pragma unroll
    for (int r = 0; r < 3; ++r) xf[r] = (float)(a.x[r * n + t] - __ldg(ce + r));
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) xf[r] = a.xh[r * n + t];
  }
}

// Learned start of every live particle at the current position, warp-level
// mma.sync form (the network is warp-collective: every lane takes part, dead
// lanes with live = false).
template <int G, bool FROM_X>
__global__ void __launch_bounds__(128) k_guess_mlp(const __grid_constant__ StageArgs a) {
  PT_MLP_PROLOGUE(true, a.mlp);
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
    const bool inr = t < n;
    // (a.st is null for pt_mlp_start: every particle with an owner in range)
    const unsigned st = inr ? (a.st ? a.st[t] : 0u) : (unsigned)PT_ST_FROZEN;
    const int e0 = inr ? a.e[t] : 0;
    const bool live = !(st & PT_ST_FROZEN) && e0 >= 0 && e0 < a.m.nelem;
    const int e = live ? e0 : 0;
    float xf[3] = {0.f, 0.f, 0.f};
    if (live) start_pos<FROM_X>(a, t, e, xf);
    float guess[3];
    start_guess_local<G, true>(a.m, a.k, sm, &a.mlp, e, xf, live, guess);
    if (live) {
#pragma unroll
      for (int r = 0; r < 3; ++r) a.guess[r * n + t] = guess[r];
    }
  }
}

// Learned start of every live particle on the tensor cores (tcgen05): one
// tile of 128 particles at a time per CTA, weights in shared memory,
// accumulators in 128 columns of tensor memory.  An MMA that does not complete
// within the wait limit counts in PT_C_TIMEOUT and ends the CTA's work.
template <int G, bool FROM_X>
__global__ void __launch_bounds__(128, 1) k_guess_tc(const __grid_constant__ StageArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  MlpTcSmem& s = *reinterpret_cast<MlpTcSmem*>(dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u));
  const int tid = threadIdx.x;
  mlp_tc_load(s, a.mlp);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s.tmem)),
                 "r"(kMlpTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem;
  uint32_t phase = 0u;
  const int64_t n = a.n;
  // the status, owner and (staged state) offset of a row, read one tile ahead
  // so that their HBM latency overlaps the previous tile's network
  auto row_in = [&](int64_t t, unsigned& st, int& e0, float* xo) {
    const bool inr = t < n;
    // (a.st is null for pt_mlp_start: every particle with an owner in range)
    st = inr ? (a.st ? a.st[t] : 0u) : (unsigned)PT_ST_FROZEN;
    e0 = inr ? a.e[t] : 0;
    if constexpr (!FROM_X) {
#pragma unroll
      for (int r = 0; r < 3; ++r) xo[r] = inr ? a.xh[r * n + t] : 0.f;
    }
  };
  const int64_t tstride = (int64_t)gridDim.x * 128;
  unsigned st_nx;
  int e_nx;
  float x_nx[3] = {0.f, 0.f, 0.f};
  row_in((int64_t)blockIdx.x * 128 + tid, st_nx, e_nx, x_nx);
  for (int64_t base = (int64_t)blockIdx.x * 128; base < n; base += tstride) {
    const int64_t t = base + tid;
    const unsigned st = st_nx;
    const int e0 = e_nx;
    float xc[3] = {x_nx[0], x_nx[1], x_nx[2]};
    if (base + tstride < n) row_in(t + tstride, st_nx, e_nx, x_nx);
    const bool live = !(st & PT_ST_FROZEN) && e0 >= 0 && e0 < a.m.nelem;
    const int e = live ? e0 : 0;
    float xf[3] = {0.f, 0.f, 0.f}, xi_tri[3], guess[3];
    if constexpr (FROM_X) {
      if (live) start_pos<FROM_X>(a, t, e, xf);
    } else {
#pragma unroll
      for (int r = 0; r < 3; ++r) xf[r] = live ? xc[r] : 0.f;
    }
    trilinear_guess(a.m, e, xf, xi_tri);
    if (!mlp_tc_tile(s, a.mlp, a.m, tmem, e, xi_tri, guess, phase)) {
      if (tid == 0) atomicAdd(a.stats + PT_C_TIMEOUT, 1ull);
      break;
    }
    if (live) {
#pragma unroll
      for (int r = 0; r < 3; ++r) a.guess[r * n + t] = guess[r];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kMlpTcCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// FP64 mode: global FP64 positions
// ---------------------------------------------------------------------------

template <int G, int NP>
__device__ __forceinline__ unsigned stage_one_f64(const StageArgs& a, int64_t t,
                                                  PushCounters& c, Hist8& h64) {
  constexpr int N3 = NP * NP * NP;
  const int64_t n = a.n;
  const int s = a.stage;
  unsigned st = a.st[t];
  if (st & PT_ST_FROZEN) return 0u;
  const int e = a.e[t];
  double* vg = reinterpret_cast<double*>(a.v);
  double* kxg = reinterpret_cast<double*>(a.kx);
  double* kvg = reinterpret_cast<double*>(a.kv);
  const double d = reinterpret_cast<const double*>(a.d)[t];
  double x[3], v[3], kx[3] = {0, 0, 0}, kv[3] = {0, 0, 0};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    x[r] = a.x[r * n + t];
    v[r] = vg[r * n + t];
    if (s > 0) {
      kx[r] = kxg[r * n + t];
      kv[r] = kvg[r * n + t];
    }
  }
  const double tau = a.k.rho_p * d * d / (18.0 * a.k.mu);
  const double* ce = a.m.ce + 3 * (size_t)e;
  double xl[3] = {x[0] - __ldg(ce), x[1] - __ldg(ce + 1), x[2] - __ldg(ce + 2)};
  const float xf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]};
  float guess[3];
  trilinear_guess(a.m, e, xf, guess);
  double xi[3];
  int i32 = 0, i64 = 0;
  const bool ok = locate_local<G, true>(a.m, a.k, e, xl, guess, xi, i32, i64);
  c.it32 += i32;
  c.it64 += i64;
  h64.add(i64);
  if (!ok) {
    a.st[t] = st | PT_ST_NEWTON_FAIL;
    return 0u;
  }
  const double mx = tmax3(xi[0], xi[1], xi[2]);
  if (mx > 1.0 + a.k.lost_tol) {
    a.st[t] = st | PT_ST_LOST;
    return 0u;
  }
  if (mx > 1.0 - a.k.band_ref) st |= near_bits(a.m, e, xi, a.k.band_ref);
  const double* Ue = reinterpret_cast<const double*>(a.U) + (size_t)e * 5 * N3;
  double l1[NP], l2[NP], l3[NP], Uv[4], acc[3];
  lagr<NP, double>(xi[0], a.k.sn, a.k.sw, l1);
  lagr<NP, double>(xi[1], a.k.sn, a.k.sw, l2);
  lagr<NP, double>(xi[2], a.k.sn, a.k.sw, l3);
  interp4<NP, double>(Ue, l1, l2, l3, Uv);
  particle_accel<G, NP, double>(a.m, a.k, Ue, e, xi, Uv, v, d, tau, st, acc);
  const double As = a.k.A[s], Bs = a.k.B[s], dt = a.dt;
  double xe[3];
  float bf[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    kx[r] = As * kx[r] + dt * v[r];
    kv[r] = As * kv[r] + dt * acc[r];
    const double dx = Bs * kx[r];
    xe[r] = x[r] + dx;
    bf[r] = (float)(xl[r] + dx);
    v[r] = v[r] + Bs * kv[r];
  }
  const int touch = slab_touch(a.m, e, xf, bf);
  unsigned list = 0u;
  if (!(touch & (a.k.track == PT_TRACK_REFERENCE ? 2 : 1))) {
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = xe[r];
    if (touch) list = 2u;
  } else {
    double* xeg = reinterpret_cast<double*>(a.xe);
#pragma unroll
    for (int r = 0; r < 3; ++r) xeg[r * n + t] = xe[r];
    list = 1u;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    a.x[r * n + t] = x[r];
    vg[r * n + t] = v[r];
    if (s < 4) {
      kxg[r * n + t] = kx[r];
      kvg[r * n + t] = kv[r];
    }
  }
  a.st[t] = st;
  if (s == 4 && !list) ++c.steps;
  return list;
}

template <int G, int NP>
__global__ void __launch_bounds__(128, PT_PUSH_MINB_F64) k_stage_f64(const __grid_constant__ StageArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count_next = 0u;
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  Hist8 h64;
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
    const unsigned want = t < n ? stage_one_f64<G, NP>(a, t, c, h64) : 0u;
    list_append(a, t, want);
  }
  stage_counters(a, c);
  h64.flush(a.stats, PT_C_H64, 8);
}

template <int G, bool CLIP>
__global__ void __launch_bounds__(128) k_track_f64(const __grid_constant__ StageArgs a) {
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  Hist8 hcr;
  const int64_t n = a.n;
  const int s = a.stage;
  const unsigned cnt = *a.count;
  double* vg = reinterpret_cast<double*>(a.v);
  double* kxg = reinterpret_cast<double*>(a.kx);
  double* kvg = reinterpret_cast<double*>(a.kv);
  const double* xeg = reinterpret_cast<const double*>(a.xe);
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned cround = (cnt + stride - 1) / stride * stride;
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < cround; j += stride) {
    if (j >= cnt) continue;
    const unsigned ent = a.list[j];
    const int64_t t = ent & ~kSettleOnly;
    unsigned st = a.st[t];
    int e = a.e[t], hits = a.hits[t];
    double x[3], v[3], kx[3], kv[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      x[r] = a.x[r * n + t];
      v[r] = vg[r * n + t];
      kx[r] = kxg[r * n + t];  // stale at the last stage of a step: not used after it
      kv[r] = kvg[r * n + t];
    }
    if (!(ent & kSettleOnly)) {
      double xe[3] = {xeg[t], xeg[n + t], xeg[2 * n + t]};
      const int cr0 = c.tc.cross;
      track_slow<G, double, CLIP>(a.m, a.k, e, x, xe, v, kx, kv, hits, st, c.tc);
      hcr.add(c.tc.cross - cr0);
    }
    if (!(st & PT_ST_FROZEN)) {
      double xi[3];
      int cr = 0, j64 = 0;
      const int rc = settle64<G>(a.m, a.k, e, x, xi, false, j64, cr);
      c.it64 += j64;
      c.tc.cross += cr;
      if (rc) st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.x[r * n + t] = x[r];
      vg[r * n + t] = v[r];
      if (s < 4) {
        kxg[r * n + t] = kx[r];
        kvg[r * n + t] = kv[r];
      }
    }
    a.e[t] = e;
    a.hits[t] = hits;
    a.st[t] = st;
    if (s == 4 && !(st & PT_ST_FROZEN)) ++c.steps;
  }
  stage_counters(a, c);
  hcr.flush(a.stats, PT_C_HCR, 4);
}

// ---------------------------------------------------------------------------
// the caller's arrays <-> the sorted state
// ---------------------------------------------------------------------------

// sorted[t] = caller[perm[t]]; an owner out of range freezes a live particle
// (PT_ST_LOST), as in the resident push
template <bool F64>
__global__ void __launch_bounds__(256) k_gather(const __grid_constant__ StageArgs a,
                                                const DevParticles p, const int* __restrict__ perm) {
  using R = typename RealOf<F64>::type;
  const int64_t n = a.n;
  const R* vc = reinterpret_cast<const R*>(p.v);
  const R* dc = reinterpret_cast<const R*>(p.d);
  R* vs = reinterpret_cast<R*>(a.v);
  R* ds = reinterpret_cast<R*>(const_cast<void*>(a.d));
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ip = perm[t];
    unsigned st = p.status[ip];
    const int e = p.elem[ip];
    const bool valid = e >= 0 && e < a.m.nelem;
    if (!valid && !(st & PT_ST_FROZEN)) st |= PT_ST_LOST;
    const double* ce = a.m.ce + 3 * (size_t)(valid ? e : 0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double xr = p.x[r * n + ip];
      if constexpr (F64) {
        a.x[r * n + t] = xr;
      } else {
        const df o = df_from_double(valid ? xr - __ldg(ce + r) : 0.0);
        a.xh[r * n + t] = o.hi;
        a.xl[r * n + t] = o.lo;
      }
      vs[r * n + t] = vc[r * n + ip];
    }
    ds[t] = dc[ip];
    a.e[t] = e;
    a.hits[t] = p.hits[ip];
    a.st[t] = st;
  }
}

// caller[perm[t]] = sorted[t] for every particle that was not frozen on entry
// (a particle whose owner was out of range keeps its position and velocity)
template <bool F64>
__global__ void __launch_bounds__(256) k_scatter_back(const __grid_constant__ StageArgs a,
                                                      DevParticles p, const int* __restrict__ perm) {
  using R = typename RealOf<F64>::type;
  const int64_t n = a.n;
  R* vc = reinterpret_cast<R*>(p.v);
  const R* vs = reinterpret_cast<const R*>(a.v);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ip = perm[t];
    if (p.status[ip] & PT_ST_FROZEN) continue;
    const int e = a.e[t];
    p.status[ip] = a.st[t];
    if (e < 0 || e >= a.m.nelem) continue;
    const double* ce = a.m.ce + 3 * (size_t)e;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if constexpr (F64)
        p.x[r * n + ip] = a.x[r * n + t];
      else
        p.x[r * n + ip] = __ldg(ce + r) + df_to_double(df{a.xh[r * n + t], a.xl[r * n + t]});
      vc[r * n + ip] = vs[r * n + t];
    }
    p.elem[ip] = e;
    p.hits[ip] = a.hits[t];
  }
}

}  // namespace pt
