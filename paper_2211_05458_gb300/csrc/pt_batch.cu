// pt_batch.cu -- many independent contexts (boxes) advanced together: one
// counting sort over the concatenated element space of all boxes, then one
// persistent push kernel whose threads look up their particle's box and run
// the push for that box's polynomial degree.  The launch sequence of a call
// is captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pt_bin.h"
#include "pt_ctx.h"
#include "pt_kernels.cuh"

namespace pt {

struct DevBox {
  DevMesh m;
  DevConsts k;
  DevParticles p;
  const void* U;
  int np;
  int eoff;     // first element of this box in the concatenated element space
  int64_t poff; // first particle of this box in the concatenated particle space
};

struct BatchArgs {
  const DevBox* boxes;
  const int64_t* poffs;  // [nbox + 1]
  int nbox;
  int64_t ptot;
  int etot;
  const int* perm;
  int nsteps;
  double dt;
  unsigned long long* stats;  // [nbox][PT_C_COUNT]
};

// largest b with poffs[b] <= gp (empty boxes are skipped automatically)
__device__ __forceinline__ int find_box(const int64_t* poffs, int nbox, int64_t gp) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(poffs + mid) <= gp)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int batch_key(const BatchArgs& a, int64_t gp) {
  const int b = find_box(a.poffs, a.nbox, gp);
  const DevBox& bx = a.boxes[b];
  const int e = bx.p.elem[gp - bx.poff];
  return (e < 0 || e >= bx.m.nelem) ? a.etot : bx.eoff + e;
}

__global__ void k_hist_batch(const BatchArgs a, int* counts) {
  for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < a.ptot;
       gp += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(counts + batch_key(a, gp), 1);
}

__global__ void k_scatter_batch(const BatchArgs a, int* cursor, int* perm) {
  for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < a.ptot;
       gp += (int64_t)gridDim.x * blockDim.x)
    perm[atomicAdd(cursor + batch_key(a, gp), 1)] = (int)gp;
}

constexpr int kMaxBoxCounters = 256;

// the boxes are straight-sided (NGeo = 1): a smaller kernel, for which 3
// resident blocks per SM (168 registers) measured faster than 2
#ifndef PT_BATCH_MINB
#define PT_BATCH_MINB 3
#endif
template <int G>
__global__ void __launch_bounds__(128, PT_BATCH_MINB) k_push_batch(const BatchArgs a) {
  __shared__ unsigned long long sc[kMaxBoxCounters][6];
  for (int i = threadIdx.x; i < kMaxBoxCounters * 6; i += blockDim.x) (&sc[0][0])[i] = 0ull;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.ptot; t += stride) {
    const int64_t gp = a.perm[t];
    const int b = find_box(a.poffs, a.nbox, gp);
    const DevBox& bx = a.boxes[b];
    const int64_t ip = gp - bx.poff;
    const float* U = reinterpret_cast<const float*>(bx.U);
    PushCounters c = {0, 0, 0, {0, 0, 0}};
    switch (bx.np) {
      case 4: push_particle_f32<G, 4, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps, a.dt, c); break;
      case 5: push_particle_f32<G, 5, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps, a.dt, c); break;
      case 6: push_particle_f32<G, 6, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps, a.dt, c); break;
      case 7: push_particle_f32<G, 7, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps, a.dt, c); break;
      default: push_particle_f32<G, 8, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps, a.dt, c); break;
    }
    const int slot = b < kMaxBoxCounters ? b : kMaxBoxCounters - 1;
    if (c.steps) atomicAdd(&sc[slot][0], c.steps);
    if (c.it32) atomicAdd(&sc[slot][1], c.it32);
    if (c.it64) atomicAdd(&sc[slot][2], c.it64);
    if (c.tc.cross) atomicAdd(&sc[slot][3], (unsigned long long)c.tc.cross);
    if (c.tc.hits) atomicAdd(&sc[slot][4], (unsigned long long)c.tc.hits);
    if (c.tc.slow) atomicAdd(&sc[slot][5], (unsigned long long)c.tc.slow);
  }
  __syncthreads();
  const int slots[6] = {PT_C_STEPS, PT_C_IT32, PT_C_IT64, PT_C_CROSS, PT_C_HITS, PT_C_SLOW};
  for (int i = threadIdx.x; i < a.nbox * 6 && i < kMaxBoxCounters * 6; i += blockDim.x) {
    const unsigned long long v = (&sc[0][0])[i];
    if (v) atomicAdd(a.stats + (size_t)(i / 6) * PT_C_COUNT + slots[i % 6], v);
  }
}

__global__ void k_status_counts_batch(const BatchArgs a) {
  for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < a.ptot;
       gp += (int64_t)gridDim.x * blockDim.x) {
    const int b = find_box(a.poffs, a.nbox, gp);
    const DevBox& bx = a.boxes[b];
    const unsigned s = bx.p.status[gp - bx.poff];
    unsigned long long* st = a.stats + (size_t)b * PT_C_COUNT;
    if (s & PT_ST_NEAR_FACE) atomicAdd(st + PT_C_NEAR, 1ull);
    if (s & PT_ST_NEWTON_FAIL) atomicAdd(st + PT_C_NFAIL, 1ull);
    if (s & PT_ST_LOST) atomicAdd(st + PT_C_LOST, 1ull);
    if (s & PT_ST_CROSS_CAP) atomicAdd(st + PT_C_CCAP, 1ull);
    if (s & PT_ST_OPEN) atomicAdd(st + PT_C_OPEN, 1ull);
    if (s & PT_ST_REP800) atomicAdd(st + PT_C_REP, 1ull);
    if (s & PT_ST_NEAR_WALL) atomicAdd(st + PT_C_NEARWALL, 1ull);
  }
}

}  // namespace pt

using namespace pt;

DevMesh pt_dev_mesh(const pt_ctx* c);
void pt_fill_consts(const pt_ctx* c, DevConsts& k);

struct pt_batch_plan {
  std::vector<const pt_ctx*> ctxs;
  std::vector<pt_particles> parts;
  int nbox = 0;
  int64_t ptot = 0;
  int etot = 0;
  DevBox* d_boxes = nullptr;
  int64_t* d_poffs = nullptr;
  int* d_scratch = nullptr;
  int* d_perm = nullptr;
  unsigned long long* d_stats = nullptr;
  int nsm = 1;
  // online block-size tuning: candidates are tried on successive chunks of
  // the first call, timed with events; the fastest is kept
  int block = 0;
  std::vector<int> tried;
  std::vector<float> tried_ms;
  int occ[3] = {0, 0, 0};  // resident blocks per SM of k_push_batch per candidate block size
  // private stream the graph is captured on (the caller's stream may be the
  // legacy default stream, which cannot be captured); the graph runs on the
  // caller's stream
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_nsteps = -1;
  double graph_dt = 0.0;
  int graph_block = 0;
  ~pt_batch_plan() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_boxes);
    cudaFree(d_poffs);
    cudaFree(d_scratch);
    cudaFree(d_perm);
    cudaFree(d_stats);
  }
};

void pt_batch_release(pt_ctx* c) {
  delete c->batch;
  c->batch = nullptr;
}

static const int kBlocks[3] = {64, 96, 128};
static const int kChunk = 10;

static void enqueue_chunk(pt_batch_plan* P, const BatchArgs& a, int block, cudaStream_t s) {
  BinLayout L;
  bin_layout(P->etot, P->d_scratch, L);
  cudaMemsetAsync(L.counts, 0, sizeof(int) * L.nbins, s);
  const int g = (int)std::min<int64_t>((P->ptot + 255) / 256, (int64_t)P->nsm * 8);
  k_hist_batch<<<std::max(g, 1), 256, 0, s>>>(a, L.counts);
  bin_scan(L, s);
  k_scatter_batch<<<std::max(g, 1), 256, 0, s>>>(a, L.cursor, P->d_perm);
  // occupancy was queried when the plan was made: no API call but stream work
  // may run here while the stream is being captured
  int occ = 1;
  for (int i = 0; i < 3; ++i)
    if (kBlocks[i] == block) occ = std::max(P->occ[i], 1);
  const int64_t want = (P->ptot + block - 1) / block;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)P->nsm * occ));
  k_push_batch<2><<<grid, block, 0, s>>>(a);
}

static bool same_plan(const pt_batch_plan* P, pt_ctx* const* ctxs, const pt_particles* parts,
                      int nbox) {
  if (!P || P->nbox != nbox) return false;
  for (int b = 0; b < nbox; ++b) {
    if (P->ctxs[b] != ctxs[b]) return false;
    if (std::memcmp(&P->parts[b], &parts[b], sizeof(pt_particles)) != 0) return false;
  }
  return true;
}

extern "C" pt_status pt_push_batch(pt_ctx* const* ctxs, const pt_particles* parts, int32_t nbox,
                                   int32_t nsteps, double dt, pt_stats* out) {
  if (!ctxs || !ctxs[0] || !parts || nbox < 1) return PT_ERR_ARG;
  pt_ctx* c0 = ctxs[0];
  if (nbox > kMaxBoxCounters) {
    c0->err = "pt_push_batch: at most 256 boxes";
    return PT_ERR_ARG;
  }
  if (nsteps < 0 || !(dt > 0)) {
    c0->err = "pt_push_batch: nsteps >= 0 and dt > 0 required";
    return PT_ERR_ARG;
  }
  for (int b = 0; b < nbox; ++b) {
    const pt_ctx* c = ctxs[b];
    if (!c || c->g != 2 || c->cfg.precision != PT_FP32 || c->N < 3 || c->N > 7 || !c->U ||
        c->dev != c0->dev || c->cfg.guess != PT_GUESS_TRILINEAR) {
      c0->err = "pt_push_batch: every box needs ngeo = 1, PT_FP32, N in 3..7, a fluid state, "
                "the trilinear start and the same device";
      return PT_ERR_ARG;
    }
    if (parts[b].n < 0 || (parts[b].n > 0 && (!parts[b].x || !parts[b].v || !parts[b].d ||
                                             !parts[b].elem || !parts[b].hits || !parts[b].status))) {
      c0->err = "pt_push_batch: bad particle arrays";
      return PT_ERR_ARG;
    }
  }
  cudaStream_t s = c0->stream;
  pt_batch_plan* P = c0->batch;
  if (!same_plan(P, ctxs, parts, nbox)) {
    delete P;
    P = c0->batch = new pt_batch_plan();
    P->nbox = nbox;
    P->nsm = c0->nsm;
    std::vector<DevBox> hb(nbox);
    std::vector<int64_t> poffs(nbox + 1, 0);
    int64_t pt = 0;
    int64_t et = 0;
    for (int b = 0; b < nbox; ++b) {
      const pt_ctx* c = ctxs[b];
      P->ctxs.push_back(c);
      P->parts.push_back(parts[b]);
      DevBox& d = hb[b];
      std::memset(&d, 0, sizeof d);
      d.m = pt_dev_mesh(c);
      pt_fill_consts(c, d.k);
      d.p = {parts[b].n, parts[b].x, parts[b].v, parts[b].d, parts[b].elem, parts[b].hits,
             parts[b].status};
      d.U = c->U;
      d.np = c->N + 1;
      d.eoff = (int)et;
      d.poff = pt;
      poffs[b] = pt;
      pt += parts[b].n;
      et += c->nelem;
    }
    poffs[nbox] = pt;
    if (pt > INT32_MAX || et > (1 << 28)) {
      c0->err = "pt_push_batch: too many particles or elements";
      return PT_ERR_ARG;
    }
    P->ptot = pt;
    P->etot = (int)et;
    cudaError_t e1 = cudaMalloc(&P->d_boxes, sizeof(DevBox) * nbox);
    cudaError_t e2 = cudaMalloc(&P->d_poffs, sizeof(int64_t) * (nbox + 1));
    cudaError_t e3 = cudaMalloc(&P->d_scratch, sizeof(int) * bin_scratch_ints(P->etot));
    cudaError_t e4 = cudaMalloc(&P->d_perm, sizeof(int) * std::max<int64_t>(pt, 1));
    cudaError_t e5 = cudaMalloc(&P->d_stats, sizeof(unsigned long long) * PT_C_COUNT * nbox);
    if (e1 || e2 || e3 || e4 || e5) {
      c0->err = "pt_push_batch: device allocation failed";
      return PT_ERR_CUDA;
    }
    cudaMemcpy(P->d_boxes, hb.data(), sizeof(DevBox) * nbox, cudaMemcpyHostToDevice);
    cudaMemcpy(P->d_poffs, poffs.data(), sizeof(int64_t) * (nbox + 1), cudaMemcpyHostToDevice);
    for (int i = 0; i < 3; ++i)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P->occ[i], k_push_batch<2>, kBlocks[i], 0);
    if (cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) != cudaSuccess) {
      c0->err = "pt_push_batch: stream creation failed";
      return PT_ERR_CUDA;
    }
  }
  BatchArgs a;
  a.boxes = P->d_boxes;
  a.poffs = P->d_poffs;
  a.nbox = nbox;
  a.ptot = P->ptot;
  a.etot = P->etot;
  a.perm = P->d_perm;
  a.dt = dt;
  a.stats = P->d_stats;
  if (P->ptot > 0 && nsteps > 0) {
    if (P->block == 0) {
      // tuning call: chunks go out one by one with candidate block sizes
      cudaMemsetAsync(P->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT * nbox, s);
      for (int s0 = 0; s0 < nsteps; s0 += kChunk) {
        a.nsteps = std::min(kChunk, nsteps - s0);
        const int cand = (int)P->tried.size();
        const int block = cand < 3 ? kBlocks[cand] : 128;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
        enqueue_chunk(P, a, block, s);
        c0->launches += 6;  // histogram, three scan kernels, scatter, push
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cand < 3) {
          P->tried.push_back(block);
          P->tried_ms.push_back(ms / std::max(a.nsteps, 1));
        }
      }
      if (P->tried.size() >= 3) {
        int best = 0;
        for (int i = 1; i < 3; ++i)
          if (P->tried_ms[i] < P->tried_ms[best]) best = i;
        P->block = P->tried[best];
      }
    } else {
      if (!P->graph || P->graph_nsteps != nsteps || P->graph_dt != dt ||
          P->graph_block != P->block) {
        if (P->graph) cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
        cudaGraph_t g = nullptr;
        // capturing only records the work: nothing runs on P->cap
        cudaError_t e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaMemsetAsync(P->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT * nbox, P->cap);
          for (int s0 = 0; s0 < nsteps; s0 += kChunk) {
            a.nsteps = std::min(kChunk, nsteps - s0);
            enqueue_chunk(P, a, P->block, P->cap);
          }
          e = cudaStreamEndCapture(P->cap, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          (void)cudaGetLastError();  // do not leave the failure to later calls
          c0->err = std::string("pt_push_batch: graph capture failed: ") + cudaGetErrorString(e);
          return PT_ERR_CUDA;
        }
        P->graph_nsteps = nsteps;
        P->graph_dt = dt;
        P->graph_block = P->block;
      }
      cudaError_t e = cudaGraphLaunch(P->graph, s);
      c0->launches += 6 * (int64_t)((nsteps + kChunk - 1) / kChunk);
      if (e != cudaSuccess) {
        c0->err = std::string("pt_push_batch: graph launch: ") + cudaGetErrorString(e);
        return PT_ERR_CUDA;
      }
    }
  } else {
    cudaMemsetAsync(P->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT * nbox, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c0->err = std::string("pt_push_batch: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  if (!out) return PT_OK;
  if (P->ptot > 0) {
    const int g = (int)std::min<int64_t>((P->ptot + 255) / 256, (int64_t)P->nsm * 8);
    k_status_counts_batch<<<std::max(g, 1), 256, 0, s>>>(a);
  }
  std::vector<unsigned long long> h((size_t)PT_C_COUNT * nbox);
  cudaMemcpyAsync(h.data(), P->d_stats, h.size() * 8, cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    c0->err = std::string("pt_push_batch: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  pt_status ret = PT_OK;
  for (int b = 0; b < nbox; ++b) {
    const unsigned long long* q = &h[(size_t)b * PT_C_COUNT];
    pt_stats& o = out[b];
    std::memset(&o, 0, sizeof o);
    o.particle_steps = (int64_t)q[PT_C_STEPS];
    o.crossings = (int64_t)q[PT_C_CROSS];
    o.wall_hits = (int64_t)q[PT_C_HITS];
    o.newton_it_fp32 = (int64_t)q[PT_C_IT32];
    o.newton_it_fp64 = (int64_t)q[PT_C_IT64];
    o.slow_track = (int64_t)q[PT_C_SLOW];
    o.near_face = (int64_t)q[PT_C_NEAR];
    o.newton_fail = (int64_t)q[PT_C_NFAIL];
    o.lost = (int64_t)q[PT_C_LOST];
    o.cross_cap = (int64_t)q[PT_C_CCAP];
    o.open = (int64_t)q[PT_C_OPEN];
    o.rep800 = (int64_t)q[PT_C_REP];
    o.near_wall = (int64_t)q[PT_C_NEARWALL];
    if (ret == PT_OK) {
      if (o.newton_fail) ret = PT_ERR_NEWTON;
      else if (o.lost) ret = PT_ERR_LOST;
      else if (o.cross_cap) ret = PT_ERR_CROSS;
    }
  }
  if (ret != PT_OK) c0->err = "pt_push_batch: some particles were frozen (see stats)";
  return ret;
}
