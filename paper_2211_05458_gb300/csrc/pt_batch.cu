// pt_batch.cu -- many independent contexts (boxes) advanced together.  The
// boxes are grouped by polynomial degree N; their elements are concatenated in
// that order, so that one counting sort over the concatenated element space
// leaves the particles of each group contiguous.  Each group is pushed by its
// own instantiation of the push kernel (registers and unrolling of that N),
// its block size chosen per group by timing the candidates on the first
// chunks of the first call; the groups' kernels run as parallel branches of a
// CUDA graph captured once per (nsteps, dt) and replayed.
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
  const int* offs;            // [etot + 2] segment offsets of the sorted order
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
// One degree group: the particles whose global element lies in [e_lo, e_hi)
// (sorted positions offs[e_lo] .. offs[e_hi]), all in boxes with N + 1 = NP.
// The last group also takes the trailing bin of owners out of range, which the
// push marks lost without touching the fluid state.
template <int G, int NP>
__global__ void __launch_bounds__(128, PT_BATCH_MINB) k_push_batch(const BatchArgs a, int e_lo,
                                                                   int e_hi) {
  __shared__ unsigned long long sc[kMaxBoxCounters][6];
  for (int i = threadIdx.x; i < kMaxBoxCounters * 6; i += blockDim.x) (&sc[0][0])[i] = 0ull;
  __syncthreads();
  const int64_t beg = a.offs[e_lo], end = a.offs[e_hi];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < end; t += stride) {
    const int64_t gp = a.perm[t];
    const int b = find_box(a.poffs, a.nbox, gp);
    const DevBox& bx = a.boxes[b];
    const int64_t ip = gp - bx.poff;
    const float* U = reinterpret_cast<const float*>(bx.U);
    PushCounters c = {0, 0, 0, {0, 0, 0}};
    push_particle_f32<G, NP, false>(bx.m, bx.k, nullptr, nullptr, U, bx.p, ip, true, a.nsteps,
                                    a.dt, c);
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

static void launch_group(int np, const BatchArgs& a, int e_lo, int e_hi, int grid, int block,
                         cudaStream_t s) {
  switch (np) {
    case 4: k_push_batch<2, 4><<<grid, block, 0, s>>>(a, e_lo, e_hi); break;
    case 5: k_push_batch<2, 5><<<grid, block, 0, s>>>(a, e_lo, e_hi); break;
    case 6: k_push_batch<2, 6><<<grid, block, 0, s>>>(a, e_lo, e_hi); break;
    case 7: k_push_batch<2, 7><<<grid, block, 0, s>>>(a, e_lo, e_hi); break;
    default: k_push_batch<2, 8><<<grid, block, 0, s>>>(a, e_lo, e_hi); break;
  }
}

static int group_occupancy(int np, int block) {
  int nb = 0;
  switch (np) {
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_batch<2, 4>, block, 0); break;
    case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_batch<2, 5>, block, 0); break;
    case 6: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_batch<2, 6>, block, 0); break;
    case 7: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_batch<2, 7>, block, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_batch<2, 8>, block, 0); break;
  }
  return std::max(nb, 1);
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

struct pt_batch_group {
  int np = 0;           // N + 1 of the group's boxes
  int e_lo = 0, e_hi = 0;  // its range of the concatenated element space
  int block = 0;        // chosen threads per block (0: still tuning)
  int occ[3] = {0, 0, 0};  // resident blocks per SM for each candidate block size
  float ms[3] = {0.f, 0.f, 0.f};  // measured time per step of each candidate
  int tried = 0;
  cudaStream_t st = nullptr;      // branch stream of the captured graph
  cudaEvent_t done = nullptr;
};

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
  std::vector<pt_batch_group> groups;
  // private stream the graph is captured on (the caller's stream may be the
  // legacy default stream, which cannot be captured); the graph runs on the
  // caller's stream
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_nsteps = -1;
  double graph_dt = 0.0;
  ~pt_batch_plan() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto& g : groups) {
      if (g.st) cudaStreamDestroy(g.st);
      if (g.done) cudaEventDestroy(g.done);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_boxes);
    cudaFree(d_poffs);
    cudaFree(d_scratch);
    cudaFree(d_perm);
    cudaFree(d_stats);
  }
  bool tuned() const {
    for (const auto& g : groups)
      if (!g.block) return false;
    return true;
  }
};

void pt_batch_release(pt_ctx* c) {
  delete c->batch;
  c->batch = nullptr;
}

static const int kBlocks[3] = {64, 96, 128};
static const int kChunk = 10;

static int group_grid(const pt_batch_plan* P, const pt_batch_group& g, int cand) {
  const int64_t want = (P->ptot + kBlocks[cand] - 1) / kBlocks[cand];
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)P->nsm * g.occ[cand]));
}

// binning of all particles over the concatenated element space
static void enqueue_bin(pt_batch_plan* P, const BatchArgs& a, cudaStream_t s) {
  BinLayout L;
  bin_layout(P->etot, P->d_scratch, L);
  cudaMemsetAsync(L.counts, 0, sizeof(int) * L.nbins, s);
  const int g = (int)std::min<int64_t>((P->ptot + 255) / 256, (int64_t)P->nsm * 8);
  k_hist_batch<<<std::max(g, 1), 256, 0, s>>>(a, L.counts);
  bin_scan(L, s);
  k_scatter_batch<<<std::max(g, 1), 256, 0, s>>>(a, L.cursor, P->d_perm);
}

static int cand_of(int block) {
  for (int i = 0; i < 3; ++i)
    if (kBlocks[i] == block) return i;
  return 2;
}

// one chunk with every group on its tuned block size; the groups as parallel
// branches (fork / join events) when par, else one after another on s
static void enqueue_chunk(pt_batch_plan* P, const BatchArgs& a, cudaStream_t s, bool par) {
  enqueue_bin(P, a, s);
  if (par) cudaEventRecord(P->fork, s);
  for (auto& g : P->groups) {
    const int cand = cand_of(g.block);
    cudaStream_t gs = par ? g.st : s;
    if (par) cudaStreamWaitEvent(gs, P->fork, 0);
    launch_group(g.np, a, g.e_lo, g.e_hi, group_grid(P, g, cand), kBlocks[cand], gs);
    if (par) {
      cudaEventRecord(g.done, gs);
      cudaStreamWaitEvent(s, g.done, 0);
    }
  }
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
    // element space ordered by degree (then box index): each degree's
    // particles form one contiguous range of the sorted order
    std::vector<int> order(nbox);
    for (int b = 0; b < nbox; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return ctxs[x]->N < ctxs[y]->N; });
    int64_t et = 0;
    for (int i = 0; i < nbox; ++i) {
      const int b = order[i];
      const pt_ctx* c = ctxs[b];
      if (P->groups.empty() || P->groups.back().np != c->N + 1) {
        pt_batch_group g;
        g.np = c->N + 1;
        g.e_lo = g.e_hi = (int)et;
        P->groups.push_back(g);
      }
      hb[b].eoff = (int)et;
      et += c->nelem;
      P->groups.back().e_hi = (int)et;
    }
    if (!P->groups.empty()) P->groups.back().e_hi = (int)et + 1;  // + the trailing bin
    int64_t pt = 0;
    for (int b = 0; b < nbox; ++b) {
      const pt_ctx* c = ctxs[b];
      P->ctxs.push_back(c);
      P->parts.push_back(parts[b]);
      DevBox& d = hb[b];
      const int eoff = d.eoff;
      std::memset(&d, 0, sizeof d);
      d.m = pt_dev_mesh(c);
      pt_fill_consts(c, d.k);
      d.p = {parts[b].n, parts[b].x, parts[b].v, parts[b].d, parts[b].elem, parts[b].hits,
             parts[b].status};
      d.U = c->U;
      d.np = c->N + 1;
      d.eoff = eoff;
      d.poff = pt;
      poffs[b] = pt;
      pt += parts[b].n;
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
    bool ok = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto& g : P->groups) {
      for (int i = 0; i < 3; ++i) g.occ[i] = group_occupancy(g.np, kBlocks[i]);
      ok = ok && cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      c0->err = "pt_push_batch: stream or event creation failed";
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
  {
    BinLayout L;
    bin_layout(P->etot, P->d_scratch, L);
    a.offs = L.offs;
  }
  a.dt = dt;
  a.stats = P->d_stats;
  if (P->ptot > 0 && nsteps > 0) {
    if (!P->tuned()) {
      // tuning call: chunk by chunk, every group still tuning runs the next
      // candidate block size, timed on its own; groups run one after another
      cudaMemsetAsync(P->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT * nbox, s);
      for (int s0 = 0; s0 < nsteps; s0 += kChunk) {
        a.nsteps = std::min(kChunk, nsteps - s0);
        enqueue_bin(P, a, s);
        c0->launches += 5;
        for (auto& g : P->groups) {
          const int cand = g.block ? cand_of(g.block) : std::min(g.tried, 2);
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          cudaEventRecord(e0, s);
          launch_group(g.np, a, g.e_lo, g.e_hi, group_grid(P, g, cand), kBlocks[cand], s);
          cudaEventRecord(e1, s);
          c0->launches += 1;
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          if (!g.block) {
            g.ms[cand] = ms / std::max(a.nsteps, 1);
            if (++g.tried == 3) {
              int best = 0;
              for (int i = 1; i < 3; ++i)
                if (g.ms[i] < g.ms[best]) best = i;
              g.block = kBlocks[best];
            }
          }
        }
      }
    } else {
      if (!P->graph || P->graph_nsteps != nsteps || P->graph_dt != dt) {
        if (P->graph) cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
        cudaGraph_t g = nullptr;
        // capturing only records the work: nothing runs on P->cap
        cudaError_t e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaMemsetAsync(P->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT * nbox, P->cap);
          for (int s0 = 0; s0 < nsteps; s0 += kChunk) {
            a.nsteps = std::min(kChunk, nsteps - s0);
            enqueue_chunk(P, a, P->cap, true);
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
      }
      cudaError_t e = cudaGraphLaunch(P->graph, s);
      c0->launches += (5 + (int64_t)P->groups.size()) * ((nsteps + kChunk - 1) / kChunk);
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

extern "C" pt_status pt_batch_tuning(pt_ctx* ctx0, int32_t* np_out, int32_t* block_out,
                                     float* ms_out, int32_t max_groups, int32_t* ngroups) {
  if (!ctx0 || !ngroups) return PT_ERR_ARG;
  const pt_batch_plan* P = ctx0->batch;
  *ngroups = P ? (int32_t)P->groups.size() : 0;
  if (!P) return PT_OK;
  for (int i = 0; i < (int)P->groups.size() && i < max_groups; ++i) {
    const auto& g = P->groups[i];
    if (np_out) np_out[i] = g.np - 1;
    if (block_out) block_out[i] = g.block;
    if (ms_out)
      for (int k = 0; k < 3; ++k) ms_out[3 * i + k] = g.ms[k];
  }
  return PT_OK;
}
