// pt_ctx.h -- the library-owned context behind the opaque pt_ctx handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pt.h"
#include "pt_internal.h"

struct pt_mlp_state;
struct pt_batch_plan;

struct pt_ctx {
  int dev = 0;
  int nsm = 1;
  cudaStream_t stream = nullptr;
  pt_config cfg{};
  // mesh
  int nelem = 0, ngeo = 0, g = 0, ncurved = 0;
  double* d_xg64 = nullptr;
  float* d_xg32 = nullptr;
  float* d_xg32lo = nullptr;
  double* d_ce = nullptr;
  float* d_tri = nullptr;
  int* d_tmask = nullptr;
  int* d_fnbr = nullptr;
  int* d_finfo = nullptr;
  float* d_slab = nullptr;
  double* d_bil = nullptr;
  float* d_bil32 = nullptr;
  double* d_shift = nullptr;
  int* d_mort = nullptr;  // [max(M,1)][9] mortar rows
  int nmortar = 0;
  unsigned long long* d_stats = nullptr;
  std::vector<void*> allocs;
  // fluid
  int N = -1, node_type = 0;
  const void* U = nullptr;
  double sn[PT_MAXN] = {0}, sw[PT_MAXN] = {0}, sq[PT_MAXN] = {0};
  // scratch (binning), permutation, host-call staging
  int* d_scratch = nullptr;
  size_t scratch_ints = 0;
  int* d_perm = nullptr;
  int64_t perm_cap = 0;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  // per-particle sources of the two-pass segmented deposition, and the
  // element-sorted order with each element's particles in index order
  float4* d_src = nullptr;
  int64_t src_cap = 0;
  int* d_perm2 = nullptr;
  // learned guess
  pt_mlp_state* mlp = nullptr;
  bool mlp_ready = false;
  float* d_mlp_pre = nullptr;
  // background grid of pt_find_element, built on its first call
  bool grid_ready = false;
  int* d_cell_start = nullptr;
  int* d_cell_elem = nullptr;
  double grid_lo[3] = {0, 0, 0}, grid_ih[3] = {0, 0, 0};
  int grid_dims[3] = {0, 0, 0};
  // batched push plan (pt_push_batch called with this context first)
  pt_batch_plan* batch = nullptr;
  // particle state of the staged schedule (sorted order), grown on demand
  void* d_state = nullptr;
  int64_t state_cap = 0;
  // pt_push_stage: the next stage expected (0: none open), the particles and
  // time step of the open sequence
  int stage_next = 0;
  pt_particles stage_p{};
  double stage_dt = 0.0;
  // kernels queued since the last pt_launch_count
  int64_t launches = 0;
  // kernel timing (pt_profile)
  bool profile = false;
  // event pairs per kernel kind: 0 the push (a whole chunk of the staged
  // schedule, the resident kernel), 1 stage kernels, 2 learned start, 3 exact
  // tracking (staged schedule)
  std::vector<cudaEvent_t> ev_free, ev_used[4];
  std::string err = "no error";
};

void pt_mlp_release(pt_ctx* c);
void pt_batch_release(pt_ctx* c);
pt_status pt_push_impl(pt_ctx* c, const pt_particles* p, int32_t nsteps, double dt, pt_stats* out);
