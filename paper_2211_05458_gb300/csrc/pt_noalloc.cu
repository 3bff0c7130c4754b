// pt_noalloc.cu -- pt_deposit_noalloc: the two-way coupling deposition without
// any device allocation.  Its scratch (the element binning counters and two
// particle permutations) lives in one fixed-size array in device memory that
// the library reserves at load time; every call reuses it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "pt_bin.h"
#include "pt_ctx.h"
#include "pt_internal.h"

// limits of the fixed scratch (sizes the array below)
#define PT_NOALLOC_MAX_ELEMS (1 << 17)      // 131072 elements
#define PT_NOALLOC_MAX_PARTICLES (1 << 20)  // 1048576 particles

namespace {
constexpr size_t kBinInts = 3 * ((size_t)PT_NOALLOC_MAX_ELEMS + 1) + 1 +
                            ((size_t)PT_NOALLOC_MAX_ELEMS + 1 + 1023) / 1024;
// binning counters | element-sorted order | the same with each element's
// particles in index order
constexpr size_t kScratchInts = kBinInts + 2 * (size_t)PT_NOALLOC_MAX_PARTICLES;
}  // namespace

// The scratch.  In host code this name is only a stand-in for the symbol, not
// a device address: the address is obtained below with cudaGetSymbolAddress.
static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int* g_dev_ptr[kMaxDevices] = {nullptr};
}  // namespace

DevMesh pt_dev_mesh(const pt_ctx* c);
void pt_fill_consts(const pt_ctx* c, DevConsts& k);
pt_status pt_validate_particles(pt_ctx* c, const pt_particles* p);

// Device address of the scratch in the current context.  A __device__ array
// has its own address in every CUDA context (and again after a device reset),
// so the address is looked up again on every call that is not being captured
// into a graph; a captured call uses the address of the last call outside
// capture on the same device.
static cudaError_t scratch_ptr(cudaStream_t stream, int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    int* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  } else if (!g_dev_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

extern "C" pt_status pt_deposit_noalloc(pt_ctx* c, const pt_particles* p, int32_t mode,
                                        float* S) {
  if (!c) return PT_ERR_ARG;
  if (c->N < 0 || !c->U) {
    c->err = "pt_deposit_noalloc: pt_set_fluid was not called";
    return PT_ERR_STATE;
  }
  const pt_status vs = pt_validate_particles(c, p);
  if (vs != PT_OK) return vs;
  if (mode & ~(PT_DEPOSIT_SEGMENTED | PT_DEPOSIT_NEAREST)) {
    c->err = "pt_deposit_noalloc: mode must be PT_DEPOSIT_ATOMIC or PT_DEPOSIT_SEGMENTED, "
             "optionally | PT_DEPOSIT_NEAREST";
    return PT_ERR_ARG;
  }
  if (!S) {
    c->err = "pt_deposit_noalloc: S is NULL";
    return PT_ERR_ARG;
  }
  if (c->nelem > PT_NOALLOC_MAX_ELEMS || p->n > PT_NOALLOC_MAX_PARTICLES) {
    c->err = "pt_deposit_noalloc: at most " + std::to_string(PT_NOALLOC_MAX_ELEMS) +
             " elements and " + std::to_string(PT_NOALLOC_MAX_PARTICLES) +
             " particles (fixed scratch); use pt_deposit for larger problems";
    return PT_ERR_ARG;
  }
  int* scratch = nullptr;
  cudaError_t e = scratch_ptr(c->stream, &scratch);
  if (e != cudaSuccess) {
    c->err = std::string("pt_deposit_noalloc: scratch lookup: ") + cudaGetErrorString(e);
    return PT_ERR_CUDA;
  }
  int* perm = scratch + kBinInts;
  int* sorted = perm + PT_NOALLOC_MAX_PARTICLES;
  const int np = c->N + 1;
  const size_t n3 = (size_t)np * np * np;
  const int64_t n = p->n;
  // the binning clears its own counters before use
  int* offs = nullptr;
  int rc = pt::bin_by_element(p->elem, n, c->nelem, scratch, perm, &offs, c->nsm, c->stream);
  if (rc) {
    c->err = std::string("pt_deposit_noalloc: binning: ") + cudaGetErrorString((cudaError_t)rc);
    return PT_ERR_CUDA;
  }
  DepositArgs a;
  a.m = pt_dev_mesh(c);
  pt_fill_consts(c, a.k);
  a.p = {n, p->x, p->v, p->d, p->elem, p->hits, p->status};
  a.U = c->U;
  a.perm = perm;
  a.offs = offs;
  a.S = S;
  a.src = nullptr;
  const bool f64 = c->cfg.precision == PT_FP64;
  if (!(mode & PT_DEPOSIT_SEGMENTED)) {
    e = cudaMemsetAsync(S, 0, sizeof(float) * 4 * n3 * c->nelem, c->stream);
    if (e != cudaSuccess) {
      c->err = std::string("pt_deposit_noalloc: ") + cudaGetErrorString(e);
      return PT_ERR_CUDA;
    }
    if (n == 0) return PT_OK;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 16);
    rc = pt::launch_deposit(c->g, f64, np, mode, a, grid, 128, c->stream);
  } else {
    // each element's particles in index order: the summation order
    rc = pt::sort_segments(perm, offs, c->nelem, sorted, c->nsm, c->stream);
    if (rc) {
      c->err = std::string("pt_deposit_noalloc: segment sort: ") +
               cudaGetErrorString((cudaError_t)rc);
      return PT_ERR_CUDA;
    }
    a.perm = sorted;
    const int grid = std::min(c->nelem, c->nsm * 32);
    rc = pt::launch_deposit(c->g, f64, np, mode, a, grid, 256, c->stream);
  }
  if (rc) {
    c->err = std::string("pt_deposit_noalloc: launch: ") + cudaGetErrorString((cudaError_t)rc);
    return PT_ERR_CUDA;
  }
  return PT_OK;
}
