// pt_bin.cu -- counting sort of particle indices by owning element (histogram,
// exclusive scan, scatter).  Gives the element-ordered visiting order of the
// push and the per-element segments of the segmented deposition.
#include <cuda_runtime.h>

#include <cstdint>

#include "pt_bin.h"

namespace pt {

__global__ void k_hist(const int* __restrict__ elem, int64_t n, int nelem, int* counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int e = elem[i];
    if (e < 0 || e >= nelem) e = nelem;  // out-of-range owners go to a trailing bin
    atomicAdd(counts + e, 1);
  }
}

// exclusive scan of 1024-element blocks; block totals to bsum
__global__ void __launch_bounds__(1024) k_scan_block(const int* __restrict__ in, int* out,
                                                     int* bsum, int n) {
  __shared__ int ws[32];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int incl = x + (w > 0 ? ws[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

// exclusive scan of the block totals by one block (sequential over chunks);
// writes the grand total to *total
__global__ void __launch_bounds__(1024) k_scan_sums(int* bsum, int nb, int* total) {
  __shared__ int ws[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int s = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? ws[w - 1] : 0) + carry;
    if (i < nb) bsum[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int* out, const int* __restrict__ bsum, int n, int* cursor) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) {
    const int o = out[i] + bsum[blockIdx.x];
    out[i] = o;
    cursor[i] = o;
  }
}

__global__ void k_scatter(const int* __restrict__ elem, int64_t n, int nelem, int* cursor,
                          int* perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int e = elem[i];
    if (e < 0 || e >= nelem) e = nelem;
    const int pos = atomicAdd(cursor + e, 1);
    perm[pos] = (int)i;
  }
}

// Sorts a[0..m) ascending in place by a bitonic network in its "flip" form:
// for each block size k, element i is compared with i ^ (k - 1) and then with
// i ^ j for j = k/4 .. 1, the smaller value always going to the lower index.
// Missing elements beyond m act as +infinity, so pairs reaching past m are
// skipped and m need not be a power of two.  Called by a whole block.
__device__ void block_bitonic(int* a, unsigned m) {
  unsigned M = 1;
  while (M < m) M <<= 1;
  for (unsigned k = 2; k <= M && k != 0; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      const unsigned mask = (j == (k >> 1)) ? k - 1 : j;
      for (unsigned i = threadIdx.x; i < M; i += blockDim.x) {
        const unsigned l = i ^ mask;
        if (l > i && l < m) {
          const int x = a[i], y = a[l];
          if (x > y) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int kSortSmem = 4096;  // segments up to this size are sorted in shared memory

__global__ void __launch_bounds__(256) k_sort_segments(const int* __restrict__ perm,
                                                       const int* __restrict__ offs, int nbins,
                                                       int* out) {
  __shared__ int sh[kSortSmem];
  for (int e = blockIdx.x; e < nbins; e += gridDim.x) {
    const int beg = offs[e], m = offs[e + 1] - beg;
    if (m <= 0) continue;
    if (m <= kSortSmem) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) sh[i] = perm[beg + i];
      __syncthreads();
      block_bitonic(sh, (unsigned)m);
      for (int i = threadIdx.x; i < m; i += blockDim.x) out[beg + i] = sh[i];
    } else {
      // large segment: the same network on the output in global memory (the
      // block's writes are visible to its threads after __syncthreads)
      for (int i = threadIdx.x; i < m; i += blockDim.x) out[beg + i] = perm[beg + i];
      __syncthreads();
      block_bitonic(out + beg, (unsigned)m);
    }
    __syncthreads();
  }
}

int sort_segments(const int* perm, const int* offs, int nelem, int* out, int nsm,
                  cudaStream_t s) {
  const int nbins = nelem + 1;
  const int g = nbins < nsm * 8 ? nbins : nsm * 8;
  k_sort_segments<<<g > 0 ? g : 1, 256, 0, s>>>(perm, offs, nbins, out);
  return (int)cudaGetLastError();
}

size_t bin_scratch_ints(int nelem) {
  const int nbins = nelem + 1;
  const int nb = (nbins + 1023) / 1024;
  // counts[nbins] | offs[nbins + 1] | cursor[nbins] | bsum[nb]
  return (size_t)nbins * 3 + 1 + nb;
}

void bin_layout(int nelem, int* scratch, BinLayout& L) {
  const int nbins = nelem + 1;
  L.nbins = nbins;
  L.nb = (nbins + 1023) / 1024;
  L.counts = scratch;
  L.offs = L.counts + nbins;
  L.cursor = L.offs + nbins + 1;
  L.bsum = L.cursor + nbins;
}

void bin_scan(const BinLayout& L, cudaStream_t s) {
  k_scan_block<<<L.nb, 1024, 0, s>>>(L.counts, L.offs, L.bsum, L.nbins);
  k_scan_sums<<<1, 1024, 0, s>>>(L.bsum, L.nb, L.offs + L.nbins);
  k_scan_add<<<L.nb, 1024, 0, s>>>(L.offs, L.bsum, L.nbins, L.cursor);
}

int bin_by_element(const int* elem, int64_t n, int nelem, int* scratch, int* perm, int** offs_out,
                   int nsm, cudaStream_t s) {
  BinLayout L;
  bin_layout(nelem, scratch, L);
  if (offs_out) *offs_out = L.offs;
  cudaMemsetAsync(L.counts, 0, sizeof(int) * L.nbins, s);
  const int g = (int)((n + 255) / 256 < (int64_t)nsm * 8 ? (n + 255) / 256 : (int64_t)nsm * 8);
  if (n > 0) k_hist<<<g > 0 ? g : 1, 256, 0, s>>>(elem, n, nelem, L.counts);
  bin_scan(L, s);
  if (n > 0) k_scatter<<<g > 0 ? g : 1, 256, 0, s>>>(elem, n, nelem, L.cursor, perm);
  return (int)cudaGetLastError();
}

}  // namespace pt
