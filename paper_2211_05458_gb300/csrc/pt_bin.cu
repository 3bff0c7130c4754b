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
