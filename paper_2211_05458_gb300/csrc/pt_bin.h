// pt_bin.h -- element binning (counting sort) used by the push and deposition.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pt {
// layout of the binning scratch: counts[nbins] | offs[nbins + 1] | cursor[nbins] | bsum[nb]
struct BinLayout {
  int nbins, nb;
  int *counts, *offs, *cursor, *bsum;
};
void bin_layout(int nelem, int* scratch, BinLayout& L);
// exclusive scan of L.counts into L.offs (and L.cursor); L.offs[nbins] = total
void bin_scan(const BinLayout& L, cudaStream_t s);
// ints of scratch bin_by_element needs for nelem elements
size_t bin_scratch_ints(int nelem);
// perm[n] receives particle indices sorted by elem (order within an element
// unspecified); *offs_out points into scratch at offs[nelem + 2]: element e's
// particles are perm[offs[e] .. offs[e+1]); bin nelem holds invalid owners.
int bin_by_element(const int* elem, int64_t n, int nelem, int* scratch, int* perm, int** offs_out,
                   int nsm, cudaStream_t s);
// out[offs[e] .. offs[e+1]) = perm[offs[e] .. offs[e+1]) in increasing order,
// for every element e < nelem (and the trailing bin): the element-sorted order
// with each element's particles in index order.  O(m log^2 m) work per
// segment of m particles (one block per segment); perm and out must differ.
int sort_segments(const int* perm, const int* offs, int nelem, int* out, int nsm, cudaStream_t s);
}  // namespace pt
