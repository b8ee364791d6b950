// Edge-balanced expansion of a vertex list, shared by the shortest-path and betweenness kernels.
//
// Entry i of a list of vertices owns ceil(deg / FX_CHUNK) chunks of FX_CHUNK consecutive edges of
// its row; off[] is the exclusive scan of the chunk counts.  A warp takes one chunk at a time (a
// grid-stride loop over off[nent], read on the device), finds the chunk's entry by binary search
// in off[] and walks its edges with one lane per edge, so that a hub on the list is spread over
// many warps and short rows cost one chunk each.
#pragma once

#include "internal.cuh"

namespace lagr {

constexpr int FX_CHUNK = 128;  // edges per chunk: four steps of a warp

// chunk counts of list[0 .. nent): cnt[i] = ceil(deg(list[i]) / FX_CHUNK)
__global__ void fx_chunk_counts(const int32_t *__restrict__ list, int32_t nent, const int32_t *__restrict__ rowptr,
                                int32_t *__restrict__ cnt);

// the list entry that owns chunk c: the last i with off[i] <= c (off[0] = 0 <= c < off[nent])
__device__ __forceinline__ int32_t fx_entry_of(const int32_t *__restrict__ off, int32_t nent, int32_t c) {
  int32_t lo = 0, hi = nent - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Per-list work space: chunk counts, their offsets and the scan's scratch, sized for lists of up to
// `cap` entries.
struct FxSpace {
  int32_t *cnt = nullptr, *off = nullptr;
  int64_t *scan = nullptr;
  int64_t cap = 0;
};
int fx_alloc(FxSpace *fx, int64_t cap, cudaStream_t s, char *msg);
void fx_free(FxSpace *fx, cudaStream_t s);
// chunk counts and offsets of list[0 .. nent) (off[nent] = total chunks, on the device)
int fx_plan(FxSpace *fx, const int32_t *list, int32_t nent, const int32_t *rowptr, cudaStream_t s, char *msg);

}  // namespace lagr
