// Edge-balanced expansion of a vertex list (see frontier.cuh).
#include "frontier.cuh"

namespace lagr {

__global__ void fx_chunk_counts(const int32_t *__restrict__ list, int32_t nent, const int32_t *__restrict__ rowptr,
                                int32_t *__restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nent; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    const int32_t d = rowptr[v + 1] - rowptr[v];
    cnt[i] = (d + FX_CHUNK - 1) / FX_CHUNK;
  }
}

int fx_alloc(FxSpace *fx, int64_t cap, cudaStream_t s, char *msg) {
  if (cap < 1) cap = 1;
  LAGR_TRY(alloc_n(&fx->cnt, (size_t)cap, s, msg, "chunk counts"));
  LAGR_TRY(alloc_n(&fx->off, (size_t)cap + 1, s, msg, "chunk offsets"));
  LAGR_TRY(alloc_n(&fx->scan, (size_t)scan_scratch_len(cap), s, msg, "chunk scan scratch"));
  fx->cap = cap;
  return LAGR_OK;
}

void fx_free(FxSpace *fx, cudaStream_t s) {
  dev_free(fx->cnt, s);
  dev_free(fx->off, s);
  dev_free(fx->scan, s);
  *fx = FxSpace();
}

int fx_plan(FxSpace *fx, const int32_t *list, int32_t nent, const int32_t *rowptr, cudaStream_t s, char *msg) {
  if (nent > fx->cap) {
    set_msg(msg, "internal: list of %d entries exceeds its work space (%lld)", nent, (long long)fx->cap);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (nent > 0) fx_chunk_counts<<<grid_for(nent, 256), 256, 0, s>>>(list, nent, rowptr, fx->cnt);
  LAGR_LAUNCH_CHECK();
  return exclusive_scan(fx->cnt, fx->off, nent, s, msg, fx->scan);
}

}  // namespace lagr
