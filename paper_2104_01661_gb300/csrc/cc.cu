// Connected components by FastSV (Alg. 7, Sec. IV-F).
//
// The forest of parent pointers f starts as n singletons.  A round is the paper's five steps:
//   1. stochastic hooking: mngf(u) <min>= min over the neighbours v of gf(v) (the min.second mxv),
//      then f(x(u)) <min>= mngf(u) with x the parent list of the round's start;
//   2. aggressive hooking: f(u) <min>= mngf(u);
//   3. shortcutting: f(u) <min>= gf(u);
//   4. grandparents: x = f, gf(u) = f(f(u));
//   5. stop when nothing changed.
// Steps 1-3 are one pass over the row blocks of the CSR (the row plan shared with the other row
// kernels): a CTA stages its block's row pointers, folds the gathered gf(v) of every entry into a
// per-row minimum in shared memory, and applies the three hooks with atomicMin.  Rows too long for
// a block are cut into chunks whose CTAs fold into mngf directly; a small kernel hooks them after.
// Steps 4-5 are one element-wise pass.
//
// The hooks of one round are applied concurrently with atomicMin instead of one GraphBLAS call
// after the other.  Every value stored is a label taken from gf or mngf, labels only decrease, and
// f(u) <= u holds throughout, so any interleaving keeps a valid forest.  The loop stops after a
// round that changes neither f nor gf: such a state is a fixed point of all five steps, where
// f(u) = f(f(u)) (so f(u) = gf(u)) and f(u) <= f(v) for every edge {u,v}, i.e. f(u) is the smallest
// id of u's component -- the result Alg. 7 reaches, independent of the order of the hooks.
#include <climits>

#include "internal.cuh"

namespace lagr {
namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_RUN = 8;  // consecutive entries per thread in the row-block fold
constexpr int CC_ROUND_CAP_EXTRA = 64;  // rounds allowed beyond 2 log2(n) before giving up

__global__ void cc_init(int32_t n, int32_t *__restrict__ f, int32_t *__restrict__ gf, int32_t *__restrict__ mngf,
                        int32_t *__restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)i;
    f[u] = u;
    gf[u] = u;
    mngf[u] = u;
    x[u] = u;
  }
}

__device__ __forceinline__ void hook(int32_t u, int32_t m, const int32_t *__restrict__ gf,
                                     const int32_t *__restrict__ x, int32_t *__restrict__ f) {
  atomicMin(&f[x[u]], m);               // step 1: f(x(u)) <min>= mngf(u)
  atomicMin(&f[u], min(m, gf[u]));      // steps 2 and 3
}

// Steps 1-3.  CTAs [0, nblk) take the row blocks (a block that is one heavy row is skipped), CTAs
// [nblk, nblk + nhc) the chunks of the heavy rows.
__global__ void __launch_bounds__(CC_THREADS)
    cc_hook(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const int32_t *__restrict__ blk,
            int32_t nblk, const uint8_t *__restrict__ hblk, const int32_t *__restrict__ heavy,
            const int32_t *__restrict__ hc_off, const int32_t *__restrict__ hc_row, int32_t hchunk,
            const int32_t *__restrict__ gf, int32_t *__restrict__ mngf, const int32_t *__restrict__ x,
            int32_t *__restrict__ f) {
  __shared__ int32_t rp[ROW_UNITS + 1];
  __shared__ int32_t rmin[ROW_UNITS];
  __shared__ int32_t red[32];
  if ((int32_t)blockIdx.x >= nblk) {  // one chunk of a heavy row: fold into mngf
    const int32_t c = blockIdx.x - nblk;
    const int32_t h = hc_row[c];
    const int32_t i = heavy[h];
    const int32_t b = rowptr[i] + (c - hc_off[h]) * hchunk;
    const int32_t e = min(rowptr[i + 1], b + hchunk);
    int32_t m = INT_MAX;
    for (int32_t k = b + threadIdx.x; k < e; k += blockDim.x) m = min(m, __ldg(&gf[__ldg(&colidx[k])]));
    m = __reduce_min_sync(LAGR_FULL_MASK, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INT_MAX;
      m = __reduce_min_sync(LAGR_FULL_MASK, m);
      if (threadIdx.x == 0) atomicMin(&mngf[i], m);
    }
    return;
  }
  if (hblk[blockIdx.x]) return;
  const int32_t r0 = blk[blockIdx.x], r1 = blk[blockIdx.x + 1];
  const int32_t nr = r1 - r0;
  for (int32_t q = threadIdx.x; q <= nr; q += blockDim.x) rp[q] = rowptr[r0 + q];
  for (int32_t q = threadIdx.x; q < nr; q += blockDim.x) rmin[q] = mngf[r0 + q];
  __syncthreads();
  // each thread folds CC_RUN consecutive entries per pass: one row search for the first, then the
  // rows advance with the entries, and a row's minimum enters rmin once per run
  const int32_t e0 = rp[0], e1 = rp[nr];
  for (int32_t k0 = e0 + threadIdx.x * CC_RUN; k0 < e1; k0 += blockDim.x * CC_RUN) {
    int32_t lo = 0, hi = nr - 1;  // the row of entry k0: the last q with rp[q] <= k0
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= k0) lo = mid; else hi = mid - 1;
    }
    const int32_t kend = min(e1, k0 + CC_RUN);
    int32_t g[CC_RUN];
#pragma unroll
    for (int j = 0; j < CC_RUN; j++) g[j] = k0 + j < kend ? __ldg(&gf[__ldg(&colidx[k0 + j])]) : INT_MAX;
    int32_t q = lo, m = INT_MAX, rend = rp[lo + 1];
#pragma unroll
    for (int j = 0; j < CC_RUN; j++) {
      if (k0 + j >= kend) break;
      while (k0 + j >= rend) {  // the row ended: fold its part, step over empty rows
        if (m != INT_MAX) atomicMin(&rmin[q], m);
        m = INT_MAX;
        q++;
        rend = rp[q + 1];
      }
      m = min(m, g[j]);
    }
    if (m != INT_MAX) atomicMin(&rmin[q], m);
  }
  __syncthreads();
  for (int32_t q = threadIdx.x; q < nr; q += blockDim.x) {
    const int32_t u = r0 + q;
    const int32_t m = rmin[q];
    mngf[u] = m;
    hook(u, m, gf, x, f);
  }
}

// the hooks of the heavy rows, once their chunks are folded into mngf
__global__ void cc_hook_heavy(const int32_t *__restrict__ heavy, int32_t nheavy, const int32_t *__restrict__ mngf,
                              const int32_t *__restrict__ gf, const int32_t *__restrict__ x, int32_t *__restrict__ f) {
  const int32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nheavy) {
    const int32_t u = heavy[h];
    hook(u, mngf[u], gf, x, f);
  }
}

// Steps 4-5: x = f, gf = f(x); *changed = 1 when f moved since the round's start or gf changed
__global__ void cc_shortcut(int32_t n, const int32_t *__restrict__ f, int32_t *__restrict__ x, int32_t *__restrict__ gf,
                            int64_t *__restrict__ changed) {
  bool ch = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t fu = f[i];
    ch |= fu != x[i];
    x[i] = fu;
    const int32_t g = f[fu];
    ch |= g != gf[i];
    gf[i] = g;
  }
  if (__any_sync(LAGR_FULL_MASK, ch) && (threadIdx.x & 31) == 0) *changed = 1;
}

}  // namespace
}  // namespace lagr

using namespace lagr;

extern "C" int lagr_connected_components(int32_t *component, int32_t *rounds, lagr_graph G, void *stream,
                                         char *msg) {
  if (!component) {
    set_msg(msg, "component is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(check_graph_arg(G, msg));
  if (G->kind != LAGR_UNDIRECTED) {
    set_msg(msg, "FastSV needs an undirected graph");
    return LAGR_ERR_INVALID_GRAPH;
  }
  if (rounds) *rounds = 0;
  const int32_t n = G->n;
  if (n == 0) {
    clear_msg(msg);
    return LAGR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  LAGR_TRY(lagr_property_AT(G, s, msg));  // undirected: A' aliases A, so the row plan is shared
  LAGR_TRY(row_plan(&P->pr_at, G->rowptr, n, s, msg));
  const RowPlan &pl = P->pr_at;
  Temp<int32_t> gf(s), mngf(s), x(s);
  LAGR_TRY(gf.alloc(n, msg, "grandparents"));
  LAGR_TRY(mngf.alloc(n, msg, "minimum neighbour grandparents"));
  LAGR_TRY(x.alloc(n, msg, "parent list"));
  int32_t *f = component;
  int64_t *changed = P->dscal + SC_COUNT0;
  cc_init<<<grid_for(n, CC_THREADS), CC_THREADS, 0, s>>>(n, f, gf.p, mngf.p, x.p);
  LAGR_LAUNCH_CHECK();
  int cap = CC_ROUND_CAP_EXTRA;
  for (int32_t v = n; v > 1; v >>= 1) cap += 2;
  int32_t k = 0;
  for (;;) {
    if (k >= cap) {
      set_msg(msg, "FastSV did not settle within %d rounds", cap);
      return LAGR_ERR_TIMEOUT;
    }
    k++;
    LAGR_CUDA_TRY(cudaMemsetAsync(changed, 0, sizeof(int64_t), s));
    cc_hook<<<pl.nblk + pl.nhc, CC_THREADS, 0, s>>>(G->rowptr, G->colidx, pl.blk, pl.nblk, pl.hblk, pl.heavy,
                                                    pl.hc_off, pl.hc_row, pl.hchunk, gf.p, mngf.p, x.p, f);
    if (pl.nheavy > 0)
      cc_hook_heavy<<<(pl.nheavy + CC_THREADS - 1) / CC_THREADS, CC_THREADS, 0, s>>>(pl.heavy, pl.nheavy, mngf.p,
                                                                                    gf.p, x.p, f);
    cc_shortcut<<<grid_for(n, CC_THREADS), CC_THREADS, 0, s>>>(n, f, x.p, gf.p, changed);
    LAGR_LAUNCH_CHECK();
    int64_t h = 0;
    LAGR_TRY(fetch_to_host(&h, changed, sizeof(int64_t), s, msg));
    if (h == 0) break;
  }
  G->last_iters = k;
  if (rounds) *rounds = k;
  clear_msg(msg);
  return LAGR_OK;
}
