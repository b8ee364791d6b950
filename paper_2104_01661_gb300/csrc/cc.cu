// Connected components by FastSV (Alg. 7, Sec. IV-F).
//
// The forest of parent pointers f starts as n singletons.  A round is the paper's five steps:
//   1. stochastic hooking: mngf(u) <min>= min over the neighbours v of gf(v) (the min.second mxv),
//      then f(x(u)) <min>= mngf(u) with x the parent list of the round's start;
//   2. aggressive hooking: f(u) <min>= mngf(u);
//   3. shortcutting: f(u) <min>= gf(u);
//   4. grandparents: x = f, gf(u) = f(f(u));
//   5. stop when nothing changed.
// Steps 1-3 are one pass over the fine row blocks of the CSR (the plan shared with the PageRank
// gather): a warp stages its block's row pointers, folds the gathered gf(v) of every entry into a
// per-row minimum in its shared memory, and applies the three hooks with atomicMin.  Rows too long
// for a block are cut into chunks whose warps fold into mngf directly; a small kernel hooks them
// after.
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

// The hooks.  Most vertices of a component share one root, so an unconditional atomicMin on
// f(x(u)) would serialise millions of atomics on one word; a hook that cannot lower the value (read
// first, through L2) is skipped.  A stale read only costs the atomic.
__device__ __forceinline__ void hook(int32_t u, int32_t m, const int32_t *__restrict__ gf,
                                     const int32_t *__restrict__ x, int32_t *__restrict__ f) {
  const int32_t p = x[u];
  if (m < __ldcg(&f[p])) atomicMin(&f[p], m);  // step 1: f(x(u)) <min>= mngf(u)
  const int32_t mm = min(m, gf[u]);
  if (mm < __ldcg(&f[u])) atomicMin(&f[u], mm);  // steps 2 and 3
}

// Steps 1-3 with persistent warps: every warp takes work items from one queue -- first the chunks
// of the rows longer than FINE_HEAVY (a warp folds its chunk into mngf), then the row blocks of the
// fine plan (at most FINE_UNITS units, so at most FINE_UNITS rows and FINE_UNITS + FINE_HEAVY
// entries).  A warp stages its block's row pointers and row minima in its own shared memory, folds
// runs of CC_RUN entries per lane into them and hooks its rows; there is no CTA barrier.
constexpr int CCW_WARPS = 4;  // 32.8 KB of staged rows per CTA
__global__ void __launch_bounds__(CCW_WARPS * 32)
    cc_hook_warp(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                 const int32_t *__restrict__ blk, int32_t nblk, const uint8_t *__restrict__ hblk,
                 const int32_t *__restrict__ heavy, const int32_t *__restrict__ hc_off,
                 const int32_t *__restrict__ hc_row, int32_t nhc, int32_t hchunk, const int32_t *__restrict__ gf,
                 int32_t *__restrict__ mngf, const int32_t *__restrict__ x, int32_t *__restrict__ f,
                 int64_t *__restrict__ queue) {
  __shared__ int32_t s_rp[CCW_WARPS][FINE_UNITS + 2];
  __shared__ int32_t s_min[CCW_WARPS][FINE_UNITS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t *rp = s_rp[warp], *rmin = s_min[warp];
  const int32_t nitems = nhc + nblk;
  for (;;) {
    int32_t it = 0;
    if (lane == 0) it = (int32_t)atomicAdd((unsigned long long *)queue, 1ull);
    it = __shfl_sync(LAGR_FULL_MASK, it, 0);
    if (it >= nitems) break;
    if (it < nhc) {  // a chunk of a heavy row
      const int32_t h = hc_row[it];
      const int32_t i = heavy[h];
      const int32_t b = rowptr[i] + (it - hc_off[h]) * hchunk;
      const int32_t e = min(rowptr[i + 1], b + hchunk);
      int32_t m = INT_MAX;
      for (int32_t k = b + lane; k < e; k += 32) m = min(m, __ldg(&gf[__ldg(&colidx[k])]));
      m = __reduce_min_sync(LAGR_FULL_MASK, m);
      if (lane == 0) atomicMin(&mngf[i], m);
      continue;
    }
    const int32_t wb = it - nhc;
    if (hblk[wb]) continue;  // a block that is one heavy row: its chunks are items of their own
    const int32_t r0 = blk[wb], r1 = blk[wb + 1];
    const int32_t nr = r1 - r0;
    for (int32_t q = lane; q <= nr; q += 32) rp[q] = rowptr[r0 + q];
    for (int32_t q = lane; q < nr; q += 32) rmin[q] = mngf[r0 + q];
    __syncwarp();
    const int32_t e0 = rp[0], e1 = rp[nr];
    for (int32_t k0 = e0 + lane * CC_RUN; k0 < e1; k0 += 32 * CC_RUN) {
      int32_t lo = 0, hi = nr - 1;  // the row of entry k0
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
        while (k0 + j >= rend) {
          if (m != INT_MAX) atomicMin(&rmin[q], m);
          m = INT_MAX;
          q++;
          rend = rp[q + 1];
        }
        m = min(m, g[j]);
      }
      if (m != INT_MAX) atomicMin(&rmin[q], m);
    }
    __syncwarp();
    for (int32_t q = lane; q < nr; q += 32) {
      const int32_t u = r0 + q;
      const int32_t m = rmin[q];
      mngf[u] = m;
      hook(u, m, gf, x, f);
    }
    __syncwarp();  // the staged arrays are rewritten by the warp's next block
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
  LAGR_TRY(row_plan(&P->pr_fwd, G->at_rowptr, n, s, msg, FINE_UNITS, FINE_HEAVY, FINE_HCHUNK));
  const RowPlan &pl = P->pr_fwd;
  const int hgrid = resident_ctas((const void *)cc_hook_warp, CCW_WARPS * 32, 0);
  int64_t *queue = P->dscal + SC_COUNT1;
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
    static_assert(SC_COUNT1 == SC_COUNT0 + 1, "slot layout");
    LAGR_CUDA_TRY(cudaMemsetAsync(changed, 0, 2 * sizeof(int64_t), s));  // the flag and the work queue
    cc_hook_warp<<<hgrid, CCW_WARPS * 32, 0, s>>>(G->rowptr, G->colidx, pl.blk, pl.nblk, pl.hblk, pl.heavy,
                                                 pl.hc_off, pl.hc_row, pl.nhc, pl.hchunk, gf.p, mngf.p, x.p, f,
                                                 queue);
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
