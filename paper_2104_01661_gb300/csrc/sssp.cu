// Single-source shortest paths by delta-stepping (Alg. 5, Sec. IV-D) over min.plus in float32.
//
// Alg. 5 splits A into light (0 < A <= delta) and heavy (A > delta) entries and settles the
// vertices bucket by bucket, bucket i holding the tentative distances in [i delta, (i+1) delta):
// light edges are relaxed from the bucket's frontier until no distance in the bucket improves,
// then the heavy edges of every vertex the bucket settled are relaxed once.  Here a relaxation is
// the float32 sum t(u) + A(u,v) and an atomicMin on the bits of t(v) (non-negative floats order
// like their bit patterns, +inf above every finite value), fused with the selects that build the
// next frontier: a vertex whose distance drops to a value inside the current bucket joins the
// next frontier once (a per-vertex stamp).  The light and heavy splits are not materialised; the
// relax kernels test each entry's value.  Buckets that hold no vertex are skipped (the next
// bucket is the one of the smallest distance beyond the current bucket), which changes no result.
//
// Results do not depend on the order of the relaxations: the distances reached are the least
// fixed point of t(v) = min(t(v), t(u) + A(u,v)) with float32 sums (every sum is rounded to
// nearest, so t(u) + A(u,v) >= t(u) for A > 0, and each relaxation only lowers a distance towards
// that fixed point), the float32 length of a shortest path.
#include "frontier.cuh"

namespace lagr {
namespace {

constexpr int SP_THREADS = 256;
constexpr int32_t SP_INF_BITS = 0x7f800000;  // +inf

enum SpSlot {
  SP_NQ = 0,    // entries appended to the next light frontier
  SP_NE = 1,    // entries of the settled list of the bucket
  SP_TMIN = 2,  // bits of the smallest distance beyond the current bucket
  SP_CUR = 3,   // the bucket being settled
  SP_NSLOT = 4
};

// the bucket of a distance, floor(t / delta), as a float32 product with 1/delta (GB300's float64
// division is slow, and the buckets only order the work: any monotone bucketing gives the same
// distances, as long as every kernel uses the same one)
__device__ __forceinline__ long long bucket_of(float t, float inv_delta) {
  return (long long)fminf(t * inv_delta, 4.0e18f);  // (t >= 0 and finite here; clamped below 2^63)
}

__global__ void sp_init(int32_t n, int32_t src, int32_t *__restrict__ tbits, int32_t *__restrict__ qst,
                        int32_t *__restrict__ est, int32_t *__restrict__ q, int64_t *__restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    tbits[i] = i == src ? 0 : SP_INF_BITS;
    qst[i] = -1;
    est[i] = -1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    q[0] = src;
    for (int k = 0; k < SP_NSLOT; k++) cnt[k] = 0;
  }
}

// the bucket's settled set e: every vertex of the light frontier, listed once per bucket
__global__ void sp_settle(const int32_t *__restrict__ list, int32_t nent, int32_t bseq, int32_t *__restrict__ est,
                          int32_t *__restrict__ elist, int64_t *__restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nent; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    if (atomicExch(&est[u], bseq) != bseq)
      elist[atomicAdd((unsigned long long *)&cnt[SP_NE], 1ull)] = u;
  }
}

// Relax the light (LIGHT) or heavy edges of the vertices of list[0 .. nent), one warp per chunk.
// Light relaxations that lower a distance into bucket `cur` append the vertex to qnext (once per
// step: stamp `step`).
template <bool LIGHT>
__global__ void __launch_bounds__(SP_THREADS)
    sp_relax(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const float *__restrict__ val,
             const int32_t *__restrict__ list, int32_t nent, const int32_t *__restrict__ off, float delta,
             float inv_delta, int32_t *__restrict__ tbits, long long cur, int32_t step, int32_t *__restrict__ qst,
             int32_t *__restrict__ qnext, int64_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = nent > 0 ? off[nent] : 0;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int32_t i = fx_entry_of(off, nent, (int32_t)c);
    const int32_t u = list[i];
    const float tu = __int_as_float(__ldcg(&tbits[u]));
    const int32_t b = rowptr[u] + ((int32_t)c - off[i]) * FX_CHUNK;
    const int32_t e = min(rowptr[u + 1], b + FX_CHUNK);
    // the chunk's (up to) four steps of 32 edges: weights and targets loaded first, then the
    // targets' distances, so that each kind of load has four in flight per lane
    constexpr int STEPS = FX_CHUNK / 32;
    float w[STEPS];
    int32_t v[STEPS], tv[STEPS];
#pragma unroll
    for (int q = 0; q < STEPS; q++) {
      const int32_t k = b + lane + 32 * q;
      w[q] = k < e ? __ldg(&val[k]) : -1.0f;  // -1: in neither class
      v[q] = k < e ? __ldg(&colidx[k]) : 0;
    }
#pragma unroll
    for (int q = 0; q < STEPS; q++) {
      const bool in = LIGHT ? (w[q] > 0.0f && w[q] <= delta) : (w[q] > delta);
      tv[q] = in ? __ldcg(&tbits[v[q]]) : INT32_MIN;  // INT32_MIN: nothing to relax
    }
#pragma unroll
    for (int q = 0; q < STEPS; q++) {
      if (tv[q] == INT32_MIN) continue;
      const float cand = __fadd_rn(tu, w[q]);
      const int32_t cb = __float_as_int(cand);
      if (cb >= tv[q]) continue;  // a stale read only costs the atomic below
      const int32_t old = atomicMin(&tbits[v[q]], cb);
      if (LIGHT && cb < old && bucket_of(cand, inv_delta) == cur && atomicExch(&qst[v[q]], step) != step)
        qnext[atomicAdd((unsigned long long *)&cnt[SP_NQ], 1ull)] = v[q];
    }
  }
}

// before the search for the next bucket: no frontier, no settled vertex, no distance found yet
__global__ void sp_reset(int64_t *__restrict__ cnt) {
  cnt[SP_NQ] = 0;
  cnt[SP_NE] = 0;
  cnt[SP_TMIN] = SP_INF_BITS;
}

// the smallest distance beyond bucket `cur` (SP_TMIN holds +inf on entry)
__global__ void sp_next_min(int32_t n, const int32_t *__restrict__ tbits, long long cur, float inv_delta,
                            int64_t *__restrict__ cnt) {
  int32_t m = SP_INF_BITS;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t tb = tbits[i];
    if (tb < SP_INF_BITS && tb < m && bucket_of(__int_as_float(tb), inv_delta) > cur) m = tb;
  }
  m = __reduce_min_sync(LAGR_FULL_MASK, m);
  if ((threadIdx.x & 31) == 0 && m < SP_INF_BITS) atomicMin((long long *)&cnt[SP_TMIN], (long long)m);
}

// the next bucket (that of the smallest distance beyond the current one) as the new frontier
__global__ void sp_build(int32_t n, const int32_t *__restrict__ tbits, float inv_delta, int32_t step,
                         int32_t *__restrict__ qst, int32_t *__restrict__ q, int64_t *__restrict__ cnt) {
  const int64_t tmin = cnt[SP_TMIN];
  if (tmin >= SP_INF_BITS) return;
  const long long nb = bucket_of(__int_as_float((int32_t)tmin), inv_delta);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t tb = tbits[i];
    if (tb < SP_INF_BITS && bucket_of(__int_as_float(tb), inv_delta) == nb) {
      qst[i] = step;
      q[atomicAdd((unsigned long long *)&cnt[SP_NQ], 1ull)] = (int32_t)i;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt[SP_CUR] = nb;
}

}  // namespace
}  // namespace lagr

using namespace lagr;

extern "C" int lagr_sssp(float *dist, int32_t *buckets, lagr_graph G, int32_t src, float delta, void *stream,
                         char *msg) {
  if (!dist) {
    set_msg(msg, "dist is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(check_graph_arg(G, msg));
  if (!G->val) {
    set_msg(msg, "shortest paths need edge values (G->val)");
    return LAGR_ERR_INVALID_VALUE;
  }
  if (src < 0 || src >= G->n) {
    set_msg(msg, "source %d out of range [0, %d)", src, G->n);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (!(delta > 0.0f) || !(delta < INFINITY)) {
    set_msg(msg, "delta must be positive and finite, got %g", (double)delta);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (buckets) *buckets = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = G->n;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  Temp<int32_t> qa(s), qb(s), el(s), qst(s), est(s);
  Temp<int64_t> cnt(s);
  LAGR_TRY(qa.alloc(n, msg, "frontier"));
  LAGR_TRY(qb.alloc(n, msg, "next frontier"));
  LAGR_TRY(el.alloc(n, msg, "settled list"));
  LAGR_TRY(qst.alloc(n, msg, "frontier stamps"));
  LAGR_TRY(est.alloc(n, msg, "settled stamps"));
  LAGR_TRY(cnt.alloc(SP_NSLOT, msg, "counters"));
  FxSpace fx;
  struct FxGuard {
    FxSpace *f;
    cudaStream_t s;
    ~FxGuard() { fx_free(f, s); }
  } fxg{&fx, s};
  LAGR_TRY(fx_alloc(&fx, n, s, msg));
  int32_t *tbits = reinterpret_cast<int32_t *>(dist);
  const double invd = 1.0 / (double)delta;
  const float inv_delta = invd < 3.0e38 ? (float)invd : 3.0e38f;  // finite for any positive delta
  const int relax_grid = resident_ctas((const void *)sp_relax<true>, SP_THREADS, 0);
  const int relax_grid_h = resident_ctas((const void *)sp_relax<false>, SP_THREADS, 0);
  sp_init<<<grid_for(n, SP_THREADS), SP_THREADS, 0, s>>>(n, src, tbits, qst.p, est.p, qa.p, cnt.p);
  LAGR_LAUNCH_CHECK();
  int32_t *q = qa.p, *qn = qb.p;
  int64_t nq = 1;
  long long cur = 0;
  int32_t step = 0, bseq = 0;
  const int64_t step_cap = 64 * (int64_t)n + 1024;
  int64_t h[SP_NSLOT];
  for (;;) {  // one bucket per pass
    bseq++;
    while (nq > 0) {  // light relaxations until the bucket's distances stop improving
      if (++step > step_cap) {
        set_msg(msg, "delta-stepping did not settle within %lld steps", (long long)step_cap);
        return LAGR_ERR_TIMEOUT;
      }
      sp_settle<<<grid_for(nq, SP_THREADS), SP_THREADS, 0, s>>>(q, (int32_t)nq, bseq, est.p, el.p, cnt.p);
      LAGR_TRY(fx_plan(&fx, q, (int32_t)nq, G->rowptr, s, msg));
      LAGR_CUDA_TRY(cudaMemsetAsync(cnt.p + SP_NQ, 0, sizeof(int64_t), s));
      sp_relax<true><<<relax_grid, SP_THREADS, 0, s>>>(G->rowptr, G->colidx, G->val, q, (int32_t)nq, fx.off, delta,
                                                      inv_delta, tbits, cur, step, qst.p, qn, cnt.p);
      LAGR_LAUNCH_CHECK();
      LAGR_TRY(fetch_to_host(h, cnt.p, sizeof(h), s, msg));
      nq = h[SP_NQ];
      int32_t *t = q;
      q = qn;
      qn = t;
    }
    // heavy relaxations from every vertex the bucket settled
    const int64_t ne = h[SP_NE];
    if (ne > 0) {
      LAGR_TRY(fx_plan(&fx, el.p, (int32_t)ne, G->rowptr, s, msg));
      sp_relax<false><<<relax_grid_h, SP_THREADS, 0, s>>>(G->rowptr, G->colidx, G->val, el.p, (int32_t)ne, fx.off,
                                                         delta, inv_delta, tbits, cur, step, qst.p, qn, cnt.p);
    }
    // the next non-empty bucket becomes the frontier
    step++;
    sp_reset<<<1, 1, 0, s>>>(cnt.p);
    sp_next_min<<<grid_for(n, SP_THREADS), SP_THREADS, 0, s>>>(n, tbits, cur, inv_delta, cnt.p);
    sp_build<<<grid_for(n, SP_THREADS), SP_THREADS, 0, s>>>(n, tbits, inv_delta, step, qst.p, q, cnt.p);
    LAGR_LAUNCH_CHECK();
    LAGR_TRY(fetch_to_host(h, cnt.p, sizeof(h), s, msg));
    nq = h[SP_NQ];
    if (nq == 0) break;
    cur = h[SP_CUR];
  }
  if (buckets) *buckets = bseq;
  G->last_iters = bseq;
  clear_msg(msg);
  return LAGR_OK;
}
