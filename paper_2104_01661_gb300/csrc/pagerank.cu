// PageRank (Alg. 3, Sec. IV-C) and its adjoint.
//
// One launch per iteration gathers a whole row of A' (a "pull" SpMV over the CSC) per group of
// G lanes and fuses every other step of Alg. 3 into it: the teleport assignment, the
// accumulation r += A' plus.second w, the next w = damping * r / d_out (eWiseMult), and the
// per-block partial sums of |t - r| (the apply(abs) + reduce of the stopping test) and of the
// dangling mass.  Rows longer than PR_HEAVY are gathered by one CTA each.  A one-block kernel
// folds the partials in a fixed order (so results do not depend on scheduling), decides
// convergence on the device and prepares the next iteration's scalar; later launches in the
// same batch see the flag and return at once.
//
// MODE 0: unweighted forward    r_i   = v_i c + sum_{j in A'(i,:)} w_j,  w_j = damping t_j / d_out(j)
// MODE 1: weighted forward      r_i   = v_i c + damping sum_j W(j,i) t_j
// MODE 2: adjoint (rows of W)   l'_i  = g_i + damping sum_j W(i,j) l_j [+ damping (v.l) if i dangling]
// where c = (1 - damping) [+ damping * (dangling mass of t) with LAGR_PR_DANGLING].
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace lagr {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_BLOCKS = 152 * 8;   // fixed grid: the partial-sum layout does not depend on n
constexpr int PR_HEAVY = 4096;       // rows longer than this are gathered by a CTA
constexpr int PR_HEAVY_BLOCKS = 152;
constexpr int PR_CHUNK = 8;          // iterations launched between host checks

struct PrState {
  double resid;   // last L1 change
  double aux;     // last auxiliary sum (dangling mass, or v . lambda)
  float coef;     // scalar for the next iteration (see the file comment)
  int done;       // set once the tolerance is met or itermax reached
  int iters;      // iterations done
  int pad;
};

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) return LAGR_FULL_MASK;
  else return ((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1));
}

// per-vertex damping / out-degree (0 for dangling rows) from the rows of A
__global__ void pr_scale(const int32_t *__restrict__ rowptr, int32_t n, float damping, float *__restrict__ sc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = rowptr[i + 1] - rowptr[i];
    sc[i] = d > 0 ? damping / (float)d : 0.0f;
  }
}

// r0 (uniform 1/n unless warm), w0 = r0 * sc, partial sums of the dangling mass of r0 (aux)
// MODE 2: l0 = g, aux = v . g
template <int MODE>
__global__ void pr_init(int32_t n, float *__restrict__ x, float *__restrict__ w, const float *__restrict__ sc,
                        const float *__restrict__ src, const float *__restrict__ vvec, float vuni,
                        double2 *__restrict__ partials) {
  __shared__ double red[32];
  double aux = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float xi = src ? src[i] : vuni;  // MODE 0/1: warm start or 1/n; MODE 2: g
    x[i] = xi;
    if (MODE == 0) w[i] = xi * sc[i];
    if (MODE == 2) aux += (double)(vvec ? vvec[i] : vuni) * (double)xi;
    else aux += (sc[i] == 0.0f) ? (double)xi : 0.0;
  }
  aux = block_sum(aux, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(0.0, aux);
}

template <int MODE>
__device__ __forceinline__ void pr_row_out(int64_t i, float acc, float damping, float coef, int dangling,
                                           const float *__restrict__ prev, float *__restrict__ out,
                                           float *__restrict__ wout, const float *__restrict__ sc,
                                           const float *__restrict__ vvec, float vuni, const float *__restrict__ gvec,
                                           double &resid, double &aux) {
  const float vi = vvec ? vvec[i] : vuni;
  const float s = sc[i];
  float r;
  if (MODE == 0) {
    r = vi * coef + acc;
    wout[i] = r * s;
  } else if (MODE == 1) {
    r = vi * coef + damping * acc;
  } else {
    r = gvec[i] + damping * acc;
    if (dangling && s == 0.0f) r += coef;
  }
  out[i] = r;
  resid += fabs((double)prev[i] - (double)r);
  if (MODE == 2) aux += (double)vi * (double)r;
  else if (s == 0.0f) aux += (double)r;
}

template <int G, int MODE>
__global__ void __launch_bounds__(PR_THREADS)
    pr_rows(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
            const float *__restrict__ val, const float *__restrict__ x, const float *__restrict__ prev,
            float *__restrict__ out, float *__restrict__ wout, const float *__restrict__ sc,
            const float *__restrict__ vvec, float vuni, const float *__restrict__ gvec, float damping, int dangling,
            const PrState *__restrict__ st, double2 *__restrict__ partials) {
  __shared__ double red[32];
  if (st->done) return;  // uniform over the grid
  const float coef = st->coef;
  const int lg = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  double resid = 0.0, aux = 0.0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < n; i += groups) {
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    if (e - b > PR_HEAVY) continue;
    float acc = 0.0f;
    for (int32_t k = b + lg; k < e; k += G) {
      const int32_t j = colidx[k];
      acc += (MODE == 0) ? __ldg(&x[j]) : __ldg(&val[k]) * __ldg(&x[j]);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gm, acc, o);
    if (lg == 0)
      pr_row_out<MODE>(i, acc, damping, coef, dangling, prev, out, wout, sc, vvec, vuni, gvec, resid, aux);
  }
  resid = block_sum(resid, red);
  aux = block_sum(aux, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(resid, aux);
}

template <int MODE>
__global__ void __launch_bounds__(512)
    pr_rows_heavy(const int32_t *__restrict__ heavy, int32_t nheavy, const int32_t *__restrict__ rowptr,
                  const int32_t *__restrict__ colidx, const float *__restrict__ val, const float *__restrict__ x,
                  const float *__restrict__ prev, float *__restrict__ out, float *__restrict__ wout,
                  const float *__restrict__ sc, const float *__restrict__ vvec, float vuni,
                  const float *__restrict__ gvec, float damping, int dangling, const PrState *__restrict__ st,
                  double2 *__restrict__ partials) {
  __shared__ float redf[32];
  if (st->done) return;
  const float coef = st->coef;
  double resid = 0.0, aux = 0.0;
  for (int32_t h = blockIdx.x; h < nheavy; h += gridDim.x) {
    const int32_t i = heavy[h];
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    float acc = 0.0f;
    for (int32_t k = b + threadIdx.x; k < e; k += blockDim.x) {
      const int32_t j = colidx[k];
      acc += (MODE == 0) ? __ldg(&x[j]) : __ldg(&val[k]) * __ldg(&x[j]);
    }
    acc = block_sum(acc, redf);
    if (threadIdx.x == 0)
      pr_row_out<MODE>(i, acc, damping, coef, dangling, prev, out, wout, sc, vvec, vuni, gvec, resid, aux);
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(resid, aux);
}

// fold the partials in a fixed order; init != 0 only prepares the first coefficient
__global__ void pr_finalize(const double2 *__restrict__ partials, int np, PrState *__restrict__ st, int mode,
                            float damping, int dangling, double tol, int itermax, int init) {
  __shared__ double red[32];
  if (!init && st->done) return;
  double r = 0.0, a = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    r += partials[i].x;
    a += partials[i].y;
  }
  r = block_sum(r, red);
  a = block_sum(a, red);
  if (threadIdx.x == 0) {
    float coef;
    if (mode == 2) coef = dangling ? (float)((double)damping * a) : 0.0f;
    else coef = (float)((1.0 - (double)damping) + (dangling ? (double)damping * a : 0.0));
    st->coef = coef;
    st->aux = a;
    if (!init) {
      st->iters += 1;
      st->resid = r;
      if (r < tol || st->iters >= itermax) st->done = 1;
    }
  }
}

// dL/dW(i,j) = damping r_i lambda_j over the rows of W (G lanes per row; heavy rows by a CTA)
template <int G>
__global__ void pr_edge_grad(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                             const float *__restrict__ r, const float *__restrict__ lam, float damping,
                             float *__restrict__ dw) {
  const int lg = threadIdx.x & (G - 1);
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < n; i += groups) {
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    if (e - b > PR_HEAVY) continue;
    const float ri = damping * r[i];
    for (int32_t k = b + lg; k < e; k += G) dw[k] = ri * __ldg(&lam[colidx[k]]);
  }
}

__global__ void pr_edge_grad_heavy(const int32_t *__restrict__ heavy, int32_t nheavy, const int32_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ colidx, const float *__restrict__ r,
                                   const float *__restrict__ lam, float damping, float *__restrict__ dw) {
  for (int32_t h = blockIdx.x; h < nheavy; h += gridDim.x) {
    const int32_t i = heavy[h];
    const float ri = damping * r[i];
    for (int32_t k = rowptr[i] + threadIdx.x; k < rowptr[i + 1]; k += blockDim.x) dw[k] = ri * __ldg(&lam[colidx[k]]);
  }
}

// dL/dv_j = ((1 - damping) + damping * delta) lambda_j, delta = st->aux (dangling mass of r)
__global__ void pr_teleport_grad(int32_t n, const float *__restrict__ lam, const PrState *__restrict__ st,
                                 float damping, int dangling, float *__restrict__ dv) {
  const double f = (1.0 - (double)damping) + (dangling ? (double)damping * st->aux : 0.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dv[i] = (float)(f * (double)lam[i]);
}

inline int grid_for(int64_t work, int threads, int cap = 152 * 16) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

inline int pick_group(int64_t nnz, int32_t n) {
  const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
  if (avg < 6) return 4;
  if (avg < 12) return 8;
  if (avg < 24) return 16;
  return 32;
}

template <int MODE>
void launch_rows(int G, int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *val, const float *x,
                 const float *prev, float *out, float *wout, const float *sc, const float *vvec, float vuni,
                 const float *gvec, float damping, int dangling, const PrState *st, double2 *partials,
                 cudaStream_t s) {
#define LAGR_PR_CASE(GG)                                                                                  \
  case GG:                                                                                                \
    pr_rows<GG, MODE><<<PR_BLOCKS, PR_THREADS, 0, s>>>(n, rowptr, colidx, val, x, prev, out, wout, sc, vvec, \
                                                       vuni, gvec, damping, dangling, st, partials);       \
    break;
  switch (G) {
    LAGR_PR_CASE(4)
    LAGR_PR_CASE(8)
    LAGR_PR_CASE(16)
    default: LAGR_PR_CASE(32)
  }
#undef LAGR_PR_CASE
}

}  // namespace

// Run the iteration of `mode` to convergence.  buf0 holds the start vector on entry (MODE 0/1,
// written here unless warm) and the result on exit.  Returns the iteration count in *iters.
static int pr_solve(int mode, lagr_graph G, Priv *P, const int32_t *rowptr, const int32_t *colidx, const float *val,
                    const int32_t *heavy, int32_t nheavy, float *buf0, const float *sc, const float *vvec,
                    const float *gvec, const float *warm, float damping, float tol, int32_t itermax, int dangling,
                    PrState *st, int32_t *iters, double *resid, cudaStream_t s, char *msg) {
  const int32_t n = G->n;
  const int64_t nnz = G->nnz;
  Temp<float> buf1(s), w0(s), w1(s);
  Temp<double2> partials(s);
  LAGR_TRY(buf1.alloc(n, msg, "PageRank work vector"));
  if (mode == 0) {
    LAGR_TRY(w0.alloc(n, msg, "PageRank w"));
    LAGR_TRY(w1.alloc(n, msg, "PageRank w"));
  }
  const int np = PR_BLOCKS + PR_HEAVY_BLOCKS;
  LAGR_TRY(partials.alloc(np, msg, "PageRank partial sums"));
  LAGR_CUDA_TRY(cudaMemsetAsync(partials.p, 0, np * sizeof(double2), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(PrState), s));
  const float vuni = 1.0f / (float)n;
  const int G_ = pick_group(nnz, n);
  float *x[2] = {buf0, buf1.p};
  float *w[2] = {w0.p, w1.p};
  // init: the start vector, w0 and the first coefficient
  const float *src = (mode == 2) ? gvec : warm;
  if (mode == 2) pr_init<2><<<PR_BLOCKS, PR_THREADS, 0, s>>>(n, buf0, nullptr, sc, src, vvec, vuni, partials.p);
  else if (mode == 1) pr_init<1><<<PR_BLOCKS, PR_THREADS, 0, s>>>(n, buf0, nullptr, sc, src, vvec, vuni, partials.p);
  else pr_init<0><<<PR_BLOCKS, PR_THREADS, 0, s>>>(n, buf0, w[0], sc, src, vvec, vuni, partials.p);
  pr_finalize<<<1, 1024, 0, s>>>(partials.p, np, st, mode, damping, dangling, (double)tol, itermax, 1);
  LAGR_LAUNCH_CHECK();
  PrState host{};
  int32_t launched = 0;
  while (launched < itermax) {
    const int32_t chunk = (itermax - launched < PR_CHUNK) ? (itermax - launched) : PR_CHUNK;
    for (int c = 0; c < chunk; c++) {
      const int k = launched + c + 1;  // iteration number
      const float *xin = x[(k - 1) & 1];
      float *xout = x[k & 1];
      const float *gx = (mode == 0) ? w[(k - 1) & 1] : xin;
      float *wo = (mode == 0) ? w[k & 1] : nullptr;
      if (mode == 0) {
        launch_rows<0>(G_, n, rowptr, colidx, val, gx, xin, xout, wo, sc, vvec, vuni, gvec, damping, dangling, st,
                       partials.p, s);
        if (nheavy > 0)
          pr_rows_heavy<0><<<PR_HEAVY_BLOCKS, 512, 0, s>>>(heavy, nheavy, rowptr, colidx, val, gx, xin, xout, wo, sc,
                                                          vvec, vuni, gvec, damping, dangling, st,
                                                          partials.p + PR_BLOCKS);
      } else if (mode == 1) {
        launch_rows<1>(G_, n, rowptr, colidx, val, gx, xin, xout, wo, sc, vvec, vuni, gvec, damping, dangling, st,
                       partials.p, s);
        if (nheavy > 0)
          pr_rows_heavy<1><<<PR_HEAVY_BLOCKS, 512, 0, s>>>(heavy, nheavy, rowptr, colidx, val, gx, xin, xout, wo, sc,
                                                          vvec, vuni, gvec, damping, dangling, st,
                                                          partials.p + PR_BLOCKS);
      } else {
        launch_rows<2>(G_, n, rowptr, colidx, val, gx, xin, xout, wo, sc, vvec, vuni, gvec, damping, dangling, st,
                       partials.p, s);
        if (nheavy > 0)
          pr_rows_heavy<2><<<PR_HEAVY_BLOCKS, 512, 0, s>>>(heavy, nheavy, rowptr, colidx, val, gx, xin, xout, wo, sc,
                                                          vvec, vuni, gvec, damping, dangling, st,
                                                          partials.p + PR_BLOCKS);
      }
      pr_finalize<<<1, 1024, 0, s>>>(partials.p, np, st, mode, damping, dangling, (double)tol, itermax, 0);
    }
    LAGR_LAUNCH_CHECK();
    launched += chunk;
    LAGR_CUDA_TRY(cudaMemcpyAsync(P->hscal, st, sizeof(PrState), cudaMemcpyDeviceToHost, s));
    LAGR_CUDA_TRY(cudaStreamSynchronize(s));
    memcpy(&host, P->hscal, sizeof(PrState));
    if (host.done) break;
  }
  if (host.iters & 1) LAGR_CUDA_TRY(cudaMemcpyAsync(buf0, x[1], (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  *iters = host.iters;
  *resid = host.resid;
  return LAGR_OK;
}

static int pr_common_checks(lagr_graph G, float damping, float tol, int32_t itermax, int32_t flags, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  if (!(damping > 0.0f && damping < 1.0f)) {
    set_msg(msg, "damping must be in (0,1), got %g", (double)damping);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (!(tol >= 0.0f) || itermax < 1) {
    set_msg(msg, "need tol >= 0 and itermax >= 1 (tol=%g itermax=%d)", (double)tol, itermax);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (flags & ~(LAGR_PR_DANGLING | LAGR_PR_WEIGHTED | LAGR_PR_WARM_START)) {
    set_msg(msg, "unknown PageRank flags 0x%x", flags);
    return LAGR_ERR_INVALID_VALUE;
  }
  if ((flags & LAGR_PR_WEIGHTED) && !G->val) {
    set_msg(msg, "LAGR_PR_WEIGHTED needs graph values");
    return LAGR_ERR_INVALID_VALUE;
  }
  return LAGR_OK;
}

// ---- plan for a fixed number of unweighted iterations (batched path) ----------------------------

struct PrPlan {
  int32_t n = 0;
  const int32_t *rowptr = nullptr, *colidx = nullptr;
  const int32_t *heavy = nullptr;
  int32_t nheavy = 0;
  const float *vvec = nullptr;
  float damping = 0.85f;
  int G = 32;
  float *sc = nullptr, *x1 = nullptr, *w0 = nullptr, *w1 = nullptr;
  double2 *partials = nullptr;
  PrState *st = nullptr;
};

int pr_plan_create(PrPlan **out, lagr_graph G, Priv *P, float damping, const float *vvec, cudaStream_t s,
                   char *msg) {
  *out = nullptr;
  LAGR_TRY(lagr_property_AT(G, s, msg));
  if (P->at_nheavy < 0) LAGR_TRY(heavy_rows(G->at_rowptr, G->n, PR_HEAVY, &P->at_heavy, &P->at_nheavy, s, msg));
  PrPlan *pl = new PrPlan();
  pl->n = G->n;
  pl->rowptr = G->at_rowptr;
  pl->colidx = G->at_colidx;
  pl->heavy = P->at_heavy;
  pl->nheavy = P->at_nheavy;
  pl->vvec = vvec;
  pl->damping = damping;
  pl->G = pick_group(G->nnz, G->n);
  int st = alloc_n(&pl->sc, (size_t)G->n, s, msg, "PageRank scale");
  if (st == LAGR_OK) st = alloc_n(&pl->x1, (size_t)G->n, s, msg, "PageRank work vector");
  if (st == LAGR_OK) st = alloc_n(&pl->w0, (size_t)G->n, s, msg, "PageRank w");
  if (st == LAGR_OK) st = alloc_n(&pl->w1, (size_t)G->n, s, msg, "PageRank w");
  if (st == LAGR_OK) st = alloc_n(&pl->partials, (size_t)(PR_BLOCKS + PR_HEAVY_BLOCKS), s, msg, "partials");
  if (st == LAGR_OK) st = alloc_n(&pl->st, 1, s, msg, "PageRank state");
  if (st < 0) {
    pr_plan_destroy(pl, s);
    return st;
  }
  pr_scale<<<grid_for(G->n, 256), 256, 0, s>>>(G->rowptr, G->n, damping, pl->sc);
  LAGR_LAUNCH_CHECK();
  *out = pl;
  return LAGR_OK;
}

int pr_plan_enqueue(PrPlan *pl, float *out, const float *warm, int32_t iters, cudaStream_t s, char *msg) {
  const int np = PR_BLOCKS + PR_HEAVY_BLOCKS;
  const float vuni = 1.0f / (float)pl->n;
  float *x[2] = {out, pl->x1};
  float *w[2] = {pl->w0, pl->w1};
  LAGR_CUDA_TRY(cudaMemsetAsync(pl->partials, 0, np * sizeof(double2), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(pl->st, 0, sizeof(PrState), s));
  pr_init<0><<<PR_BLOCKS, PR_THREADS, 0, s>>>(pl->n, out, w[0], pl->sc, warm, pl->vvec, vuni, pl->partials);
  pr_finalize<<<1, 1024, 0, s>>>(pl->partials, np, pl->st, 0, pl->damping, 0, 0.0, iters, 1);
  for (int k = 1; k <= iters; k++) {
    const float *xin = x[(k - 1) & 1];
    launch_rows<0>(pl->G, pl->n, pl->rowptr, pl->colidx, nullptr, w[(k - 1) & 1], xin, x[k & 1], w[k & 1], pl->sc,
                   pl->vvec, vuni, nullptr, pl->damping, 0, pl->st, pl->partials, s);
    if (pl->nheavy > 0)
      pr_rows_heavy<0><<<PR_HEAVY_BLOCKS, 512, 0, s>>>(pl->heavy, pl->nheavy, pl->rowptr, pl->colidx, nullptr,
                                                      w[(k - 1) & 1], xin, x[k & 1], w[k & 1], pl->sc, pl->vvec, vuni,
                                                      nullptr, pl->damping, 0, pl->st, pl->partials + PR_BLOCKS);
    pr_finalize<<<1, 1024, 0, s>>>(pl->partials, np, pl->st, 0, pl->damping, 0, 0.0, iters, 0);
  }
  LAGR_LAUNCH_CHECK();
  if (iters & 1)
    LAGR_CUDA_TRY(cudaMemcpyAsync(out, pl->x1, (size_t)pl->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return LAGR_OK;
}

void pr_plan_destroy(PrPlan *pl, cudaStream_t s) {
  if (!pl) return;
  dev_free(pl->sc, s);
  dev_free(pl->x1, s);
  dev_free(pl->w0, s);
  dev_free(pl->w1, s);
  dev_free(pl->partials, s);
  dev_free(pl->st, s);
  delete pl;
}

// forward solve into `rank` (device [n]); shared by lagr_pagerank and the recompute path of the
// backward
static int pr_forward(float *rank, int32_t *iters, double *resid, lagr_graph G, Priv *P, float damping, float tol,
                      int32_t itermax, const float *teleport, int32_t flags, const float *sc, PrState *st,
                      cudaStream_t s, char *msg) {
  LAGR_TRY(lagr_property_AT(G, s, msg));
  if (P->at_nheavy < 0) LAGR_TRY(heavy_rows(G->at_rowptr, G->n, PR_HEAVY, &P->at_heavy, &P->at_nheavy, s, msg));
  const int mode = (flags & LAGR_PR_WEIGHTED) ? 1 : 0;
  const float *warm = (flags & LAGR_PR_WARM_START) ? rank : nullptr;
  return pr_solve(mode, G, P, G->at_rowptr, G->at_colidx, G->at_val, P->at_heavy, P->at_nheavy, rank, sc, teleport,
                  nullptr, warm, damping, tol, itermax, (flags & LAGR_PR_DANGLING) ? 1 : 0, st, iters, resid, s, msg);
}

}  // namespace lagr

using namespace lagr;

extern "C" int lagr_pagerank(float *rank, int32_t *iters, lagr_graph G, float damping, float tol, int32_t itermax,
                             const float *teleport, int32_t flags, void *stream, char *msg) {
  if (!rank) {
    set_msg(msg, "rank is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(pr_common_checks(G, damping, tol, itermax, flags, msg));
  if (iters) *iters = 0;
  if (G->n == 0) {
    clear_msg(msg);
    return LAGR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  Temp<float> sc(s);
  Temp<PrState> st(s);
  LAGR_TRY(sc.alloc(G->n, msg, "PageRank scale"));
  LAGR_TRY(st.alloc(1, msg, "PageRank state"));
  pr_scale<<<grid_for(G->n, 256), 256, 0, s>>>(G->rowptr, G->n, damping, sc.p);
  LAGR_LAUNCH_CHECK();
  int32_t k = 0;
  double resid = 0.0;
  LAGR_TRY(pr_forward(rank, &k, &resid, G, P, damping, tol, itermax, teleport, flags, sc.p, st.p, s, msg));
  G->last_iters = k;
  G->last_resid = resid;
  if (iters) *iters = k;
  if (tol > 0.0f && !(resid < (double)tol)) {
    set_msg(msg, "PageRank stopped at itermax=%d with L1 change %g >= tol %g", itermax, resid, (double)tol);
    return LAGR_WARN_NOT_CONVERGED;
  }
  clear_msg(msg);
  return LAGR_OK;
}

extern "C" int lagr_pagerank_backward(float *dL_dw, float *dL_dteleport, int32_t *iters, const float *dL_drank,
                                      const float *rank, lagr_graph G, float damping, float tol, int32_t itermax,
                                      const float *teleport, int32_t flags, void *stream, char *msg) {
  if (!dL_drank) {
    set_msg(msg, "dL_drank is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(pr_common_checks(G, damping, tol, itermax, flags, msg));
  if (!(flags & LAGR_PR_WEIGHTED)) {
    set_msg(msg, "the adjoint is defined for the weighted form (LAGR_PR_WEIGHTED)");
    return LAGR_ERR_INVALID_VALUE;
  }
  if (iters) *iters = 0;
  if (G->n == 0) {
    clear_msg(msg);
    return LAGR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  const int dangling = (flags & LAGR_PR_DANGLING) ? 1 : 0;
  Temp<float> sc(s), rfwd(s), lam(s);
  Temp<PrState> st(s);
  LAGR_TRY(sc.alloc(G->n, msg, "PageRank scale"));
  LAGR_TRY(st.alloc(1, msg, "PageRank state"));
  LAGR_TRY(lam.alloc(G->n, msg, "adjoint vector"));
  pr_scale<<<grid_for(G->n, 256), 256, 0, s>>>(G->rowptr, G->n, damping, sc.p);
  LAGR_LAUNCH_CHECK();
  const float *r = rank;
  if (!r) {  // recompute the forward fixed point instead of keeping it
    LAGR_TRY(rfwd.alloc(G->n, msg, "recomputed rank"));
    int32_t k = 0;
    double res = 0.0;
    LAGR_TRY(pr_forward(rfwd.p, &k, &res, G, P, damping, tol, itermax, teleport, flags & ~LAGR_PR_WARM_START,
                        sc.p, st.p, s, msg));
    r = rfwd.p;
  }
  if (P->a_nheavy < 0) LAGR_TRY(heavy_rows(G->rowptr, G->n, PR_HEAVY, &P->a_heavy, &P->a_nheavy, s, msg));
  int32_t k = 0;
  double resid = 0.0;
  LAGR_TRY(pr_solve(2, G, P, G->rowptr, G->colidx, G->val, P->a_heavy, P->a_nheavy, lam.p, sc.p, teleport,
                    dL_drank, nullptr, damping, tol, itermax, dangling, st.p, &k, &resid, s, msg));
  if (dL_dw && G->nnz > 0) {
    const int G_ = pick_group(G->nnz, G->n);
    const int gb = grid_for((int64_t)G->n * G_, 256);
    switch (G_) {
      case 4: pr_edge_grad<4><<<gb, 256, 0, s>>>(G->n, G->rowptr, G->colidx, r, lam.p, damping, dL_dw); break;
      case 8: pr_edge_grad<8><<<gb, 256, 0, s>>>(G->n, G->rowptr, G->colidx, r, lam.p, damping, dL_dw); break;
      case 16: pr_edge_grad<16><<<gb, 256, 0, s>>>(G->n, G->rowptr, G->colidx, r, lam.p, damping, dL_dw); break;
      default: pr_edge_grad<32><<<gb, 256, 0, s>>>(G->n, G->rowptr, G->colidx, r, lam.p, damping, dL_dw); break;
    }
    if (P->a_nheavy > 0)
      pr_edge_grad_heavy<<<PR_HEAVY_BLOCKS, 512, 0, s>>>(P->a_heavy, P->a_nheavy, G->rowptr, G->colidx, r, lam.p,
                                                         damping, dL_dw);
    LAGR_LAUNCH_CHECK();
  }
  if (dL_dteleport) {
    // delta = dangling mass of r, through the init reduction of the forward (aux slot)
    Temp<double2> partials(s);
    Temp<float> scratch(s);
    LAGR_TRY(partials.alloc(PR_BLOCKS, msg, "partials"));
    LAGR_TRY(scratch.alloc(G->n, msg, "scratch"));
    pr_init<1><<<PR_BLOCKS, PR_THREADS, 0, s>>>(G->n, scratch.p, nullptr, sc.p, r, teleport, 1.0f / (float)G->n,
                                              partials.p);
    pr_finalize<<<1, 1024, 0, s>>>(partials.p, PR_BLOCKS, st.p, 1, damping, dangling, 0.0, 1, 1);
    pr_teleport_grad<<<grid_for(G->n, 256), 256, 0, s>>>(G->n, lam.p, st.p, damping, dangling, dL_dteleport);
    LAGR_LAUNCH_CHECK();
  }
  LAGR_CUDA_TRY(cudaStreamSynchronize(s));
  if (iters) *iters = k;
  G->last_iters = k;
  G->last_resid = resid;
  if (tol > 0.0f && !(resid < (double)tol)) {
    set_msg(msg, "adjoint stopped at itermax=%d with L1 change %g >= tol %g", itermax, resid, (double)tol);
    return LAGR_WARN_NOT_CONVERGED;
  }
  clear_msg(msg);
  return LAGR_OK;
}
