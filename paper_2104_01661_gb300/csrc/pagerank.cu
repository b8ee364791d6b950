// PageRank (Alg. 4, Sec. IV-C) and its adjoint.
//
// One iteration is one gather over the rows of A' (a "pull" SpMV over the CSC) that fuses every
// other step of Alg. 4: the teleport assignment, the accumulation r += A' plus.second w, the next
// w = damping * r / d_out (eWiseMult), and per-CTA partial sums of |t - r| (the apply(abs) +
// reduce of the stopping test) and of the dangling mass.
//
// Work partition (a RowPlan, built once per graph and cached): rows of at most ROW_HEAVY entries
// are grouped into blocks of at most PR_UNITS units, a unit being one entry or one row (so long
// runs of isolated vertices cannot pile up in one block).  One warp sums one block: its entries
// are contiguous in the CSR, so the warp reads colidx in coalesced steps and keeps a step's
// gathers x[colidx] in flight together; rows are joined across lanes by a segmented scan, in a
// fixed order (deterministic results).  Rows longer than ROW_HEAVY are cut into fixed chunks,
// summed by trailing CTAs of the same launch, and a small kernel adds each such row's chunk sums
// in chunk order.  A one-block kernel folds the per-block partials in a fixed order, decides
// convergence on the device and prepares the next iteration's scalar; later launches of the same
// batch see the flag and return at once.
//
// MODE 0: unweighted forward    r_i  = v_i c + sum_{j in A'(i,:)} w_j,   w_j = damping t_j / d_out(j)
// MODE 1: weighted forward      r_i  = v_i c + damping sum_j W(j,i) t_j
// MODE 2: adjoint (rows of W)   l'_i = g_i + damping sum_j W(i,j) l_j [+ damping (v.l) if i dangling]
// where c = (1 - damping) [+ damping * (dangling mass of t) with LAGR_PR_DANGLING].
#include <cmath>
#include <cstddef>
#include <cstring>

#include "internal.cuh"

namespace lagr {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_UNITS = ROW_UNITS;                 // units (entries + rows) per edge-gradient block
constexpr int PR_WUNITS = FINE_UNITS;   // units per block of the gathers' row plans (one warp's work item)
constexpr int PR_WHEAVY = FINE_HEAVY;   // longer rows are cut into chunks of PR_WHCHUNK entries
constexpr int PR_WHCHUNK = FINE_HCHUNK;
constexpr int PR_CHUNK = 8;                         // iterations launched between host checks

constexpr int PR_FIN_BLOCKS = 32;  // CTAs of the partial-sum fold

// the per-CTA partial sums of an iteration: residual, auxiliary sum (dangling mass or v . lambda),
// L1 norm of the new iterate (adjoint only)
struct __align__(16) PrSums {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ PrSums pr_sums(double x, double y, double z, double w) { return PrSums{x, y, z, w}; }

struct PrState {
  // read by the host (the first PR_STATE_HOST bytes)
  double resid;   // last L1 change
  double aux;     // last auxiliary sum (dangling mass, or v . lambda)
  float coef;     // scalar for the next iteration (see the file comment)
  int done;       // set once the tolerance is met or itermax reached
  int iters;      // iterations done
  int queue;      // next row block of the running gather (reset by pr_finalize)
  // device only: the fold's per-CTA sums (residual, auxiliary sum, L1 norm of the iterate) and its
  // arrival counter
  PrSums fold[PR_FIN_BLOCKS];
  unsigned int arrive;
};
constexpr size_t PR_STATE_HOST = 32;  // resid, aux, coef, done, iters, queue

// per-vertex damping / out-degree (0 for dangling rows) from the rows of A
__global__ void pr_scale(const int32_t *__restrict__ rowptr, int32_t n, float damping, float *__restrict__ sc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = rowptr[i + 1] - rowptr[i];
    sc[i] = d > 0 ? damping / (float)d : 0.0f;
  }
}

// ---- the iteration --------------------------------------------------------------------------------

// r0 (uniform 1/n unless warm), w0 = r0 * sc, partial sums of the dangling mass of r0 (aux)
// MODE 2: l0 = g, aux = v . g
template <int MODE>
__global__ void pr_init(int32_t n, float *__restrict__ x, float *__restrict__ w, const float *__restrict__ sc,
                        const float *__restrict__ src, const float *__restrict__ vvec, float vuni,
                        PrSums *__restrict__ partials) {
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
  if (threadIdx.x == 0) partials[blockIdx.x] = pr_sums(0.0, aux, 0.0, 0.0);
}

struct IterArgs {
  const int32_t *rowptr, *colidx;
  const float *val;   // MODE 1/2
  const float *x;     // gathered vector (w for MODE 0, t for MODE 1, lambda for MODE 2)
  const float *prev;  // previous iterate (residual)
  float *out;         // new iterate
  float *wout;        // MODE 0: new w
  const float *sc;    // damping / d_out, 0 on dangling rows
  const float *vvec;  // teleport vector or NULL (uniform vuni)
  float vuni;
  const float *gvec;  // MODE 2: dL/dr
  float damping;
  int dangling;
  float *hpart;       // partial sums of the heavy-row chunks
  int vec;            // colidx (and val) are 16-byte aligned: steps load them as vectors
  float *acc;         // the row sums of the gather, turned into the outputs by pr_epilogue
};

template <int MODE>
__device__ __forceinline__ float gather_one(const IterArgs &a, int32_t k) {
  const int32_t j = __ldg(a.colidx + k);
  if (MODE == 0) return __ldg(&a.x[j]);
  return __ldg(&a.val[k]) * __ldg(&a.x[j]);
}

// a row's output from its sum; resid / aux collect this thread's share in float (a thread's
// few rows), the block reduction continues in double (GB300's float64 rate is a small fraction
// of its float32 rate)
template <int MODE>
__device__ __forceinline__ void row_out(const IterArgs &a, int32_t i, float acc, float coef, float &resid,
                                        float &aux, float &nrm) {
  const float vi = a.vvec ? a.vvec[i] : a.vuni;
  const float s = a.sc[i];
  float r;
  if (MODE == 0) {
    r = vi * coef + acc;
    a.wout[i] = r * s;
  } else if (MODE == 1) {
    r = vi * coef + a.damping * acc;
  } else {
    r = a.gvec[i] + a.damping * acc;
    if (a.dangling && s == 0.0f) r += coef;
  }
  a.out[i] = r;
  resid += fabsf(a.prev[i] - r);
  if (MODE == 2) nrm += fabsf(r);
  if (MODE == 2) aux += vi * r;
  else if (s == 0.0f) aux += r;
}

// ---- one warp per row block ----------------------------------------------------------------------
//
// A warp walks its block's entries in steps of 32 x PR_EPL: lane l takes the PR_EPL consecutive
// entries at step_start + PR_EPL * l (colidx read as 16-byte vectors where aligned, so a step is one
// contiguous, coalesced read), issues all their gathers, then adds them up in entry order, closing
// a row whenever its end passes.  A row that runs over lane (or step) boundaries is joined by one
// segmented scan over the lanes per step: lane l contributes the open part of its last row, and the
// lane where the row ends adds the joined prefix to its own part.  The next step's column indices
// are loaded while the current step is summed.  Sums are in a fixed order (deterministic).
// Empty rows are written by a separate pass over the block's rows.  A row longer than ROW_HEAVY is
// a block of its own, skipped here (its chunks are summed by the trailing CTAs).

constexpr int PR_EPL = 8;                  // entries per lane per step
constexpr int PR_STEP = 32 * PR_EPL;       // entries per warp step

// the column indices (and values) of entries k .. k + PR_EPL - 1; those outside [lo, hi) read as -1
template <int MODE>
__device__ __forceinline__ void load_step(const IterArgs &a, int32_t k, int32_t lo, int32_t hi, int32_t (&c)[PR_EPL],
                                          float (&v)[PR_EPL]) {
  const int32_t *__restrict__ cols = a.colidx;
  if (a.vec && k >= 0 && k + PR_EPL <= hi) {
    const int4 c0 = __ldg(reinterpret_cast<const int4 *>(cols + k));
    const int4 c1 = __ldg(reinterpret_cast<const int4 *>(cols + k + 4));
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    if (MODE != 0) {
      const float4 v0 = __ldg(reinterpret_cast<const float4 *>(a.val + k));
      const float4 v1 = __ldg(reinterpret_cast<const float4 *>(a.val + k + 4));
      v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w;
      v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
    }
#pragma unroll
    for (int j = 0; j < PR_EPL; j++)
      if (k + j < lo) c[j] = -1;
  } else {
#pragma unroll
    for (int j = 0; j < PR_EPL; j++) {
      const bool ok = k + j >= lo && k + j < hi;
      c[j] = ok ? __ldg(cols + k + j) : -1;
      if (MODE != 0) v[j] = ok ? __ldg(a.val + k + j) : 0.0f;
    }
  }
}

__device__ __forceinline__ float gather_x(const IterArgs &a, int32_t c) {
  return c < 0 ? 0.0f : __ldg(a.x + c);
}

// last row index q in [lo, hi] with rp[q] <= k (rp[lo] <= k holds); rp in shared memory
__device__ __forceinline__ int32_t srow_of(const int32_t *rp, int32_t lo, int32_t hi, int32_t k) {
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// one row block (at most PR_WUNITS units), one warp: writes the block's row sums to a.acc.  srp:
// this warp's shared-memory copy of the block's row pointers.
template <int MODE>
__device__ __forceinline__ void warp_block(const IterArgs &a, const int32_t *__restrict__ blk,
                                           const uint8_t *__restrict__ hblk, int32_t wb, int32_t *srp) {
  const int lane = threadIdx.x & 31;
  const int32_t r0 = blk[wb], r1 = blk[wb + 1];
  const int32_t nr = r1 - r0;
  if (!hblk[wb]) {  // (a block that is one heavy row is summed by the chunk items)
    for (int32_t q = lane; q <= nr; q += 32) srp[q] = __ldg(a.rowptr + r0 + q);
    __syncwarp();
    for (int32_t q = lane; q < nr; q += 32)  // empty rows
      if (srp[q] == srp[q + 1]) a.acc[r0 + q] = 0.0f;
    const int32_t e0 = srp[0], e1 = srp[nr];
    const int32_t kb = e0 & ~3;  // steps start 16-byte aligned
    int32_t rc = 0;              // the block row holding the first entry of the current step
    float carry = 0.0f;          // the open part of the row running into the current step
    int32_t cn[PR_EPL];
    float vn[PR_EPL];
    load_step<MODE>(a, kb + PR_EPL * lane, e0, e1, cn, vn);
    for (int32_t gs = kb; gs < e1; gs += PR_STEP) {
      const int32_t k0 = gs + PR_EPL * lane;
      float g[PR_EPL];
#pragma unroll
      for (int j = 0; j < PR_EPL; j++) {
        const float xv = gather_x(a, cn[j]);
        g[j] = MODE == 0 ? xv : vn[j] * xv;
      }
      if (gs + PR_STEP < e1) load_step<MODE>(a, k0 + PR_STEP, e0, e1, cn, vn);
      // this lane's entries [ks, ke)
      const int32_t ks = max(k0, e0), ke = min(k0 + PR_EPL, e1);
      float v = 0.0f;       // open part of the lane's last row (passed on by the scan)
      bool fresh = false;   // the scan restarts at this lane (nothing open flows through it)
      bool hclose = false;  // the lane closes a row that began before it (needs the joined prefix)
      float hsum = 0.0f;
      int32_t hrow = 0;
      int32_t qend = rc;  // the row holding this lane's last entry
      if (ks < ke) {
        int32_t q = srow_of(srp, rc, nr - 1, ks);
        int32_t rs = srp[q], re = srp[q + 1];
        const bool open_head = rs < ks;
        bool first = true;
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < PR_EPL; j++) {
          const int32_t k = k0 + j;
          if (k < ks || k >= ke) continue;
          while (k >= re) {  // the row ended before k: close it, step over empty rows
            if (re > rs) {
              if (first && open_head) {
                hclose = true;
                hsum = acc;
                hrow = q;
              } else {
                a.acc[r0 + q] = acc;
              }
            }
            first = false;
            acc = 0.0f;
            q++;
            rs = re;
            re = srp[q + 1];
          }
          acc += g[j];
        }
        qend = q;
        if (re == ke) {  // the last row ends with this lane's entries
          if (first && open_head) {
            hclose = true;
            hsum = acc;
            hrow = q;
          } else {
            a.acc[r0 + q] = acc;
          }
          fresh = true;
        } else {
          v = acc;
          fresh = !(first && open_head);
        }
      }
      // segmented inclusive scan of (v, fresh) over the lanes; the step's carry enters at lane 0
      float sv = v;
      bool sf = fresh;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float tv = __shfl_up_sync(LAGR_FULL_MASK, sv, o);
        const bool tf = __shfl_up_sync(LAGR_FULL_MASK, (int)sf, o) != 0;
        if (lane >= o) {
          if (!sf) sv += tv;
          sf = sf || tf;
        }
      }
      if (!sf) sv += carry;
      float before = __shfl_up_sync(LAGR_FULL_MASK, sv, 1);
      if (lane == 0) before = carry;
      if (hclose) a.acc[r0 + hrow] = before + hsum;
      carry = __shfl_sync(LAGR_FULL_MASK, sv, 31);
      // the next step starts inside the row that holds this step's last entry (found by the lane
      // that holds that entry)
      rc = __shfl_sync(LAGR_FULL_MASK, qend, (min(gs + PR_STEP, e1) - 1 - gs) / PR_EPL);
    }
    __syncwarp();  // srp is rewritten by the warp's next block
  }
}

// one chunk of hchunk entries of a heavy row, one warp: its sum in hpart[cidx] (pr_heavy_finish
// adds a row's chunks up in chunk order)
template <int MODE>
__device__ __forceinline__ void warp_chunk(const IterArgs &a, const int32_t *__restrict__ heavy,
                                           const int32_t *__restrict__ hc_off, const int32_t *__restrict__ hc_row,
                                           int32_t hchunk, int32_t cidx) {
  const int lane = threadIdx.x & 31;
  const int32_t h = hc_row[cidx];
  const int32_t i = heavy[h];
  const int32_t b = __ldg(a.rowptr + i) + (cidx - hc_off[h]) * hchunk;
  const int32_t e = min(__ldg(a.rowptr + i + 1), b + hchunk);
  float acc = 0.0f;
  for (int32_t gs = b & ~3; gs < e; gs += PR_STEP) {
    int32_t c[PR_EPL];
    float v[PR_EPL];
    load_step<MODE>(a, gs + PR_EPL * lane, b, e, c, v);
#pragma unroll
    for (int j = 0; j < PR_EPL; j++) {
      const float xv = gather_x(a, c[j]);
      acc += MODE == 0 ? xv : v[j] * xv;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) a.hpart[cidx] = acc;
}

// Persistent CTAs: their warps take work items from one queue until none is left: first the
// chunks of the heavy rows, then the row blocks.
template <int MODE>
__global__ void __launch_bounds__(PR_THREADS, MODE == 0 ? 5 : 4)
    pr_warp(IterArgs a, const int32_t *__restrict__ blk, int32_t nblk, const uint8_t *__restrict__ hblk,
            const int32_t *__restrict__ heavy, const int32_t *__restrict__ hc_off, const int32_t *__restrict__ hc_row,
            int32_t nhc, int32_t hchunk, PrState *__restrict__ st) {
  __shared__ int32_t s_rp[PR_THREADS / 32][PR_WUNITS + 2];  // each warp's row pointers
  if (st->done) return;  // uniform over the grid
  const int lane = threadIdx.x & 31;
  int32_t *srp = s_rp[threadIdx.x >> 5];
  const int32_t nitems = nhc + nblk;
  for (;;) {
    int32_t q = 0;
    if (lane == 0) q = atomicAdd(&st->queue, 1);
    q = __shfl_sync(LAGR_FULL_MASK, q, 0);
    if (q >= nitems) break;
    if (q < nhc) warp_chunk<MODE>(a, heavy, hc_off, hc_row, hchunk, q);
    else warp_block<MODE>(a, blk, hblk, q - nhc, srp);
  }
}

// the heavy rows: add each row's chunk sums in chunk order
constexpr int PR_HF_THREADS = 256;
__global__ void __launch_bounds__(PR_HF_THREADS)
    pr_heavy_finish(IterArgs a, const int32_t *__restrict__ heavy, int32_t nheavy, const int32_t *__restrict__ hc_off,
                    const PrState *__restrict__ st) {
  if (st->done) return;
  const int32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nheavy) {
    float acc = 0.0f;
    for (int32_t c = hc_off[h]; c < hc_off[h + 1]; c++) acc += a.hpart[c];
    a.acc[heavy[h]] = acc;
  }
}

// The element-wise rest of the iteration over the row sums: each row's output (the teleport or
// adjoint term, the next gathered value, the residual and the dangling / v.lambda sum).  A fixed
// grid of epi_blocks() CTAs, each with a fixed share of the rows, writes one partial pair per CTA
// (deterministic).
template <int MODE>
__global__ void __launch_bounds__(PR_THREADS)
    pr_epilogue(IterArgs a, int32_t n, const PrState *__restrict__ st, PrSums *__restrict__ partials) {
  __shared__ double red[32];
  if (st->done) return;
  const float coef = st->coef;
  float fr = 0.0f, fa = 0.0f, fn = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    row_out<MODE>(a, (int32_t)i, a.acc[i], coef, fr, fa, fn);
  const double resid = block_sum((double)fr, red);
  const double aux = block_sum((double)fa, red);
  const double nrm = MODE == 2 ? block_sum((double)fn, red) : 0.0;
  if (threadIdx.x == 0) partials[blockIdx.x] = pr_sums(resid, aux, nrm, 0.0);
}

// Fold the partials in a fixed order: CTA b sums the b-th contiguous share (a fixed tree), and the
// CTA that arrives last adds the PR_FIN_BLOCKS sums in order and updates the state (the result does
// not depend on which CTA is last).  init != 0 only prepares the first coefficient.  The forward
// stops when the L1 change is below tol (Alg. 4); the adjoint (mode 2) when it is below tol times
// the L1 norm of the new iterate (its scale is that of dL/dr, so an absolute bound would be below
// float32 resolution on large graphs).
constexpr int PR_FIN_THREADS = 512;
__global__ void __launch_bounds__(PR_FIN_THREADS)
    pr_finalize(const PrSums *__restrict__ partials, int np, PrState *__restrict__ st, int mode, float damping,
                int dangling, double tol, int itermax, int init) {
  __shared__ double red[32];
  __shared__ bool last;
  if (!init && st->done) return;  // uniform: done changes only at the end of a fold
  const int per = (np + PR_FIN_BLOCKS - 1) / PR_FIN_BLOCKS;
  const int lo = blockIdx.x * per, hi = min(np, lo + per);
  double r = 0.0, a = 0.0, nr = 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    r += partials[i].x;
    a += partials[i].y;
    nr += partials[i].z;
  }
  r = block_sum(r, red);
  a = block_sum(a, red);
  nr = block_sum(nr, red);
  if (threadIdx.x == 0) {
    st->fold[blockIdx.x] = pr_sums(r, a, nr, 0.0);
    __threadfence();
    last = atomicAdd(&st->arrive, 1u) == PR_FIN_BLOCKS - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  r = 0.0;
  a = 0.0;
  nr = 0.0;
  for (int b = 0; b < PR_FIN_BLOCKS; b++) {
    const volatile double *f = reinterpret_cast<volatile double *>(&st->fold[b]);
    r += f[0];
    a += f[1];
    nr += f[2];
  }
  if (mode == 2) r = nr > 0.0 ? r / nr : r;  // the adjoint's change relative to its L1 norm
  float coef;
  if (mode == 2) coef = dangling ? (float)((double)damping * a) : 0.0f;
  else coef = (float)((1.0 - (double)damping) + (dangling ? (double)damping * a : 0.0));
  st->coef = coef;
  st->aux = a;
  st->queue = 0;  // the next gather starts its row-block queue afresh
  st->arrive = 0;
  if (!init) {
    st->iters += 1;
    st->resid = r;
    if (r < tol || st->iters >= itermax) st->done = 1;
  }
}

// dL/dW(i,j) = damping r_i lambda_j over the rows of W: each row block's CTA walks its contiguous
// entries (coalesced colidx and dW) and finds each entry's row in its staged row pointers
__global__ void __launch_bounds__(PR_THREADS)
    pr_edge_grad(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                 const int32_t *__restrict__ blk, const float *__restrict__ r, const float *__restrict__ lam,
                 float damping, float *__restrict__ dw) {
  __shared__ int32_t rp[PR_UNITS + 1];
  const int32_t r0 = blk[blockIdx.x], r1 = blk[blockIdx.x + 1];
  const int32_t nr = r1 - r0;
  if (nr == 0) return;
  for (int32_t q = threadIdx.x; q <= nr; q += PR_THREADS) rp[q] = rowptr[r0 + q];
  __syncthreads();
  const int32_t e0 = rp[0], e1 = rp[nr];
  for (int32_t k = e0 + threadIdx.x; k < e1; k += PR_THREADS) {
    int32_t lo = 0, hi = nr - 1;  // last q with rp[q] <= k
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= k) lo = mid; else hi = mid - 1;
    }
    dw[k] = damping * r[r0 + lo] * __ldg(&lam[colidx[k]]);
  }
}

// dL/dv_j = ((1 - damping) + damping * delta) lambda_j, delta = st->aux (dangling mass of r)
__global__ void pr_teleport_grad(int32_t n, const float *__restrict__ lam, const PrState *__restrict__ st,
                                 float damping, int dangling, float *__restrict__ dv) {
  const double f = (1.0 - (double)damping) + (dangling ? (double)damping * st->aux : 0.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dv[i] = (float)(f * (double)lam[i]);
}

}  // namespace

static inline int heavy_finish_blocks(const RowPlan &pl) {
  return (pl.nheavy + PR_HF_THREADS - 1) / PR_HF_THREADS;
}

// fixed grids of the element-wise kernels (the fold's order depends only on the grid): four and
// eight CTAs per multiprocessor
static inline int epi_blocks() { return 4 * sm_count(); }
static inline int init_blocks() { return 8 * sm_count(); }
static inline int n_partials() { return epi_blocks() > init_blocks() ? epi_blocks() : init_blocks(); }

static inline int aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// one iteration: the row-sum gather, the heavy rows' chunk sums, the element-wise epilogue and the
// fold of its partials
template <int MODE>
static void launch_iter(const RowPlan &pl, const IterArgs &a, int32_t n, PrState *st, PrSums *partials,
                        int32_t itermax, double tol, cudaStream_t s) {
  // as many persistent CTAs as can be resident at once (no more than there are warp items)
  const int resident = resident_ctas((const void *)pr_warp<MODE>, PR_THREADS, 0);
  const int64_t items = (int64_t)pl.nhc + pl.nblk;
  const int64_t need = (items * 32 + PR_THREADS - 1) / PR_THREADS;
  const int grid = (int)(need < resident ? (need > 0 ? need : 1) : resident);
  {
    KTimer kt(TK_PR_GATHER, s);
    pr_warp<MODE><<<grid, PR_THREADS, 0, s>>>(a, pl.blk, pl.nblk, pl.hblk, pl.heavy, pl.hc_off, pl.hc_row, pl.nhc,
                                              pl.hchunk, st);
  }
  const int hfb = heavy_finish_blocks(pl);
  if (hfb > 0) pr_heavy_finish<<<hfb, PR_HF_THREADS, 0, s>>>(a, pl.heavy, pl.nheavy, pl.hc_off, st);
  const int eb = epi_blocks();
  pr_epilogue<MODE><<<eb, PR_THREADS, 0, s>>>(a, n, st, partials);
  pr_finalize<<<PR_FIN_BLOCKS, PR_FIN_THREADS, 0, s>>>(partials, eb, st, MODE, a.damping, a.dangling, tol,
                                                       itermax, 0);
}

// start vector, w0 and the first coefficient (the init partials use the first init_blocks() slots)
static void launch_init(int mode, int32_t n, float *x, float *w, const float *sc, const float *src, const float *vvec,
                        float vuni, PrState *st, PrSums *partials, float damping, int dangling, int32_t itermax,
                        double tol, cudaStream_t s) {
  const int ib = init_blocks();
  if (mode == 2)
    pr_init<2><<<ib, PR_THREADS, 0, s>>>(n, x, nullptr, sc, src, vvec, vuni, partials);
  else if (mode == 1)
    pr_init<1><<<ib, PR_THREADS, 0, s>>>(n, x, nullptr, sc, src, vvec, vuni, partials);
  else
    pr_init<0><<<ib, PR_THREADS, 0, s>>>(n, x, w, sc, src, vvec, vuni, partials);
  pr_finalize<<<PR_FIN_BLOCKS, PR_FIN_THREADS, 0, s>>>(partials, ib, st, mode, damping, dangling, tol,
                                                       itermax, 1);
}

// Run the iteration of `mode` to convergence.  buf0 holds the start vector on entry (MODE 0/1,
// written here unless warm) and the result on exit.  Returns the iteration count in *iters.
static int pr_solve(int mode, lagr_graph G, Priv *P, const RowPlan &pl, const int32_t *rowptr, const int32_t *colidx,
                    const float *val, float *buf0, const float *sc,
                    const float *vvec, const float *gvec, const float *warm, float damping, float tol,
                    int32_t itermax, int dangling, PrState *st, int32_t *iters, double *resid, cudaStream_t s,
                    char *msg) {
  const int32_t n = G->n;
  const int vec = aligned16(colidx) && (val == nullptr || aligned16(val));
  Temp<float> buf1(s), w0(s), w1(s), hpart(s), rsum(s);
  Temp<PrSums> partials(s);
  LAGR_TRY(buf1.alloc(n, msg, "PageRank work vector"));
  LAGR_TRY(rsum.alloc(n, msg, "PageRank row sums"));
  LAGR_TRY(hpart.alloc((size_t)pl.nhc + 1, msg, "heavy chunk sums"));
  if (mode == 0) {
    LAGR_TRY(w0.alloc(n, msg, "PageRank w"));
    LAGR_TRY(w1.alloc(n, msg, "PageRank w"));
  }
  const int np = n_partials();
  LAGR_TRY(partials.alloc(np, msg, "PageRank partial sums"));
  LAGR_CUDA_TRY(cudaMemsetAsync(partials.p, 0, np * sizeof(PrSums), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(PrState), s));
  const float vuni = 1.0f / (float)n;
  float *x[2] = {buf0, buf1.p};
  float *w[2] = {w0.p, w1.p};
  launch_init(mode, n, buf0, w[0], sc, (mode == 2) ? gvec : warm, vvec, vuni, st, partials.p, damping, dangling,
              itermax, (double)tol, s);
  LAGR_LAUNCH_CHECK();
  PrState host{};
  int32_t launched = 0;
  while (launched < itermax) {
    const int32_t chunk = (itermax - launched < PR_CHUNK) ? (itermax - launched) : PR_CHUNK;
    for (int c = 0; c < chunk; c++) {
      const int k = launched + c + 1;  // iteration number
      IterArgs a{rowptr, colidx, val, nullptr, x[(k - 1) & 1], x[k & 1], nullptr, sc, vvec, vuni, gvec, damping,
                 dangling, hpart.p, vec, rsum.p};
      if (mode == 0) {
        a.x = w[(k - 1) & 1];
        a.wout = w[k & 1];
        launch_iter<0>(pl, a, n, st, partials.p, itermax, (double)tol, s);
      } else if (mode == 1) {
        a.x = x[(k - 1) & 1];
        launch_iter<1>(pl, a, n, st, partials.p, itermax, (double)tol, s);
      } else {
        a.x = x[(k - 1) & 1];
        launch_iter<2>(pl, a, n, st, partials.p, itermax, (double)tol, s);
      }
    }
    LAGR_LAUNCH_CHECK();
    launched += chunk;
    static_assert(PR_STATE_HOST == offsetof(PrState, fold) && PR_STATE_HOST <= LAGR_NHOST * sizeof(int64_t),
                  "host part of the state");
    LAGR_TRY(fetch_to_host(&host, st, PR_STATE_HOST, s, msg));
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
  RowPlan rows;  // borrowed from the graph's private state
  const float *vvec = nullptr;
  float damping = 0.85f;
  float *sc = nullptr, *x1 = nullptr, *w0 = nullptr, *w1 = nullptr, *hpart = nullptr, *rsum = nullptr;
  PrSums *partials = nullptr;
  int np = 0;
  PrState *st = nullptr;
};

int pr_plan_create(PrPlan **out, lagr_graph G, Priv *P, float damping, const float *vvec, cudaStream_t s,
                   char *msg) {
  *out = nullptr;
  LAGR_TRY(lagr_property_AT(G, s, msg));
  LAGR_TRY(row_plan(&P->pr_fwd, G->at_rowptr, G->n, s, msg, PR_WUNITS, PR_WHEAVY, PR_WHCHUNK));
  PrPlan *pl = new PrPlan();
  pl->n = G->n;
  pl->rowptr = G->at_rowptr;
  pl->colidx = G->at_colidx;
  pl->rows = P->pr_fwd;
  pl->vvec = vvec;
  pl->damping = damping;
  pl->np = n_partials();
  int st = alloc_n(&pl->sc, (size_t)G->n, s, msg, "PageRank scale");
  if (st == LAGR_OK) st = alloc_n(&pl->x1, (size_t)G->n, s, msg, "PageRank work vector");
  if (st == LAGR_OK) st = alloc_n(&pl->w0, (size_t)G->n, s, msg, "PageRank w");
  if (st == LAGR_OK) st = alloc_n(&pl->w1, (size_t)G->n, s, msg, "PageRank w");
  if (st == LAGR_OK) st = alloc_n(&pl->partials, (size_t)pl->np, s, msg, "partials");
  if (st == LAGR_OK) st = alloc_n(&pl->hpart, (size_t)P->pr_fwd.nhc + 1, s, msg, "heavy chunk sums");
  if (st == LAGR_OK) st = alloc_n(&pl->rsum, (size_t)G->n, s, msg, "PageRank row sums");
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
  const float vuni = 1.0f / (float)pl->n;
  float *x[2] = {out, pl->x1};
  float *w[2] = {pl->w0, pl->w1};
  LAGR_CUDA_TRY(cudaMemsetAsync(pl->partials, 0, pl->np * sizeof(PrSums), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(pl->st, 0, sizeof(PrState), s));
  launch_init(0, pl->n, out, w[0], pl->sc, warm, pl->vvec, vuni, pl->st, pl->partials, pl->damping, 0, iters, 0.0, s);
  for (int k = 1; k <= iters; k++) {
    IterArgs a{pl->rowptr, pl->colidx, nullptr, w[(k - 1) & 1], x[(k - 1) & 1], x[k & 1], w[k & 1], pl->sc,
               pl->vvec, vuni, nullptr, pl->damping, 0, pl->hpart, aligned16(pl->colidx), pl->rsum};
    launch_iter<0>(pl->rows, a, pl->n, pl->st, pl->partials, iters, 0.0, s);
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
  dev_free(pl->hpart, s);
  dev_free(pl->rsum, s);
  dev_free(pl->st, s);
  delete pl;
}

// forward solve into `rank` (device [n]); shared by lagr_pagerank and the recompute path of the
// backward
static int pr_forward(float *rank, int32_t *iters, double *resid, lagr_graph G, Priv *P, float damping, float tol,
                      int32_t itermax, const float *teleport, int32_t flags, const float *sc, PrState *st,
                      cudaStream_t s, char *msg) {
  LAGR_TRY(lagr_property_AT(G, s, msg));
  LAGR_TRY(row_plan(&P->pr_fwd, G->at_rowptr, G->n, s, msg, PR_WUNITS, PR_WHEAVY, PR_WHCHUNK));
  const int mode = (flags & LAGR_PR_WEIGHTED) ? 1 : 0;
  const float *warm = (flags & LAGR_PR_WARM_START) ? rank : nullptr;
  return pr_solve(mode, G, P, P->pr_fwd, G->at_rowptr, G->at_colidx, G->at_val, rank, sc, teleport, nullptr, warm,
                  damping, tol, itermax, (flags & LAGR_PR_DANGLING) ? 1 : 0, st, iters, resid, s, msg);
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
  LAGR_TRY(row_plan(&P->pr_a, G->rowptr, G->n, s, msg));
  LAGR_TRY(row_plan(&P->pr_adj, G->rowptr, G->n, s, msg, PR_WUNITS, PR_WHEAVY, PR_WHCHUNK));
  int32_t k = 0;
  double resid = 0.0;
  LAGR_TRY(pr_solve(2, G, P, P->pr_adj, G->rowptr, G->colidx, G->val, lam.p, sc.p, teleport, dL_drank, nullptr,
                    damping, tol, itermax, dangling, st.p, &k, &resid, s, msg));
  if (dL_dw && G->nnz > 0) {
    // every row, heavy ones included, lies in some block's contiguous entry range
    pr_edge_grad<<<P->pr_a.nblk, PR_THREADS, 0, s>>>(G->rowptr, G->colidx, P->pr_a.blk, r, lam.p, damping, dL_dw);
    LAGR_LAUNCH_CHECK();
  }
  if (dL_dteleport) {
    // delta = dangling mass of r, through the init reduction (aux slot)
    Temp<PrSums> partials(s);
    Temp<float> scratch(s);
    const int ib = init_blocks();
    LAGR_TRY(partials.alloc(ib, msg, "partials"));
    LAGR_TRY(scratch.alloc(G->n, msg, "scratch"));
    pr_init<1><<<ib, PR_THREADS, 0, s>>>(G->n, scratch.p, nullptr, sc.p, r, teleport, 1.0f / (float)G->n,
                                                   partials.p);
    pr_finalize<<<PR_FIN_BLOCKS, PR_FIN_THREADS, 0, s>>>(partials.p, ib, st.p, 1, damping, dangling, 0.0,
                                                         1, 1);
    pr_teleport_grad<<<grid_for(G->n, 256), 256, 0, s>>>(G->n, lam.p, st.p, damping, dangling, dL_dteleport);
    LAGR_LAUNCH_CHECK();
  }
  LAGR_CUDA_TRY(cudaStreamSynchronize(s));
  if (iters) *iters = k;
  G->last_iters = k;
  G->last_resid = resid;
  if (tol > 0.0f && !(resid < (double)tol)) {
    set_msg(msg, "adjoint stopped at itermax=%d with relative L1 change %g >= tol %g", itermax, resid, (double)tol);
    return LAGR_WARN_NOT_CONVERGED;
  }
  clear_msg(msg);
  return LAGR_OK;
}
