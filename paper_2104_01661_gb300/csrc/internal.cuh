// Internal helpers shared by the library's translation units: error/message
// handling, the allocator hook, device-side warp/block primitives and the
// private per-graph state.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "lagr.h"

#define LAGR_FULL_MASK 0xffffffffu

namespace lagr {

// ---------------------------------------------------------------------------------------------
// messages and error propagation (return codes: 0 ok, < 0 error, > 0 warning)
// ---------------------------------------------------------------------------------------------

void set_msg(char *msg, const char *fmt, ...);
inline void clear_msg(char *msg) {
  if (msg) msg[0] = 0;
}

#define LAGR_CUDA_TRY(call)                                                                   \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess) {                                                                 \
      cudaGetLastError(); /* a failed call must not leave its code for the next check */      \
      ::lagr::set_msg(msg, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
      return LAGR_ERR_CUDA;                                                                   \
    }                                                                                         \
  } while (0)

#define LAGR_LAUNCH_CHECK() LAGR_CUDA_TRY(cudaGetLastError())

#define LAGR_TRY(call)      \
  do {                      \
    int st__ = (call);      \
    if (st__ < 0) return st__; \
  } while (0)

// ---------------------------------------------------------------------------------------------
// device memory through the user-settable allocator
// ---------------------------------------------------------------------------------------------

void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// allocate `count` elements of T into *p; reports LAGR_ERR_OUT_OF_MEMORY with a message
template <class T>
int alloc_n(T **p, size_t count, cudaStream_t s, char *msg, const char *what) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  *p = static_cast<T *>(dev_alloc(bytes, s));
  if (!*p) {
    set_msg(msg, "out of device memory allocating %s (%zu bytes)", what, bytes);
    return LAGR_ERR_OUT_OF_MEMORY;
  }
  return LAGR_OK;
}

// scoped temporary: freed (stream-ordered) when it goes out of scope
template <class T>
struct Temp {
  T *p = nullptr;
  cudaStream_t s = nullptr;
  explicit Temp(cudaStream_t st) : s(st) {}
  ~Temp() {
    if (p) dev_free(p, s);
  }
  int alloc(size_t count, char *msg, const char *what) { return alloc_n(&p, count, s, msg, what); }
  Temp(const Temp &) = delete;
  Temp &operator=(const Temp &) = delete;
};

// ---------------------------------------------------------------------------------------------
// private per-graph state (behind lagr_graph_struct::priv)
// ---------------------------------------------------------------------------------------------

// Partition of the rows of a CSR for the row-block kernels (PageRank gathers, the triangle-count
// orientation): rows of at most ROW_HEAVY entries are grouped into blocks of at most ROW_UNITS
// units (a unit is one entry or one row); longer rows are listed in `heavy` (ascending), each a
// block of its own, and handled by CTAs of their own.  A block's entries are contiguous, at most
// ROW_UNITS + ROW_HEAVY of them unless the block is a heavy row.
constexpr int ROW_UNITS = 4096;
constexpr int ROW_HEAVY = 4096;
struct RowPlan {
  int32_t *blk = nullptr;    // [nblk + 1] first row of each block, blk[nblk] = n
  int32_t nblk = -1;         // -1 until built
  int32_t *heavy = nullptr;  // [nheavy] rows longer than the threshold
  int32_t nheavy = 0;
  // heavy rows are cut into chunks of ROW_HCHUNK entries: chunks hc_off[h] .. hc_off[h+1]-1
  // belong to heavy[h]; hc_row[c] is the heavy index of chunk c
  int32_t *hc_off = nullptr;  // [nheavy + 1]
  int32_t *hc_row = nullptr;  // [nhc]
  int32_t nhc = 0;
  uint8_t *hblk = nullptr;    // [nblk] 1 where the block is one heavy row (every heavy row is a block of its own)
  int32_t units = 0, heavy_len = 0, hchunk = 0;  // the plan's block size, heavy-row threshold and chunk
};
constexpr int ROW_HCHUNK = 8192;
// the finer plan of the warp-per-block gathers (PageRank, FastSV): blocks of one warp's work
constexpr int FINE_UNITS = 1024;   // units per block
constexpr int FINE_HEAVY = 1024;   // longer rows are cut into chunks of FINE_HCHUNK entries
constexpr int FINE_HCHUNK = 2048;

struct Priv {
  // small device scratch: counters and flags used by every algorithm
  int64_t *dscal = nullptr;  // LAGR_NSCAL int64 slots
  int64_t *hscal = nullptr;      // pinned host mirror (LAGR_NHOST slots) ...
  int64_t *hscal_dev = nullptr;  // ... and its address for kernels, which write it directly
  // triangle counting: anchors of the warp class and CTA-class items (x, first neighbour)
  int32_t *tc_listw = nullptr;
  int2 *tc_listc = nullptr;
  int32_t *tc_rank = nullptr;   // degree rank (the A(p,p) labels of Alg. 6) or the id
  int32_t *tc_sortbuf = nullptr;  // 4n keys/values/work for the rank sort
  int32_t *tc_radix = nullptr;  // radix scratch
  int64_t *tc_radix_scan = nullptr;
  int64_t tc_capc = 0;
  int2 *tc_listwh = nullptr;  // warp items of the warp anchors with many neighbours
  int64_t tc_capwh = 0;
  // row plans: over the rows of A' (shared by the triangle orientation and the 64-source BFS pull)
  // and of A (the adjoint's edge gradient), in blocks of ROW_UNITS; and the finer plans of the
  // PageRank gathers (blocks of one warp's work) over A' (forward) and A (adjoint)
  RowPlan pr_at, pr_a, pr_fwd, pr_adj;
};

enum ScalarSlot {
  SC_ERR = 0,      // device error flag (LAGR_ERR_* or 0)
  SC_COUNT0 = 1,   // generic counters
  SC_COUNT1 = 2,
  SC_COUNT2 = 3,
  SC_COUNT3 = 4,
  SC_COUNT4 = 5,
  SC_COUNT5 = 6,
  SC_COUNT6 = 7,
  SC_COUNT7 = 8,
  SC_COUNT8 = 9,
  SC_COUNT9 = 10,
  SC_COUNT10 = 11,
  SC_COUNT11 = 12,
  SC_COUNT12 = 13,
  LAGR_NSCAL = 16,
  LAGR_NHOST = 64  // int64 slots of the pinned host mirror (also stages up to 64 int32 sources)
};

int priv_get(lagr_graph G, cudaStream_t s, char *msg, Priv **out);

// Small device-to-host reads that bypass the copy engines (a large copy queued on another stream
// would delay them): a one-warp kernel stores the values into pinned, device-mapped host memory,
// the stream is synchronised, and the values are copied out.  fetch_to_host reads `bytes`
// contiguous bytes (a multiple of 4, at most LAGR_NHOST * 8); fetch_i32s gathers `count` (<= 8)
// scalars from separate addresses.
int fetch_to_host(void *dst, const void *dsrc, size_t bytes, cudaStream_t s, char *msg);
// the recycled pinned, device-mapped blocks behind them (LAGR_NHOST int64 each: h for the host,
// d for kernels); get returns false when pinned memory runs out
struct HostBlock {
  int64_t *h, *d;
};
bool host_block_get(HostBlock *b);
void host_block_put(HostBlock b);
int fetch_i32s(int32_t *dst, const int32_t *const *srcs, int count, cudaStream_t s, char *msg);

// build (once; no-op when pl->nblk >= 0) the row plan of a CSR.  Synchronises the stream.
int row_plan(RowPlan *pl, const int32_t *rowptr, int32_t n, cudaStream_t s, char *msg, int32_t units = ROW_UNITS,
             int32_t heavy = ROW_HEAVY, int32_t hchunk = ROW_HCHUNK);

// Opt-in device timing of the hot kernels (lagr_timing_*): construct a KTimer right before a
// launch and let it go out of scope right after; it records an event pair on the stream when
// timing is on and the stream is not capturing.
enum TimedKernel { TK_PR_GATHER = 0, TK_TC_CTA, TK_TC_WARP, TK_BFS_SMALL, TK_BFS_LB, TK_BFS_PULL, TK_COUNT };
struct KTimer {
  KTimer(TimedKernel k, cudaStream_t s);
  ~KTimer();
  KTimer(const KTimer &) = delete;
  KTimer &operator=(const KTimer &) = delete;
  TimedKernel k;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
};
void priv_release(lagr_graph G, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// launch geometry: grids are sized from the device they run on, never from one GPU model's
// multiprocessor count
// ---------------------------------------------------------------------------------------------

// multiprocessors of the current device (queried once per device)
int sm_count();
// CTAs of `kernel` with `threads` threads and `smem` bytes of dynamic shared memory that are
// resident on the current device at once (occupancy query x sm_count(), cached per kernel and
// device); at least sm_count()
int resident_ctas(const void *kernel, int threads, size_t smem);
// grid of a grid-stride kernel over `work` items: one CTA per `threads` items, at most `waves`
// CTAs per multiprocessor
int grid_for(int64_t work, int threads, int waves = 16);
// count a launch that does not go through <<<...>>> (a cooperative launch) in lagr_kernel_launches
void note_launch();

// validation shared by the entry points
int check_graph_arg(lagr_graph G, char *msg);

// ---------------------------------------------------------------------------------------------
// triangle counting internals (tc.cu), shared with the batched path
// ---------------------------------------------------------------------------------------------

struct TcParams {
  int chunk;  // neighbours per CTA work item
  int wmax;   // anchors with d+ <= wmax (and moderate degree) run one per warp
};
TcParams tc_default_params();
int tc_alloc(lagr_graph G, Priv *P, TcParams prm, cudaStream_t s, char *msg);
int tc_launch(lagr_graph G, Priv *P, int method, TcParams prm, const int32_t *voff, int32_t ngraphs,
              unsigned long long *counts, bool orient, cudaStream_t s, char *msg, bool count = true);
unsigned long long *tc_total_slot(Priv *P);

// ---------------------------------------------------------------------------------------------
// PageRank internals (pagerank.cu), shared with the batched path: a plan holds every buffer of
// the unweighted (GAP form) iteration so that a fixed number of iterations can be enqueued
// without allocation or host synchronisation.
// ---------------------------------------------------------------------------------------------

struct PrPlan;
int pr_plan_create(PrPlan **out, lagr_graph G, Priv *P, float damping, const float *vvec, cudaStream_t s,
                   char *msg);
int pr_plan_enqueue(PrPlan *pl, float *out, const float *warm, int32_t iters, cudaStream_t s, char *msg);
void pr_plan_destroy(PrPlan *pl, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// scans (scan.cu)
// ---------------------------------------------------------------------------------------------

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total.  The total must fit int32
// (device flag SC_ERR is not used; callers pass sizes where this holds).
// scratch: NULL (allocated here) or scan_scratch_len(n) int64 work slots (nothing is allocated then,
// so the call can be captured in a CUDA graph).
int exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, char *msg,
                   int64_t *scratch = nullptr);
int64_t scan_scratch_len(int64_t n);

// stable ascending radix sort of (keys, vals) by the low `bits` bits of keys.  keys/vals are
// sorted in place; tmp_k/tmp_v are work arrays of the same length.  scratch: NULL or
// radix_scratch_len(n) int32 slots, scan_scratch: NULL or scan_scratch_len(radix_scratch_len(n))
// int64 slots (with both given nothing is allocated).
int64_t radix_scratch_len(int64_t n);
int radix_sort_pairs(int32_t *keys, int32_t *vals, int32_t *tmp_k, int32_t *tmp_v, int64_t n,
                     int bits, cudaStream_t s, char *msg, int32_t *scratch = nullptr,
                     int64_t *scan_scratch = nullptr);


// CSR -> CSC (A' by row) with rows sorted; at_val may be NULL when val is NULL.
int transpose_csr(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                  const float *val, int32_t *at_rowptr, int32_t *at_colidx, float *at_val,
                  cudaStream_t s, char *msg);

// ---------------------------------------------------------------------------------------------
// device primitives
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LAGR_FULL_MASK, v, o);
  return v;
}

// inclusive prefix sum over the 32 lanes
__device__ __forceinline__ int warp_inclusive_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(LAGR_FULL_MASK, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// sum over a whole block; every thread must call it; result valid in every thread
template <class T>
__device__ T block_sum(T v, T *smem /* >= 32 elements */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  T r = (threadIdx.x < nwarps) ? smem[threadIdx.x] : T(0);
  if (warp == 0) r = warp_sum(r);
  if (threadIdx.x == 0) smem[0] = r;
  __syncthreads();
  r = smem[0];
  __syncthreads();
  return r;
}

// Load-balanced walk over 32 segments (one per lane: start st, length len, a per-segment tag;
// len 0 = empty).  Calls f(valid, tag_of_segment, position_in_segment, global_index) once per
// round on EVERY lane, spreading the elements of all segments evenly over the 32 lanes; lanes
// with valid == false have no element this round (their other arguments are meaningless).
// Because every lane calls f, f may use warp-collective operations.  Warp-collective itself.
template <class F>
__device__ __forceinline__ void warp_segments(int st, int len, int tag, F &&f) {
  const int lane = threadIdx.x & 31;
  const int incl = warp_inclusive_scan(len);
  const int total = __shfl_sync(LAGR_FULL_MASK, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int k = base + lane;
    int lo = 0, hi = 31;
#pragma unroll
    for (int step = 0; step < 5; step++) {
      const int mid = (lo + hi) >> 1;
      const int v = __shfl_sync(LAGR_FULL_MASK, incl, mid);
      if (v > k) hi = mid; else lo = mid + 1;
    }
    const int s = lo;
    const int incl_s = __shfl_sync(LAGR_FULL_MASK, incl, s);
    const int len_s = __shfl_sync(LAGR_FULL_MASK, len, s);
    const int st_s = __shfl_sync(LAGR_FULL_MASK, st, s);
    const int tag_s = __shfl_sync(LAGR_FULL_MASK, tag, s);
    const int off = k - (incl_s - len_s);
    f(k < total, tag_s, off, st_s + off);
  }
}

}  // namespace lagr
