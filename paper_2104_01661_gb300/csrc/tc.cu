// Triangle counting (Alg. 6, Sec. IV-E): t = sum(C) with C<s(L)> = L plus.pair U', fused so
// that C is never formed (the materialised C is what the paper blames for its 3x gap to GAP).
//
// Labels.  Alg. 6 relabels A by the ascending-degree permutation p (A(p,p)) before splitting it
// into L = tril and U = triu.  Here p comes from a stable radix sort of the degrees (ties by id),
// and rank[v] is v's position in it (rank[v] = v when Alg. 6 decides not to sort).  The rows of A
// are not moved: U(v,:) = { rank(u) : u in A(v,:), rank(u) > rank(v) } is stored for every
// original vertex v, its entries being ranks, which is triu(A(p,p),1) with the rows renamed back.
// L = U', so for every stored (i,j) of L, C(i,j) = |L(i,:) n U(j,:)| = |U(i,:) n U(j,:)| in rank
// space: the count of each undirected edge {x,y} is the intersection of the two oriented lists,
// and summed over the edges this counts each triangle once.
//
// Intersection.  Each edge {x,y} is anchored at the endpoint with the larger (d+, id); the
// anchor's list goes into a shared-memory set once and the other (shorter) list is probed.  The
// set is a bitmap over the top ranks (the window) plus a small hash table for the entries below
// it: after the degree ordering nearly every entry of a long list is a high-degree vertex, so a
// probe is one shared-memory word, and an entry ranked below the anchor is rejected without any
// lookup (it cannot be in the anchor's list).  Anchors with short lists run one per warp; long
// lists or many neighbours run one CTA per (anchor, chunk of neighbours).
#include <algorithm>
#include <atomic>
#include <cstring>

#include "internal.cuh"

namespace lagr {
namespace {

constexpr int TCW_WARPS = 8;          // warps per CTA in the warp-anchor kernel
constexpr int TCW_SLOTS = 512;        // hash slots per warp (entries below the window)
constexpr int TCW_MAXD = TCW_SLOTS / 2;  // warp anchors: d+ <= wmax <= 256 ...
constexpr int TCW_MAXDEG = 4096;      // ... and degree <= 4096
constexpr int TCW_HEAVY = 8192;      // warp anchors with deg * d+ above this are queued first
constexpr int TCW_ITEMWORK = 65536;  // ... and above this cut into items of TCW_CHUNK neighbours
constexpr int TCW_CHUNK = 256;
constexpr int TCW_GRAB = 8;          // whole-anchor warp items taken per queue atomic
constexpr int TCW_WIN_LOG = 15;       // per-warp window: the top 32768 ranks (4 KB of bits)
constexpr int TCC_THREADS = 512;      // CTA-anchor kernel
constexpr int TCC_SLOTS = 8192;       // hash slots per CTA (32 KB)
constexpr int TCC_WIN_LOG = 17;       // per-CTA window: the top 131072 ranks (16 KB of bits)
constexpr int TCC_CHUNK = 4096;       // default neighbours per CTA work item
constexpr int TCC_MAXCHUNK = 4096;    // most neighbours per CTA work item
constexpr int32_t EMPTY = -1;
constexpr size_t TCW_SMEM = (size_t)TCW_WARPS * (((1 << TCW_WIN_LOG) / 32) * 4 + TCW_SLOTS * 4);
constexpr size_t TCC_SMEM = ((1 << TCC_WIN_LOG) / 32) * 4 + TCC_SLOTS * 4;

// slots of the per-graph device scalars used here
constexpr int SL_SORT = SC_COUNT0;
constexpr int SL_DECIDE = SC_COUNT1;
constexpr int SL_NW = SC_COUNT2;
constexpr int SL_NC = SC_COUNT3;
constexpr int SL_NWL = SC_COUNT4;  // light warp anchors (one item each), stored from the end of listw
constexpr int SL_QW = SC_COUNT5;   // queue cursor of the chunked warp items (SL_NW of them)
constexpr int SL_QC = SC_COUNT6;
constexpr int SL_TOTAL = SC_COUNT7;
constexpr int SL_QWL = SC_COUNT8;  // queue cursor of the whole-anchor warp items
constexpr int SL_NWF = SC_COUNT9;  // heavier warp anchors (one item each), stored from the front of listw
constexpr int SL_NSW = SC_COUNT10;  // U rows listed for the warp sorter, up to TC_SORT_SMALL entries
constexpr int SL_NSC = SC_COUNT11;  // U rows listed for the CTA sorter
constexpr int SL_NSM = SC_COUNT12;  // U rows listed for the warp sorter, longer than TC_SORT_SMALL

__device__ __forceinline__ uint32_t hslot(int32_t w, int logT) {
  return ((uint32_t)w * 0x9E3779B1u) >> (32 - logT);
}

__device__ __forceinline__ void hinsert(int32_t *tab, int logT, int32_t w) {
  const uint32_t mask = (1u << logT) - 1;
  uint32_t h = hslot(w, logT);
  // the table holds at least twice the entries inserted, so a free slot exists; the bound only
  // guarantees termination
  for (uint32_t i = 0; i <= mask && atomicCAS(&tab[h], EMPTY, w) != EMPTY; i++) h = (h + 1) & mask;
}

__device__ __forceinline__ int hprobe(const int32_t *tab, int logT, int32_t w) {
  const uint32_t mask = (1u << logT) - 1;
  uint32_t h = hslot(w, logT);
  for (uint32_t i = 0; i <= mask; i++) {
    const int32_t v = tab[h];
    if (v == w) return 1;
    if (v == EMPTY) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

// The anchor's list as a set of ranks: a bitmap over the window [w0, w0 + window) and a hash table
// for the entries below w0.  `scan` (CTA anchors only): too many entries below the window for the
// table, so those are found by scanning the list in memory instead.
struct RankSet {
  uint32_t *bm;
  int32_t *tab;
  int logT;
  int32_t w0, rx;
  const int32_t *list;  // the anchor's list in memory (scan mode)
  int32_t len;
  bool scan;   // entries below the window are found by scanning `list`
  bool below;  // the anchor has entries below the window (otherwise the table is not used at all)
  __device__ __forceinline__ void insert(int32_t w) const {
    if (w >= w0) atomicOr(&bm[(w - w0) >> 5], 1u << ((w - w0) & 31));
    else if (!scan) hinsert(tab, logT, w);
  }
  __device__ __forceinline__ void erase(int32_t w) const {
    if (w >= w0) bm[(w - w0) >> 5] = 0u;
  }
  // the anchor has no entries below the window (below == false): the bitmap decides alone, with
  // no branch (ranks below w0 read word 0 and are masked off)
  __device__ __forceinline__ uint32_t has_window(int32_t w) const {
    const int32_t d = w - w0;
    return (bm[max(d, 0) >> 5] >> (d & 31)) & (uint32_t)(d >= 0);
  }
  __device__ __forceinline__ uint32_t has(int32_t w) const {
    const int32_t d = w - w0;
    // in the window the bitmap decides alone (it holds no rank <= rx); the word is read with a
    // clamped index so that the common case has no branch
    const uint32_t in = (bm[max(d, 0) >> 5] >> (d & 31)) & 1u;
    if (d >= 0) return in;
    if (w <= rx || !below) return 0;  // the anchor's entries all rank above it
    if (!scan) return (uint32_t)hprobe(tab, logT, w);
    for (int32_t q = 0; q < len; q++)
      if (list[q] == w) return 1;
    return 0;
  }
};

__device__ __forceinline__ int ceil_log2(int32_t x) {  // x >= 1
  return x <= 1 ? 0 : 32 - __clz(x - 1);
}

// member graph of vertex x in a block-diagonal batch (voff has g+1 entries)
__device__ __forceinline__ int32_t member_of(const int32_t *__restrict__ voff, int32_t g, int32_t x) {
  int32_t lo = 0, hi = g - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (voff[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---- Alg. 6 degree heuristic: mean > 4 * median, in exact integer arithmetic -------------------
// With X = ceil(nnz / (4n)), the lower-middle median m satisfies 4nm < nnz iff m < X iff at least
// floor((n-1)/2) + 1 vertices have degree < X.
__global__ void tc_decide(const int32_t *__restrict__ rowptr, int32_t n, int64_t xstar, int64_t *__restrict__ dscal) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (int64_t)(rowptr[i + 1] - rowptr[i]) < xstar;
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long *)&dscal[SL_DECIDE], c);
}

__global__ void tc_set_mode(int32_t n, int method, int64_t *__restrict__ dscal) {
  int sort;
  if (method == LAGR_TC_SORT) sort = 1;
  else if (method == LAGR_TC_NOSORT) sort = 0;
  else sort = dscal[SL_DECIDE] >= (int64_t)((n - 1) / 2) + 1;
  dscal[SL_SORT] = sort;
}

// keys = degrees, vals = ids: their stable sort is the ascending-degree permutation of Alg. 6
__global__ void tc_rank_keys(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ keys,
                             int32_t *__restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = rowptr[i + 1] - rowptr[i];
    vals[i] = (int32_t)i;
  }
}

// rank[p[i]] = i after sorting, rank[v] = v when Alg. 6 does not sort; rank[n + 1 + i] = the vertex
// of rank i (rank has 2(n + 1) slots)
__global__ void tc_rank_scatter(const int32_t *__restrict__ vals, int32_t n, const int64_t *__restrict__ dscal,
                                int32_t *__restrict__ rank) {
  const int sort = (int)dscal[SL_SORT];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = sort ? vals[i] : (int32_t)i;
    rank[v] = (int32_t)i;
    rank[n + 1 + i] = v;  // the vertex of rank i
  }
}

// ---- orientation: d+ per vertex, then the oriented rows -------------------------------------------

// One CTA per row block (see RowPlan): the ranks of the block's neighbours are gathered into
// shared memory with coalesced colidx loads, then each short row is oriented by one thread and
// each longer row by one warp, in one pass: U(v,:) (the ranks above rank(v), in the order of
// A(v,:); ballots keep the order inside a warp) is written into the first slots of A's row v, and
// its length d+(v) to dplus[v].  Rows longer than ROW_HEAVY are left to tc_orient_heavy.
constexpr int OR_STAGE = ROW_UNITS + ROW_HEAVY + 64;
constexpr int OR_SHORT = 32;

__global__ void __launch_bounds__(256)
    tc_orient_rows(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                   const int32_t *__restrict__ rank, const int32_t *__restrict__ blk,
                   const uint8_t *__restrict__ hblk, int32_t *__restrict__ dplus, int32_t *__restrict__ u_colidx) {
  __shared__ int32_t stage[OR_STAGE];
  __shared__ int32_t longrows[ROW_UNITS / (OR_SHORT + 1) + 2];
  __shared__ int n_long;
  if (hblk[blockIdx.x]) return;  // a heavy row alone: tc_orient_heavy orients it
  const int32_t r0 = blk[blockIdx.x], r1 = blk[blockIdx.x + 1];
  const int32_t e0 = rowptr[r0], e1 = rowptr[r1];
  const bool staged = e1 - e0 <= OR_STAGE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) n_long = 0;
  if (staged) {
    int32_t k = e0 + threadIdx.x;
    for (; k + 7 * 256 < e1; k += 8 * 256) {  // eight gathers per thread in flight
      int32_t d[8];
#pragma unroll
      for (int i = 0; i < 8; i++) d[i] = __ldg(&rank[colidx[k + i * 256]]);
#pragma unroll
      for (int i = 0; i < 8; i++) stage[k + i * 256 - e0] = d[i];
    }
    for (; k < e1; k += 256) stage[k - e0] = __ldg(&rank[colidx[k]]);
  }
  __syncthreads();
  auto ru_of = [&](int32_t q) { return staged ? stage[q - e0] : __ldg(&rank[colidx[q]]); };
  for (int32_t v = r0 + threadIdx.x; v < r1; v += 256) {
    const int32_t b = rowptr[v], e = rowptr[v + 1], dv = e - b;
    if (dv <= OR_SHORT) {
      const int32_t rv = rank[v];
      int32_t out = b;
      for (int32_t q = b; q < e; q++) {
        const int32_t ru = ru_of(q);
        if (ru > rv) u_colidx[out++] = ru;  // out < e: the slots of row v
      }
      dplus[v] = out - b;
    } else if (dv <= ROW_HEAVY) {
      longrows[atomicAdd(&n_long, 1)] = v;
    }
  }
  __syncthreads();
  const unsigned lt = lanemask_lt();
  for (int q = warp; q < n_long; q += 8) {
    const int32_t v = longrows[q];
    const int32_t b = rowptr[v], e = rowptr[v + 1], rv = rank[v];
    int32_t out = b;
    for (int32_t base = b; base < e; base += 32) {
      const int32_t k = base + lane;
      int32_t ru = 0;
      bool f = false;
      if (k < e) {
        ru = ru_of(k);
        f = ru > rv;
      }
      const unsigned bal = __ballot_sync(LAGR_FULL_MASK, f);
      if (f) u_colidx[out + __popc(bal & lt)] = ru;
      out += __popc(bal);
    }
    if (lane == 0) dplus[v] = out - b;
  }
}

// The rows longer than ROW_HEAVY, in the row plan's chunks of ROW_HCHUNK entries, a CTA per chunk,
// so that a hub row is spread over many SMs: each warp gathers the ranks of 256 entries at a time
// (eight per lane in flight), compacts those above rank(v) with ballots and reserves their slots
// of U(v) with one atomic on d+(v) (zeroed first by tc_orient_heavy_zero).  U(v) then keeps A's
// order within each warp's run but not between runs, which nothing relies on: the U rows of 32 to
// 16384 entries are sorted afterwards, and the other lists are walked or probed whole.
constexpr int OH_THREADS = 256;
constexpr int OH_PER = 8;  // entries per lane per round

__global__ void tc_orient_heavy_zero(const int32_t *__restrict__ heavy, int32_t nh, int32_t *__restrict__ dplus) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x)
    dplus[heavy[h]] = 0;
}

__global__ void __launch_bounds__(OH_THREADS)
    tc_orient_heavy(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                    const int32_t *__restrict__ rank, int32_t *__restrict__ dplus, int32_t *__restrict__ u_colidx,
                    const int32_t *__restrict__ heavy, const int32_t *__restrict__ hc_off,
                    const int32_t *__restrict__ hc_row, int32_t nhc, int32_t hchunk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  for (int64_t c = blockIdx.x; c < nhc; c += gridDim.x) {
    const int32_t h = hc_row[c];
    const int32_t v = heavy[h];
    const int32_t rv = rank[v], row0 = rowptr[v];
    const int32_t b = row0 + (int32_t)(c - hc_off[h]) * hchunk;
    const int32_t e = min(rowptr[v + 1], b + hchunk);
    for (int32_t base = b + warp * 32 * OH_PER; base < e; base += OH_THREADS * OH_PER) {
      int32_t u[OH_PER];
      unsigned bal[OH_PER];
      int tot = 0;
#pragma unroll
      for (int i = 0; i < OH_PER; i++) {
        const int32_t k = base + i * 32 + lane;
        u[i] = k < e ? __ldg(&rank[colidx[k]]) : -1;
      }
#pragma unroll
      for (int i = 0; i < OH_PER; i++) {
        bal[i] = __ballot_sync(LAGR_FULL_MASK, u[i] > rv);
        tot += __popc(bal[i]);
      }
      int32_t out = 0;
      if (lane == 0 && tot) out = atomicAdd(&dplus[v], tot);
      out = row0 + __shfl_sync(LAGR_FULL_MASK, out, 0);
#pragma unroll
      for (int i = 0; i < OH_PER; i++) {
        if (u[i] > rv) u_colidx[out + __popc(bal[i] & lt)] = u[i];
        out += __popc(bal[i]);
      }
    }
  }
}

// ---- U rows in descending rank order ------------------------------------------------------------
//
// A probe list of at least 32 entries is walked by a whole warp (anchor_batch), and such a walk can
// stop at the list's first entry ranked at or below the anchor if the list is in descending rank
// order: no later entry can be in the anchor's list.  So every U row of 32 .. TC_SORT_MAX entries
// is sorted (bitonic networks: by a warp in registers up to TC_SORT_WARP entries, by a CTA in
// shared memory above); shorter rows are probed entry by entry anyway, and longer rows keep their
// order and are walked to the end.  The rows to sort are listed first.
constexpr int TC_SORT_MIN = 32;
constexpr int TC_SORT_SMALL = 256;  // rows up to this long are sorted by the low-register warp sorter
constexpr int TC_SORT_WARP = 1024;
constexpr int TC_SORT_MAX = 16384;
constexpr int TCS_WARPS = 4;  // warps per CTA of the warp sorter

// the rows to sort, as (first entry, length) pairs: TC_SORT_MIN..TC_SORT_SMALL entries to lists
// from the front, TC_SORT_SMALL..TC_SORT_WARP to listm from its end backwards, longer to listc
// from the front (listm and listc share n slots: a vertex is in at most one list)
__global__ void tc_sort_collect(const int32_t *__restrict__ ustart, const int32_t *__restrict__ dplus, int32_t n,
                                int2 *__restrict__ lists, int2 *__restrict__ listc, int2 *__restrict__ listm_end,
                                int64_t *__restrict__ dscal) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane;
    const int32_t d = v < n ? dplus[v] : 0;
    const bool w = d >= TC_SORT_MIN && d <= TC_SORT_SMALL, m = d > TC_SORT_SMALL && d <= TC_SORT_WARP,
               c = d > TC_SORT_WARP && d <= TC_SORT_MAX;
    const unsigned bw = __ballot_sync(LAGR_FULL_MASK, w), bm = __ballot_sync(LAGR_FULL_MASK, m),
                   bc = __ballot_sync(LAGR_FULL_MASK, c);
    unsigned long long pw = 0, pm = 0, pc = 0;
    if (lane == 0 && bw) pw = atomicAdd((unsigned long long *)&dscal[SL_NSW], (unsigned long long)__popc(bw));
    if (lane == 0 && bm) pm = atomicAdd((unsigned long long *)&dscal[SL_NSM], (unsigned long long)__popc(bm));
    if (lane == 0 && bc) pc = atomicAdd((unsigned long long *)&dscal[SL_NSC], (unsigned long long)__popc(bc));
    pw = __shfl_sync(LAGR_FULL_MASK, pw, 0);
    pm = __shfl_sync(LAGR_FULL_MASK, pm, 0);
    pc = __shfl_sync(LAGR_FULL_MASK, pc, 0);
    if (w) lists[pw + __popc(bw & lt)] = make_int2(ustart[v], d);
    if (m) *(listm_end - 1 - (int64_t)(pm + __popc(bm & lt))) = make_int2(ustart[v], d);
    if (c) listc[pc + __popc(bc & lt)] = make_int2(ustart[v], d);
  }
}

__device__ __forceinline__ void cmpx_desc(int32_t *s, int32_t i, int32_t ixj, bool desc) {
  const int32_t a = s[i], b = s[ixj];
  if ((a < b) == desc) {
    s[i] = b;
    s[ixj] = a;
  }
}

// one compare-exchange of a bitonic stage between lanes lane and lane ^ j (j < 32): in a descending
// segment the lower index keeps the larger value
__device__ __forceinline__ int32_t shfl_cmpx(int32_t x, int j, bool desc, int lane) {
  const int32_t y = __shfl_xor_sync(LAGR_FULL_MASK, x, j);
  return (((lane & j) == 0) == desc) ? max(x, y) : min(x, y);
}

// one stage of partner distance 32 * JR between the registers of one lane (element i = lane + 32 r
// sits in register r): in a descending segment (bit k of i clear) the lower index keeps the larger
template <int R, int JR>
__device__ __forceinline__ void cx_regs(int32_t (&v)[R], int k) {
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((r & JR) == 0) {
      const bool desc = ((32 * r) & k) == 0;
      const int32_t a = v[r], b = v[r | JR];
      v[r] = desc ? max(a, b) : min(a, b);
      v[r | JR] = desc ? min(a, b) : max(a, b);
    }
}

template <int R>
__device__ __forceinline__ void cx_regs_any(int32_t (&v)[R], int jr, int k) {
  if constexpr (R >= 2) if (jr == 1) return cx_regs<R, 1>(v, k);
  if constexpr (R >= 4) if (jr == 2) return cx_regs<R, 2>(v, k);
  if constexpr (R >= 8) if (jr == 4) return cx_regs<R, 4>(v, k);
  if constexpr (R >= 16) if (jr == 8) return cx_regs<R, 8>(v, k);
  if constexpr (R >= 32) if (jr == 16) return cx_regs<R, 16>(v, k);
}

// Bitonic sort of one row of at most P entries by one warp, in registers: element i sits in lane
// i % 32, register i / 32.  A stage of partner distance j >= 32 pairs registers of one lane, below
// 32 it pairs lanes (shuffles).  The stages run as loops over one unrolled copy of each kind of
// stage, which keeps the code small (a fully unrolled network of 1024 entries alone is thousands
// of instructions, more than the instruction caches hold for all the warps of an SM).
template <int P>
__device__ __forceinline__ void warp_sort_desc(int32_t *__restrict__ row, int32_t d, int lane) {
  constexpr int R = P / 32;
  int32_t v[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int32_t i = lane + 32 * r;
    v[r] = i < d ? row[i] : INT32_MIN;
  }
#pragma unroll 1
  for (int k = 2; k <= P; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j >= 32; j >>= 1) cx_regs_any<R>(v, j >> 5, k);
#pragma unroll 1
    for (int j = min(k >> 1, 16); j > 0; j >>= 1) {
#pragma unroll
      for (int r = 0; r < R; r++) v[r] = shfl_cmpx(v[r], j, ((lane + 32 * r) & k) == 0, lane);
    }
  }
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int32_t i = lane + 32 * r;
    if (i < d) row[i] = v[r];
  }
}

// The listed rows of up to PMAX entries: one warp each, in registers; a warp takes every nw-th row
// and loads the next row's pair while it sorts the current one.  Two instances: PMAX =
// TC_SORT_SMALL for most rows (few registers, so many warps per SM hide the shuffle latencies),
// PMAX = TC_SORT_WARP for the longer ones (list read backwards from its end when `back`).
template <int PMAX>
__global__ void __launch_bounds__(TCS_WARPS * 32)
    tc_sort_rows_warp(const int2 *__restrict__ list, int back, const int64_t *__restrict__ dscal, int slot,
                      int32_t *__restrict__ u_colidx) {
  const int lane = threadIdx.x & 31;
  const int64_t nl = dscal[slot];
  const int64_t nw = (int64_t)gridDim.x * TCS_WARPS;
  auto at = [&](int64_t i) { return back ? list[-1 - i] : list[i]; };
  int64_t it = (int64_t)blockIdx.x * TCS_WARPS + (threadIdx.x >> 5);
  int2 cur = it < nl ? at(it) : make_int2(0, 0);
  for (; it < nl; it += nw) {
    const int2 nxt = it + nw < nl ? at(it + nw) : make_int2(0, 0);
    int32_t *row = u_colidx + cur.x;
    const int32_t d = cur.y;
    if (d <= 32) warp_sort_desc<32>(row, d, lane);
    else if (d <= 64) warp_sort_desc<64>(row, d, lane);
    else if (PMAX <= 128 || d <= 128) warp_sort_desc<(PMAX < 128 ? PMAX : 128)>(row, d, lane);
    else if (PMAX <= 256 || d <= 256) warp_sort_desc<(PMAX < 256 ? PMAX : 256)>(row, d, lane);
    else if (PMAX <= 512 || d <= 512) warp_sort_desc<(PMAX < 512 ? PMAX : 512)>(row, d, lane);
    else warp_sort_desc<PMAX>(row, d, lane);
    cur = nxt;
  }
}

// one wave of a warp sorter instance: every warp resident at once
template <int PMAX>
int sort_wave_ctas() {
  return resident_ctas((const void *)tc_sort_rows_warp<PMAX>, TCS_WARPS * 32, 0);
}

// the rows of TC_SORT_WARP < d+ <= TC_SORT_MAX: one CTA each (dynamic shared memory TC_SORT_MAX ints)
constexpr int TCS_CTA_THREADS = 1024;
__global__ void __launch_bounds__(TCS_CTA_THREADS)
    tc_sort_rows_cta(const int2 *__restrict__ list, const int64_t *__restrict__ dscal,
                     int32_t *__restrict__ u_colidx) {
  extern __shared__ int32_t sbig[];
  const int64_t nl = dscal[SL_NSC];
  for (int64_t it = blockIdx.x; it < nl; it += gridDim.x) {
    const int2 item = list[it];
    const int32_t d = item.y;
    int32_t *row = u_colidx + item.x;
    int32_t P = TC_SORT_WARP * 2;
    while (P < d) P <<= 1;
    for (int32_t i = threadIdx.x; i < P; i += blockDim.x) sbig[i] = i < d ? row[i] : INT32_MIN;
    __syncthreads();
    for (int32_t k = 2; k <= P; k <<= 1)
      for (int32_t j = k >> 1; j > 0; j >>= 1) {
        for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
          const int32_t ixj = i ^ j;
          if (ixj > i) cmpx_desc(sbig, i, ixj, (i & k) == 0);
        }
        __syncthreads();
      }
    for (int32_t i = threadIdx.x; i < d; i += blockDim.x) row[i] = sbig[i];
    __syncthreads();
  }
}

// ---- anchors: warp class (short list, moderate degree) and CTA items -------------------------------

__global__ void tc_classify(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ dplus, int32_t n,
                            int32_t *__restrict__ listw, int2 *__restrict__ listwh, int64_t capwh,
                            int2 *__restrict__ listc, int64_t capc, int64_t *__restrict__ dscal, int wmax,
                            int chunk, const int32_t *__restrict__ by_rank) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    // anchors in descending rank order: the CTA items of the top ranks first, whose walks read
    // the top of the same lists, so that anchors in flight together share more of them in L2
    const int64_t i = base + lane;
    const int64_t v = i < n ? (int64_t)by_rank[n - 1 - i] : i;
    int32_t a = 0, dg = 0;
    if (i < n) {
      a = dplus[v];
      dg = rowptr[v + 1] - rowptr[v];
    }
    const bool active = a > 0;
    const bool is_w = active && a <= wmax && dg <= TCW_MAXDEG;
    const int nch = (active && !is_w) ? (dg + chunk - 1) / chunk : 0;
    // warp-class anchors: the few whose deg * d+ exceeds TCW_ITEMWORK are cut into items of
    // TCW_CHUNK neighbours (no warp item much longer than the others); the rest are one item each,
    // the heavier ones (deg * d+ above TCW_HEAVY) from the front of listw, the others from its
    // end, so that the warps take the long items first and the short ones last
    const int64_t work = (int64_t)dg * a;
    const bool wi = is_w && work > TCW_ITEMWORK;
    const bool wf = is_w && !wi && work > TCW_HEAVY, wl = is_w && !wi && !wf;
    const unsigned bf = __ballot_sync(LAGR_FULL_MASK, wf), bl = __ballot_sync(LAGR_FULL_MASK, wl);
    unsigned long long pf = 0, pl = 0;
    if (lane == 0 && bf) pf = atomicAdd((unsigned long long *)&dscal[SL_NWF], (unsigned long long)__popc(bf));
    if (lane == 0 && bl) pl = atomicAdd((unsigned long long *)&dscal[SL_NWL], (unsigned long long)__popc(bl));
    pf = __shfl_sync(LAGR_FULL_MASK, pf, 0);
    pl = __shfl_sync(LAGR_FULL_MASK, pl, 0);
    if (wf) listw[pf + __popc(bf & lt)] = (int32_t)v;
    if (wl) listw[(int64_t)n - 1 - (int64_t)(pl + __popc(bl & lt))] = (int32_t)v;
    const int nwi = wi ? (dg + TCW_CHUNK - 1) / TCW_CHUNK : 0;
    const int winc = warp_inclusive_scan(nwi);
    const int wtot = __shfl_sync(LAGR_FULL_MASK, winc, 31);
    unsigned long long pw = 0;
    if (lane == 31 && wtot) pw = atomicAdd((unsigned long long *)&dscal[SL_NW], (unsigned long long)wtot);
    pw = __shfl_sync(LAGR_FULL_MASK, pw, 31);
    for (int c = 0; c < nwi; c++) {
      const int64_t p = (int64_t)pw + winc - nwi + c;
      if (p < capwh) listwh[p] = make_int2((int32_t)v, c * TCW_CHUNK);
      else dscal[SC_ERR] = LAGR_ERR_INVALID_GRAPH;
    }
    // CTA items, one per chunk of `chunk` neighbours
    const int incl = warp_inclusive_scan(nch);
    const int tot = __shfl_sync(LAGR_FULL_MASK, incl, 31);
    unsigned long long pc = 0;
    if (lane == 31 && tot) pc = atomicAdd((unsigned long long *)&dscal[SL_NC], (unsigned long long)tot);
    pc = __shfl_sync(LAGR_FULL_MASK, pc, 31);
    for (int c = 0; c < nch; c++) {
      const int64_t p = (int64_t)pc + incl - nch + c;
      if (p < capc) listc[p] = make_int2((int32_t)v, c * chunk);
      else dscal[SC_ERR] = LAGR_ERR_INVALID_GRAPH;
    }
  }
}

// ---- intersection counts --------------------------------------------------------------------------

// The next long list of a batch (lowest lane set in `longs`, which is cleared), with its first
// four 32-entry groups loaded: entry base + lane of group q, or -1 past the end (-1 is in no set
// and ranks at or below every anchor, so it ends a sorted walk and counts nothing).
__device__ __forceinline__ const int32_t *next_long(unsigned &longs, int32_t st, int32_t len,
                                                    const int32_t *__restrict__ u_colidx, int32_t &ls, int32_t &f0,
                                                    int32_t &f1, int32_t &f2, int32_t &f3) {
  const int lane = threadIdx.x & 31;
  const int sl = __ffs(longs) - 1;
  longs &= longs - 1;
  const int32_t *lst = u_colidx + __shfl_sync(LAGR_FULL_MASK, st, sl);
  ls = __shfl_sync(LAGR_FULL_MASK, len, sl);  // >= 32
  f0 = lst[lane];
  f1 = lane + 32 < ls ? lst[lane + 32] : -1;
  f2 = lane + 64 < ls ? lst[lane + 64] : -1;
  f3 = lane + 96 < ls ? lst[lane + 96] : -1;
  return lst;
}

// One long list (32 entries or more) probed by the whole warp, its first block already loaded.  A
// list sorted by descending rank ends its useful part at its first entry <= rx: the walk stops
// after the first 32-entry group whose last entry is at or below rx.  Longer lists keep their
// order and are walked to the end.
template <class Probe>
__device__ __forceinline__ uint32_t walk_long(const int32_t *__restrict__ lst, int32_t ls, int32_t rx, int32_t w0,
                                              int32_t w1, int32_t w2, int32_t w3, Probe &&probe) {
  const int lane = threadIdx.x & 31;
  const bool sorted = ls >= TC_SORT_MIN && ls <= TC_SORT_MAX;
  uint32_t c = 0;
  for (int32_t base = 0;;) {  // warp-uniform: every lane runs every round
    c += probe(w0);
    if ((sorted && __shfl_sync(LAGR_FULL_MASK, w0, 31) <= rx) || base + 32 >= ls) break;
    c += probe(w1);
    if ((sorted && __shfl_sync(LAGR_FULL_MASK, w1, 31) <= rx) || base + 64 >= ls) break;
    c += probe(w2);
    if ((sorted && __shfl_sync(LAGR_FULL_MASK, w2, 31) <= rx) || base + 96 >= ls) break;
    c += probe(w3);
    if ((sorted && __shfl_sync(LAGR_FULL_MASK, w3, 31) <= rx) || base + 128 >= ls) break;
    base += 128;
    const int32_t k = base + lane;
    w0 = k < ls ? lst[k] : -1;
    w1 = k + 32 < ls ? lst[k + 32] : -1;
    w2 = k + 64 < ls ? lst[k + 64] : -1;
    w3 = k + 96 < ls ? lst[k + 96] : -1;
  }
  return c;
}

// One batch of (up to) 32 neighbours A(x, jb..min(jb+32,e)): for every neighbour y anchored at x
// (smaller (d+, id)), probe each element of U(y,:) = u_colidx[ustart[y] .. ustart[y] + dplus[y])
// against x's set.  Warp-collective.  PIPE: the long lists are software-pipelined (the first block
// of the next list is loaded while the current one is probed, and a list's first four groups come
// in one round trip); otherwise each list is walked on its own, a load issued only while the walk
// goes on (the CTA kernel: fewer registers, more resident warps).
template <bool PIPE, class Probe>
__device__ __forceinline__ unsigned long long anchor_batch(int32_t x, int32_t a, int32_t rx, int32_t jb, int32_t e,
                                                           const int32_t *__restrict__ colidx,
                                                           const int32_t *__restrict__ ustart,
                                                           const int32_t *__restrict__ u_colidx,
                                                           const int32_t *__restrict__ dplus, Probe &&probe) {
  const int lane = threadIdx.x & 31;
  uint32_t c = 0;  // this lane's matches in the batch: fewer than nnz, so 32 bits hold them
  const int32_t j = jb + lane;
  int32_t st = 0, len = 0;
  if (j < e) {
    const int32_t y = colidx[j];
    const int32_t dy = dplus[y];
    if (dy > 0 && (dy < a || (dy == a && y < x))) {
      st = ustart[y];
      len = dy;
    }
  }
  // lists of 32 or more: the whole warp walks one list at a time.  Shorter lists: when their
  // lengths are even enough (the longest at most twice the mean), each lane walks its own list;
  // otherwise the load-balanced walk spreads their elements over the lanes.
  unsigned longs = __ballot_sync(LAGR_FULL_MASK, len >= 32);
  // PIPE: the first long list's first block is loaded before the short lists are walked
  int32_t ls = 0, f0 = -1, f1 = -1, f2 = -1, f3 = -1;
  const int32_t *lst = (PIPE && longs) ? next_long(longs, st, len, u_colidx, ls, f0, f1, f2, f3) : nullptr;
  const int32_t slen = len >= 32 ? 0 : len;
  const unsigned total = __reduce_add_sync(LAGR_FULL_MASK, (unsigned)slen);
  const unsigned lmax = __reduce_max_sync(LAGR_FULL_MASK, (unsigned)slen);
  if (32u * lmax <= 2u * total) {
    const int32_t *own = u_colidx + st;
    int32_t q = 0;
    for (; q + 3 < slen; q += 4) {  // four independent loads in flight
      const int32_t w0 = own[q], w1 = own[q + 1], w2 = own[q + 2], w3 = own[q + 3];
      c += probe(w0) + probe(w1) + probe(w2) + probe(w3);
    }
    for (; q < slen; q++) c += probe(own[q]);
  } else if (total > 0) {
    warp_segments(st, slen, 0, [&](bool valid, int, int, int gidx) {
      if (valid) c += probe(u_colidx[gidx]);
    });
  }
  if (!PIPE) {
    while (longs) {
      const int sl = __ffs(longs) - 1;
      longs &= longs - 1;
      const int32_t *l = u_colidx + __shfl_sync(LAGR_FULL_MASK, st, sl);
      const int32_t len_s = __shfl_sync(LAGR_FULL_MASK, len, sl);
      // a sorted list (descending ranks) ends its useful part at its first entry <= rx
      const bool sorted = len_s >= TC_SORT_MIN && len_s <= TC_SORT_MAX;
      int32_t base = 0;  // warp-uniform: every lane runs every round
      if (sorted) {
        // four loads per lane in flight; the walk stops after the first 32-entry group whose last
        // entry is at or below rx
        for (; base + 128 <= len_s; base += 128) {
          const int32_t k = base + lane;
          const int32_t w0 = l[k], w1 = l[k + 32], w2 = l[k + 64], w3 = l[k + 96];
          c += probe(w0);
          if (__shfl_sync(LAGR_FULL_MASK, w0, 31) <= rx) { base = len_s; break; }
          c += probe(w1);
          if (__shfl_sync(LAGR_FULL_MASK, w1, 31) <= rx) { base = len_s; break; }
          c += probe(w2);
          if (__shfl_sync(LAGR_FULL_MASK, w2, 31) <= rx) { base = len_s; break; }
          c += probe(w3);
          if (__shfl_sync(LAGR_FULL_MASK, w3, 31) <= rx) { base = len_s; break; }
        }
      } else {
        for (; base + 128 <= len_s; base += 128) {  // four loads per lane in flight
          const int32_t k = base + lane;
          const int32_t w0 = l[k], w1 = l[k + 32], w2 = l[k + 64], w3 = l[k + 96];
          c += (probe(w0) + probe(w1)) + (probe(w2) + probe(w3));
        }
      }
      for (; base < len_s; base += 32) {
        const int32_t k = base + lane;
        const int32_t w = k < len_s ? l[k] : 0;
        if (k < len_s) c += probe(w);
        if (sorted && __shfl_sync(LAGR_FULL_MASK, w, min(31, len_s - 1 - base)) <= rx) break;
      }
    }
  } else if (lst) {
    for (;;) {
      int32_t nls = 0, g0 = -1, g1 = -1, g2 = -1, g3 = -1;
      const int32_t *nlst = longs ? next_long(longs, st, len, u_colidx, nls, g0, g1, g2, g3) : nullptr;
      c += walk_long(lst, ls, rx, f0, f1, f2, f3, probe);
      if (!nlst) break;
      lst = nlst;
      ls = nls;
      f0 = g0;
      f1 = g1;
      f2 = g2;
      f3 = g3;
    }
  }
  return c;
}

__global__ void __launch_bounds__(TCW_WARPS * 32, 4)
    tc_count_warp(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                  const int32_t *__restrict__ ustart, const int32_t *__restrict__ u_colidx,
                  const int32_t *__restrict__ dplus, const int32_t *__restrict__ rank,
                  const int32_t *__restrict__ listw, int32_t n, const int2 *__restrict__ listwh, int64_t capwh,
                  int64_t *__restrict__ dscal, int32_t w0,
                  const int32_t *__restrict__ voff, int32_t ngraphs, unsigned long long *__restrict__ counts) {
  extern __shared__ uint32_t wsm[];  // per warp: window bits, then hash slots
  __shared__ unsigned long long red[32];
  constexpr int WORDS = (1 << TCW_WIN_LOG) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *bm = wsm + warp * (WORDS + TCW_SLOTS);
  int32_t *tab = reinterpret_cast<int32_t *>(bm + WORDS);
  for (int i = lane; i < WORDS; i += 32) bm[i] = 0u;
  __syncwarp();
  const int64_t nwh = min(dscal[SL_NW], capwh), nwf = dscal[SL_NWF], nwl = nwf + dscal[SL_NWL];
  unsigned long long mine = 0;
  // Work items: first the chunks of the long anchors (one per queue atomic), then whole anchors,
  // TCW_GRAB per queue atomic (most are tiny: one atomic each would serialise the warps on the
  // counter), the heavier ones from the front of listw first.
  bool chunks = true;
  long long it = 0, it_end = 0;
  for (;;) {
    int32_t x, jb0, je;
    if (chunks) {
      long long c = 0;
      if (lane == 0) c = (long long)atomicAdd((unsigned long long *)&dscal[SL_QW], 1ull);
      c = __shfl_sync(LAGR_FULL_MASK, c, 0);
      if (c < nwh) {
        const int2 w = listwh[c];
        x = w.x;
        jb0 = rowptr[x] + w.y;
        je = min(rowptr[x + 1], jb0 + TCW_CHUNK);
      } else {
        chunks = false;
      }
    }
    if (!chunks) {
      if (it == it_end) {
        if (lane == 0) it = (long long)atomicAdd((unsigned long long *)&dscal[SL_QWL], (unsigned long long)TCW_GRAB);
        it = __shfl_sync(LAGR_FULL_MASK, it, 0);
        it_end = min(it + TCW_GRAB, (long long)nwl);
      }
      if (it >= nwl) break;
      x = it < nwf ? listw[it] : listw[n - 1 - (it - nwf)];
      jb0 = rowptr[x];
      je = rowptr[x + 1];
      it++;
    }
    // the anchor x's neighbours [jb0, je) against x's set (the table is cleared for every item,
    // so it is valid whether or not entries fall below w0)
    const int32_t a = dplus[x];
    const int32_t ub = ustart[x];
    RankSet rs{bm, tab, ceil_log2(2 * a), w0, rank[x], nullptr, 0, false, true};
    const int T = 1 << rs.logT;
    for (int i = lane; i < T; i += 32) tab[i] = EMPTY;
    __syncwarp();
    bool lb = false;  // entries below the window: without any, the bitmap decides alone
    for (int i = lane; i < a; i += 32) {
      const int32_t w = u_colidx[ub + i];
      lb |= w < w0;
      rs.insert(w);
    }
    rs.below = __any_sync(LAGR_FULL_MASK, lb);
    __syncwarp();
    unsigned long long c = 0;
    if (rs.below) {
      for (int32_t jb = jb0; jb < je; jb += 32)
        c += anchor_batch<true>(x, a, rs.rx, jb, je, colidx, ustart, u_colidx, dplus,
                                [&](int32_t w) { return rs.has(w); });
    } else {
      for (int32_t jb = jb0; jb < je; jb += 32)
        c += anchor_batch<true>(x, a, rs.rx, jb, je, colidx, ustart, u_colidx, dplus,
                                [&](int32_t w) { return rs.has_window(w); });
    }
    __syncwarp();
    for (int i = lane; i < a; i += 32) rs.erase(u_colidx[ub + i]);
    if (voff) {
      c = warp_sum(c);
      if (lane == 0 && c) atomicAdd(&counts[member_of(voff, ngraphs, x)], c);
    } else {
      mine += c;
    }
    __syncwarp();
  }
  if (!voff) {
    mine = block_sum(mine, red);
    if (threadIdx.x == 0 && mine) atomicAdd(&counts[0], mine);
  }
}

__global__ void __launch_bounds__(TCC_THREADS)
    tc_count_cta(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                 const int32_t *__restrict__ ustart, const int32_t *__restrict__ u_colidx,
                 const int32_t *__restrict__ dplus, const int32_t *__restrict__ rank, const int2 *__restrict__ listc,
                 int64_t *__restrict__ dscal, int32_t w0, const int32_t *__restrict__ voff, int32_t ngraphs,
                 unsigned long long *__restrict__ counts, int chunk, int64_t capc) {
  extern __shared__ uint32_t csm[];  // window bits, then hash slots
  constexpr int WORDS = (1 << TCC_WIN_LOG) / 32;
  uint32_t *bm = csm;
  int32_t *tab = reinterpret_cast<int32_t *>(csm + WORDS);
  __shared__ long long s_it;
  __shared__ int32_t s_next;  // next neighbour batch of the current item
  __shared__ int32_t s_below;  // entries of the anchor's list below the window
  __shared__ unsigned long long red[32];
  const int lane = threadIdx.x & 31;
  const int64_t nc = min(dscal[SL_NC], capc);  // never read past the list (an overflow sets SC_ERR)
  for (int i = threadIdx.x; i < WORDS; i += blockDim.x) bm[i] = 0u;
  unsigned long long mine = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_it = (long long)atomicAdd((unsigned long long *)&dscal[SL_QC], 1ull);
      if (s_it < nc) s_next = rowptr[listc[s_it].x] + listc[s_it].y;
      s_below = 0;
    }
    __syncthreads();
    const long long it = s_it;
    if (it >= nc) break;
    const int2 item = listc[it];
    const int32_t x = item.x;
    const int32_t a = dplus[x];
    const int32_t ub = ustart[x];
    // how many entries fall below the window decides between the hash table and a scan
    int below = 0;
    for (int i = threadIdx.x; i < a; i += blockDim.x) below += u_colidx[ub + i] < w0;
    below = __reduce_add_sync(LAGR_FULL_MASK, below);
    if (lane == 0 && below) atomicAdd(&s_below, below);
    __syncthreads();
    const int32_t nb = s_below;
    const bool scan = nb > TCC_SLOTS / 2;
    const RankSet rs{bm, tab, (nb > 0 && !scan) ? ceil_log2(2 * nb) : 1, w0, rank[x], u_colidx + ub, a, scan, nb > 0};
    if (nb > 0 && !scan) {
      const int T = 1 << rs.logT;
      for (int i = threadIdx.x; i < T; i += blockDim.x) tab[i] = EMPTY;
      __syncthreads();
    }
    for (int i = threadIdx.x; i < a; i += blockDim.x) rs.insert(u_colidx[ub + i]);
    __syncthreads();
    const int32_t b = rowptr[x] + item.y;
    const int32_t e = min(rowptr[x + 1], b + chunk);
    unsigned long long c = 0;
    // warps take the item's neighbour batches one at a time, so they reach the barrier together
    for (;;) {
      int32_t jb = 0;
      if (lane == 0) jb = atomicAdd(&s_next, 32);
      jb = __shfl_sync(LAGR_FULL_MASK, jb, 0);
      if (jb >= e) break;
      c += anchor_batch<false>(x, a, rs.rx, jb, e, colidx, ustart, u_colidx, dplus,
                               [&](int32_t w) { return rs.has(w); });
    }
    if (voff) {
      c = warp_sum(c);
      if (lane == 0 && c) atomicAdd(&counts[member_of(voff, ngraphs, x)], c);
    } else {
      mine += c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a; i += blockDim.x) rs.erase(u_colidx[ub + i]);
    __syncthreads();
  }
  if (!voff) {
    mine = block_sum(mine, red);
    if (threadIdx.x == 0 && mine) atomicAdd(&counts[0], mine);
  }
}

// ---- C<s(L)> kept (the unfused form of Alg. 6) --------------------------------------------------
//
// C(i,j) at an entry of L (rank i > rank j) counts the k with j < k < i adjacent to both, i.e. the
// k in U(j) whose own list U(k) holds i.  So the lowest vertex j of each triangle is the anchor:
// the entries of its row A(j,:) that rank above j go into a hash table keyed by rank, each slot
// holding the entry's position in the CSR and a counter; every list U(k) of such a k is probed
// against it, and a hit on key i counts one triangle (j, k, i) for C(i, j).  The anchor then writes
// its counts to the positions of its own entries (j, i) -- the U side; a second pass moves each
// value to the mirror entry (i, j) on the L side (found by binary search in the lower vertex's
// row j, short after the degree ordering) and clears the U entry it read.  Every anchor owns its table, so
// the counts are exact; their sum is t.  Anchors with d+ <= 256 run one per warp (a 512-slot
// table in shared memory), those up to KEPT_CTA_MAXD one per CTA (the table in shared memory),
// longer ones one per CTA with the table in global memory.

constexpr int KEPT_WSLOTS = 512;
constexpr int KEPT_WMAXD = KEPT_WSLOTS / 2;
constexpr int KEPT_CTA_MAXD = 4096;
constexpr int KEPT_THREADS = 256;
constexpr int KEPT_WIN_LOG = 13;  // warp anchors' window filter: the top 8192 ranks (1 KB of bits)
constexpr int KEPT_WWARPS = 4;                     // warps per CTA of the warp-anchor kernel
constexpr int KEPT_SLOTS_MAX = 2 * KEPT_CTA_MAXD;  // table slots of the largest shared-memory table
enum KeptSlot { KS_NW = 0, KS_NC = 1, KS_NH = 2, KS_QW = 3, KS_QC = 4, KS_QH = 5, KS_TOTAL = 6, KS_NSLOT = 8 };

// a counting table: keys (ranks), the CSR position of each key's entry, a counter.  The table may
// live in global memory, where its keys and counters change by atomics (performed at L2) while
// earlier plain loads may have left the lines in L1: every read is a volatile load, which does not
// use L1.
__device__ __forceinline__ int32_t vload(const int32_t *p) { return *(const volatile int32_t *)p; }
__device__ __forceinline__ uint32_t vload(const uint32_t *p) { return *(const volatile uint32_t *)p; }

struct KeptTable {
  int32_t *key, *pos;
  uint32_t *cnt;
  int logT;
  bool global;    // the table is in global memory (reads bypass L1)
  uint32_t *bm;   // in shared memory: one bit per rank of [w0, n) held by the table (a filter)
  int32_t w0;
  __device__ __forceinline__ int32_t rkey(int h) const { return global ? vload(&key[h]) : key[h]; }
  __device__ __forceinline__ void insert(int32_t r, int32_t p) const {
    if (r >= w0) atomicOr(&bm[(r - w0) >> 5], 1u << ((r - w0) & 31));
    const uint32_t mask = (1u << logT) - 1;
    uint32_t h = hslot(r, logT);
    // at least twice as many slots as keys: a free slot exists; the bound only ends the loop
    for (uint32_t i = 0; i <= mask; i++) {
      if (atomicCAS(&key[h], EMPTY, r) == EMPTY) {
        pos[h] = p;
        return;
      }
      h = (h + 1) & mask;
    }
  }
  // after the degree ordering most probes rank in the window, and most miss: one bitmap word
  // settles them before the table
  __device__ __forceinline__ void count(int32_t r) const {
    if (r >= w0 && !((bm[(r - w0) >> 5] >> ((r - w0) & 31)) & 1u)) return;
    const uint32_t mask = (1u << logT) - 1;
    uint32_t h = hslot(r, logT);
    for (uint32_t i = 0; i <= mask; i++) {
      const int32_t k = rkey((int)h);
      if (k == r) {
        atomicAdd(&cnt[h], 1u);
        return;
      }
      if (k == EMPTY) return;
      h = (h + 1) & mask;
    }
  }
};

// the anchors by class; the global tables of the longest ones get their slot counts in hsz
__global__ void tc_kept_classify(const int32_t *__restrict__ dplus, int32_t n, int32_t *__restrict__ lw,
                                 int32_t *__restrict__ lc, int32_t *__restrict__ lh, int32_t *__restrict__ hsz,
                                 int64_t *__restrict__ ks) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = dplus[v];
    if (a <= 0) continue;
    if (a <= KEPT_WMAXD) {
      lw[atomicAdd((unsigned long long *)&ks[KS_NW], 1ull)] = (int32_t)v;
    } else if (a <= KEPT_CTA_MAXD) {
      lc[atomicAdd((unsigned long long *)&ks[KS_NC], 1ull)] = (int32_t)v;
    } else {
      const unsigned long long p = atomicAdd((unsigned long long *)&ks[KS_NH], 1ull);
      lh[p] = (int32_t)v;
      hsz[p] = 1 << ceil_log2(2 * a);
    }
  }
}

// The load-balanced walk over 32 segments (warp_segments) with four elements per lane per round:
// the four positions are found first and their loads issued together, so that a lane keeps four
// list loads in flight.  f(gidx) is called for each valid element.  Warp-collective.
template <class F>
__device__ __forceinline__ void warp_segments4(int st, int len, F &&f) {
  const int lane = threadIdx.x & 31;
  const int incl = warp_inclusive_scan(len);
  const int total = __shfl_sync(LAGR_FULL_MASK, incl, 31);
  for (int base = 0; base < total; base += 128) {
    int g[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int k = base + 32 * j + lane;
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; step++) {
        const int mid = (lo + hi) >> 1;
        const int v = __shfl_sync(LAGR_FULL_MASK, incl, mid);
        if (v > k) hi = mid; else lo = mid + 1;
      }
      const int incl_s = __shfl_sync(LAGR_FULL_MASK, incl, lo);
      const int len_s = __shfl_sync(LAGR_FULL_MASK, len, lo);
      const int st_s = __shfl_sync(LAGR_FULL_MASK, st, lo);
      g[j] = k < total ? st_s + (k - (incl_s - len_s)) : -1;
    }
    int32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; j++) w[j] = g[j] >= 0 ? g[j] : 0;
    f(w, g);
  }
}

// One anchor v, processed by `ng` warps of a group (warp index gw within it) with the table t;
// sync() is the group's barrier.  Writes the anchor's counts to the positions of its U entries in
// c (cleared before the pass) and adds their sum into *total.
template <class Sync>
__device__ __forceinline__ void kept_anchor(int32_t v, const int32_t *__restrict__ rowptr,
                                            const int32_t *__restrict__ colidx, const int32_t *__restrict__ dplus,
                                            const int32_t *__restrict__ u_colidx, const int32_t *__restrict__ rank,
                                            const KeptTable &t, int gw, int ng, int gtid, int gsize, Sync &&sync,
                                            uint32_t *__restrict__ c, unsigned long long *__restrict__ total) {
  const int lane = threadIdx.x & 31;
  const int32_t rv = rank[v];
  const int32_t b = rowptr[v], e = rowptr[v + 1];
  const int T = 1 << t.logT;
  for (int i = gtid; i < T; i += gsize) {
    t.key[i] = EMPTY;
    t.cnt[i] = 0u;
  }
  sync();
  for (int32_t p = b + gtid; p < e; p += gsize) {
    const int32_t r = rank[colidx[p]];
    if (r > rv) t.insert(r, p);
  }
  sync();
  // the middle vertices k (entries of A(v,:) ranked above v), 32 row entries per warp batch: every
  // entry of U(k) is probed.  Lists of 32 or more are walked by the whole warp, shorter ones by the
  // load-balanced segment walk.
  const int32_t a = dplus[v];
  for (int32_t jb = b + gw * 32; jb < e; jb += ng * 32) {
    const int32_t j = jb + lane;
    int32_t st = 0, len = 0, rk = 0;
    if (j < e) {
      const int32_t k = colidx[j];
      rk = rank[k];
      if (rk > rv) {
        st = rowptr[k];
        len = dplus[k];
      }
    }
    unsigned longs = __ballot_sync(LAGR_FULL_MASK, len >= 32);
    warp_segments4(st, len >= 32 ? 0 : len, [&](int32_t (&pos)[4], const int (&g)[4]) {
      int32_t r[4];
#pragma unroll
      for (int q = 0; q < 4; q++) r[q] = u_colidx[pos[q]];  // four loads in flight
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (g[q] >= 0) t.count(r[q]);
    });
    while (longs) {
      const int sl = __ffs(longs) - 1;
      longs &= longs - 1;
      const int32_t st_s = __shfl_sync(LAGR_FULL_MASK, st, sl), len_s = __shfl_sync(LAGR_FULL_MASK, len, sl);
      const int32_t rk_s = __shfl_sync(LAGR_FULL_MASK, rk, sl);
      // A long U(k) sorted by descending rank is searched for the entries of U(v) instead of being
      // walked, when that takes fewer rounds: a hit is the same triangle (v, k, r)
      const int32_t search_rounds = ((a + 31) >> 5) * (32 - __clz(len_s));
      if (len_s >= TC_SORT_MIN && len_s <= TC_SORT_MAX && search_rounds < ((len_s + 31) >> 5)) {
        const int32_t *lst = u_colidx + st_s;
        for (int32_t q = lane; q < a; q += 32) {
          const int32_t r = u_colidx[b + q];
          if (r <= rk_s) continue;  // U(k) holds only ranks above k's
          int32_t lo = 0, hi = len_s;  // the first position holding a rank <= r
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (lst[mid] > r) lo = mid + 1; else hi = mid;
          }
          if (lo < len_s && lst[lo] == r) t.count(r);
        }
        continue;
      }
      // four groups per round trip, the last round's loads masked at the list's end (every entry is
      // probed, so no load is wasted and a list of 32 to 128 entries costs one round trip)
      for (int32_t q = lane; q < len_s; q += 128) {
        const int32_t w0 = u_colidx[st_s + q];
        const int32_t w1 = q + 32 < len_s ? u_colidx[st_s + q + 32] : -1;
        const int32_t w2 = q + 64 < len_s ? u_colidx[st_s + q + 64] : -1;
        const int32_t w3 = q + 96 < len_s ? u_colidx[st_s + q + 96] : -1;
        t.count(w0);
        if (w1 >= 0) t.count(w1);
        if (w2 >= 0) t.count(w2);
        if (w3 >= 0) t.count(w3);
      }
    }
  }
  sync();
  // the anchor's counts at the positions of its entries (v, i)
  unsigned long long mine = 0;
  for (int q = gtid; q < T; q += gsize) {
    if (t.rkey(q) == EMPTY) continue;
    const uint32_t cv = t.global ? vload(&t.cnt[q]) : t.cnt[q];
    if (cv == 0) continue;  // c is cleared before the pass
    c[t.global ? vload(&t.pos[q]) : t.pos[q]] = cv;
    mine += cv;
  }
  mine = warp_sum(mine);
  if (lane == 0 && mine) atomicAdd(total, mine);
  for (int32_t q = gtid; q < a; q += gsize) {  // leave the filter clear for the next anchor
    const int32_t r = u_colidx[b + q];
    if (r >= t.w0) t.bm[(r - t.w0) >> 5] = 0u;
  }
  sync();
}

// warp-class anchors: one per warp, table in shared memory
__global__ void __launch_bounds__(KEPT_WWARPS * 32)
    tc_kept_warp(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                 const int32_t *__restrict__ dplus, const int32_t *__restrict__ u_colidx,
                 const int32_t *__restrict__ rank, const int32_t *__restrict__ list, int64_t *__restrict__ ks,
                 uint32_t *__restrict__ c, int32_t w0w) {
  __shared__ int32_t skey[KEPT_WWARPS][KEPT_WSLOTS];
  __shared__ int32_t spos[KEPT_WWARPS][KEPT_WSLOTS];
  __shared__ uint32_t scnt[KEPT_WWARPS][KEPT_WSLOTS];
  __shared__ uint32_t sbm[KEPT_WWARPS][(1 << KEPT_WIN_LOG) / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = lane; i < (1 << KEPT_WIN_LOG) / 32; i += 32) sbm[warp][i] = 0u;
  __syncwarp();
  const int64_t nl = ks[KS_NW];
  for (;;) {
    long long it = 0;
    if (lane == 0) it = (long long)atomicAdd((unsigned long long *)&ks[KS_QW], 1ull);
    it = __shfl_sync(LAGR_FULL_MASK, it, 0);
    if (it >= nl) break;
    const int32_t v = list[it];
    const KeptTable t{skey[warp], spos[warp], scnt[warp], ceil_log2(2 * dplus[v]), false, sbm[warp], w0w};
    kept_anchor(v, rowptr, colidx, dplus, u_colidx, rank, t, 0, 1, lane, 32, [] { __syncwarp(); }, c,
                (unsigned long long *)&ks[KS_TOTAL]);
  }
}

// CTA-class anchors (table in dynamic shared memory) or, with gkey != NULL, the longest anchors
// (table at offset hoff[i] of the global arrays)
__global__ void __launch_bounds__(KEPT_THREADS)
    tc_kept_cta(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                const int32_t *__restrict__ dplus, const int32_t *__restrict__ u_colidx,
                const int32_t *__restrict__ rank, const int32_t *__restrict__ list, int64_t *__restrict__ ks,
                int slot_n, int slot_q, int32_t *__restrict__ gkey, int32_t *__restrict__ gpos,
                uint32_t *__restrict__ gcnt, const int32_t *__restrict__ hoff, uint32_t *__restrict__ c,
                int32_t w0c) {
  extern __shared__ int32_t ksm[];
  __shared__ long long s_it;
  // the window filter: after the shared-memory table, or alone when the tables are global
  uint32_t *bm = reinterpret_cast<uint32_t *>(gkey ? ksm : ksm + 3 * KEPT_SLOTS_MAX);
  for (int i = threadIdx.x; i < (1 << TCC_WIN_LOG) / 32; i += blockDim.x) bm[i] = 0u;
  __syncthreads();
  const int64_t nl = ks[slot_n];
  for (;;) {
    if (threadIdx.x == 0) s_it = (long long)atomicAdd((unsigned long long *)&ks[slot_q], 1ull);
    __syncthreads();
    const long long it = s_it;
    __syncthreads();
    if (it >= nl) break;
    const int32_t v = list[it];
    KeptTable t;
    t.logT = ceil_log2(2 * dplus[v]);
    t.global = gkey != nullptr;
    t.bm = bm;
    t.w0 = w0c;
    if (gkey) {
      t.key = gkey + hoff[it];
      t.pos = gpos + hoff[it];
      t.cnt = gcnt + hoff[it];
    } else {
      t.key = ksm;
      t.pos = ksm + KEPT_SLOTS_MAX;
      t.cnt = reinterpret_cast<uint32_t *>(ksm + 2 * KEPT_SLOTS_MAX);
    }
    kept_anchor(v, rowptr, colidx, dplus, u_colidx, rank, t, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x,
                blockDim.x, [] { __syncthreads(); }, c, (unsigned long long *)&ks[KS_TOTAL]);
  }
}

// The counts sit at the U side (v, i); move each to the mirror entry (i, v) of L and clear it.  One
// thread per entry of L: the mirror is in the row of the lower vertex.
__global__ void tc_kept_mirror(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                               const int32_t *__restrict__ rank, const int32_t *__restrict__ blk, int32_t nblk,
                               uint32_t *__restrict__ c) {
  // one CTA per row block of the plan; entries walked in order, rows found in staged pointers
  __shared__ int32_t rp[ROW_UNITS + 1];
  for (int32_t bb = blockIdx.x; bb < nblk; bb += gridDim.x) {
    const int32_t r0 = blk[bb], r1 = blk[bb + 1];
    const int32_t nr = r1 - r0;
    __syncthreads();
    for (int32_t q = threadIdx.x; q <= nr; q += blockDim.x) rp[q] = rowptr[r0 + q];
    __syncthreads();
    const int32_t e0 = rp[0], e1 = rp[nr];
    for (int32_t k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
      int32_t lo = 0, hi = nr - 1;  // the row of entry k
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= k) lo = mid; else hi = mid - 1;
      }
      const int32_t i = r0 + lo, j = colidx[k];
      if (rank[i] <= rank[j]) continue;  // a U-side entry: cleared by the thread of its mirror
      int32_t a = rowptr[j], z = rowptr[j + 1];  // (j, i) in row j
      while (a < z) {
        const int32_t mid = a + ((z - a) >> 1);
        if (colidx[mid] < i) a = mid + 1; else z = mid;
      }
      if (a < rowptr[j + 1] && colidx[a] == i) {
        // the U-side entry (j, i) is the mirror of this entry only, so this thread alone reads and
        // clears it; no thread reads an L-side entry
        const uint32_t v = c[a];
        c[k] = v;
        if (v) c[a] = 0u;
      }
    }
  }
}

}  // namespace

TcParams tc_default_params() { return TcParams{TCC_CHUNK, TCW_MAXD}; }

// capacities of the anchor lists forced by lagr_debug_tc_capacity (0: computed from the graph)
static std::atomic<int64_t> g_force_capc{0}, g_force_capwh{0};

// Allocate the orientation U (on G) and the anchor lists / orientation scratch (in the private
// state) for the given work partition.  No kernels.
int tc_alloc(lagr_graph G, Priv *P, TcParams prm, cudaStream_t s, char *msg) {
  const int32_t n = G->n;
  const int64_t nnz = G->nnz;
  if (prm.wmax < 1 || prm.wmax > TCW_MAXD || prm.chunk < 32 || prm.chunk > TCC_MAXCHUNK) {
    set_msg(msg, "bad triangle-count partition (wmax=%d, chunk=%d)", prm.wmax, prm.chunk);
    return LAGR_ERR_INVALID_VALUE;
  }
  // Capacity of the CTA item list: anchors outside the warp class have d+ > wmax (at most
  // m_L / (wmax + 1) = nnz / (2 (wmax + 1)) of them, as the d+ sum to m_L) or degree > TCW_MAXDEG
  // (at most nnz / (TCW_MAXDEG + 1)), and each has ceil(deg / chunk) <= deg / chunk + 1 items: at
  // most nnz / chunk + nnz / (2 (wmax + 1)) + nnz / (TCW_MAXDEG + 1) items in all on a symmetric
  // graph.  Writes past the capacity are skipped and flag SC_ERR; the count kernels read at most
  // the capacity (see tc_classify, tc_count_cta, tc_count_warp).
  const int64_t fc = g_force_capc.load(), fwh = g_force_capwh.load();
  const int64_t capc = fc > 0 ? fc : 2 * (nnz / (prm.wmax + 1) + nnz / (TCW_MAXDEG + 1)) + nnz / prm.chunk + 64;
  const int64_t capwh = fwh > 0 ? fwh : 2 * (nnz / TCW_CHUNK) + 64;
  if (G->u_colidx && P->tc_listw && P->tc_capc >= capc && P->tc_capwh >= capwh &&
      (fc == 0 || P->tc_capc == capc) && (fwh == 0 || P->tc_capwh == capwh))
    return LAGR_OK;
  dev_free(G->u_dplus, s);
  dev_free(G->u_colidx, s);
  G->u_dplus = G->u_colidx = nullptr;
  dev_free(P->tc_listw, s);
  dev_free(P->tc_listwh, s);
  dev_free(P->tc_listc, s);
  dev_free(P->tc_rank, s);
  dev_free(P->tc_sortbuf, s);
  dev_free(P->tc_radix, s);
  dev_free(P->tc_radix_scan, s);
  P->tc_radix_scan = nullptr;
  P->tc_listw = P->tc_rank = P->tc_sortbuf = P->tc_radix = nullptr;
  P->tc_listc = nullptr;
  P->tc_listwh = nullptr;
  P->tc_capc = 0;
  P->tc_capwh = 0;
  G->u_order = -1;
  LAGR_TRY(lagr_property_row_degree(G, s, msg));
  LAGR_TRY(lagr_property_AT(G, s, msg));  // undirected: A' aliases A, so the row plan is shared
  LAGR_TRY(row_plan(&P->pr_at, G->rowptr, n, s, msg));
  LAGR_TRY(alloc_n(&G->u_dplus, (size_t)n + 1, s, msg, "d+"));
  LAGR_TRY(alloc_n(&G->u_colidx, (size_t)(nnz > 0 ? nnz : 1), s, msg, "U column indices"));
  LAGR_TRY(alloc_n(&P->tc_listw, (size_t)n + 1, s, msg, "warp anchors"));
  // warp anchors cut into items: ceil(deg / TCW_CHUNK) <= 2 deg / TCW_CHUNK items each (deg > TCW_CHUNK),
  // capacity capwh above
  LAGR_TRY(alloc_n(&P->tc_listwh, (size_t)capwh, s, msg, "warp anchor items"));
  P->tc_capwh = capwh;
  LAGR_TRY(alloc_n(&P->tc_listc, (size_t)capc, s, msg, "CTA anchors"));
  LAGR_TRY(alloc_n(&P->tc_rank, 2 * ((size_t)n + 1), s, msg, "degree ranks and their order"));
  LAGR_TRY(alloc_n(&P->tc_sortbuf, 4 * (size_t)n + 4, s, msg, "rank sort buffers"));
  LAGR_TRY(alloc_n(&P->tc_radix, (size_t)radix_scratch_len(n), s, msg, "radix scratch"));
  LAGR_TRY(alloc_n(&P->tc_radix_scan, (size_t)scan_scratch_len(radix_scratch_len(n)), s, msg, "radix scan scratch"));
  P->tc_capc = capc;
  return LAGR_OK;
}

// Orientation, anchor classification and the two counting kernels: kernel launches and
// memsets only (capturable in a CUDA graph).  counts[] receives the total (or per-member totals
// when voff != NULL; counts is zeroed here).  The Alg. 6 sort decision is taken on the device.
int tc_launch(lagr_graph G, Priv *P, int method, TcParams prm, const int32_t *voff, int32_t ngraphs,
              unsigned long long *counts, bool orient, cudaStream_t s, char *msg, bool count) {
  const int32_t n = G->n;
  const int64_t nnz = G->nnz;
  LAGR_CUDA_TRY(cudaFuncSetAttribute(tc_sort_rows_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(TC_SORT_MAX * sizeof(int32_t))));
  LAGR_CUDA_TRY(cudaFuncSetAttribute(tc_count_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCC_SMEM));
  LAGR_CUDA_TRY(cudaFuncSetAttribute(tc_count_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCW_SMEM));
  if (orient) {
    LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal, 0, LAGR_NSCAL * sizeof(int64_t), s));
    if (method == LAGR_TC_AUTO) {
      const int64_t xstar = (nnz + 4 * (int64_t)n - 1) / (4 * (int64_t)n);
      tc_decide<<<grid_for(n, 256), 256, 0, s>>>(G->rowptr, n, xstar, P->dscal);
    }
    tc_set_mode<<<1, 1, 0, s>>>(n, method, P->dscal);
    // ranks: the stable ascending-degree order (the relabelling of Alg. 6), or the ids
    int32_t *keys = P->tc_sortbuf, *vals = keys + n, *tk = vals + n, *tv = tk + n;
    tc_rank_keys<<<grid_for(n, 256), 256, 0, s>>>(G->rowptr, n, keys, vals);
    LAGR_LAUNCH_CHECK();
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) bits++;
    LAGR_TRY(radix_sort_pairs(keys, vals, tk, tv, n, bits, s, msg, P->tc_radix, P->tc_radix_scan));
    tc_rank_scatter<<<grid_for(n, 256), 256, 0, s>>>(vals, n, P->dscal, P->tc_rank);
    const RowPlan &rp = P->pr_at;
    if (rp.nheavy > 0)
      tc_orient_heavy_zero<<<grid_for(rp.nheavy, 256), 256, 0, s>>>(rp.heavy, rp.nheavy, G->u_dplus);
    tc_orient_rows<<<rp.nblk, 256, 0, s>>>(G->rowptr, G->colidx, P->tc_rank, rp.blk, rp.hblk, G->u_dplus,
                                           G->u_colidx);
    if (rp.nhc > 0)
      tc_orient_heavy<<<std::min(rp.nhc, resident_ctas((const void *)tc_orient_heavy, OH_THREADS, 0)), OH_THREADS, 0,
                        s>>>(G->rowptr, G->colidx, P->tc_rank, G->u_dplus, G->u_colidx, rp.heavy, rp.hc_off,
                             rp.hc_row, rp.nhc, rp.hchunk);
    {  // the rows to sort are listed in the rank-sort buffers (4n ints, free again once the ranks
       // are made): n pairs for the short rows, then n shared by the CTA rows and the long ones
      int2 *lw = reinterpret_cast<int2 *>(P->tc_sortbuf), *lc = lw + n, *lm_end = lw + 2 * (int64_t)n;
      tc_sort_collect<<<grid_for(n, 256), 256, 0, s>>>(G->rowptr, G->u_dplus, n, lw, lc, lm_end, P->dscal);
      tc_sort_rows_warp<TC_SORT_SMALL><<<sort_wave_ctas<TC_SORT_SMALL>(), TCS_WARPS * 32, 0, s>>>(
          lw, 0, P->dscal, SL_NSW, G->u_colidx);
      tc_sort_rows_warp<TC_SORT_WARP><<<sort_wave_ctas<TC_SORT_WARP>(), TCS_WARPS * 32, 0, s>>>(
          lm_end, 1, P->dscal, SL_NSM, G->u_colidx);
      tc_sort_rows_cta<<<sm_count(), TCS_CTA_THREADS, TC_SORT_MAX * sizeof(int32_t), s>>>(lc, P->dscal, G->u_colidx);
    }
    tc_classify<<<grid_for(n, 256), 256, 0, s>>>(G->rowptr, G->u_dplus, n, P->tc_listw, P->tc_listwh,
                                                 P->tc_capwh, P->tc_listc, P->tc_capc, P->dscal, prm.wmax,
                                                 prm.chunk, P->tc_rank + n + 1);
    LAGR_LAUNCH_CHECK();
  } else {
    static_assert(SL_QC == SL_QW + 1 && SL_TOTAL == SL_QC + 1, "slot layout");
    LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal + SL_QW, 0, 3 * sizeof(int64_t), s));
    LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal + SL_QWL, 0, sizeof(int64_t), s));
  }
  if (!count) return LAGR_OK;  // the orientation alone (the kept-C form counts on its own)
  if (counts != (unsigned long long *)(P->dscal + SL_TOTAL))
    LAGR_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)ngraphs * sizeof(unsigned long long), s));
  // windows: the top ranks [n - window, n) (or all of them on small graphs)
  const int32_t w0c = n > (1 << TCC_WIN_LOG) ? n - (1 << TCC_WIN_LOG) : 0;
  const int32_t w0w = n > (1 << TCW_WIN_LOG) ? n - (1 << TCW_WIN_LOG) : 0;
  {
    KTimer kt(TK_TC_CTA, s);
    tc_count_cta<<<resident_ctas((const void *)tc_count_cta, TCC_THREADS, TCC_SMEM), TCC_THREADS, TCC_SMEM, s>>>(G->rowptr, G->colidx, G->rowptr, G->u_colidx, G->u_dplus,
                                                        P->tc_rank, P->tc_listc, P->dscal, w0c, voff, ngraphs, counts,
                                                        prm.chunk, P->tc_capc);
  }
  {
    KTimer kt(TK_TC_WARP, s);
    tc_count_warp<<<resident_ctas((const void *)tc_count_warp, TCW_WARPS * 32, TCW_SMEM), TCW_WARPS * 32, TCW_SMEM, s>>>(G->rowptr, G->colidx, G->rowptr, G->u_colidx,
                                                            G->u_dplus, P->tc_rank, P->tc_listw, n, P->tc_listwh,
                                                            P->tc_capwh, P->dscal, w0w,
                                                            voff, ngraphs, counts);
  }
  LAGR_LAUNCH_CHECK();
  return LAGR_OK;
}

unsigned long long *tc_total_slot(Priv *P) { return (unsigned long long *)(P->dscal + SL_TOTAL); }

}  // namespace lagr

using namespace lagr;

extern "C" int lagr_tc(uint64_t *ntriangles, lagr_graph G, int32_t method, void *stream, char *msg) {
  if (!ntriangles) {
    set_msg(msg, "ntriangles is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(check_graph_arg(G, msg));
  if (method != LAGR_TC_AUTO && method != LAGR_TC_SORT && method != LAGR_TC_NOSORT) {
    set_msg(msg, "unknown triangle-count method %d", method);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (G->kind != LAGR_UNDIRECTED) {
    set_msg(msg, "triangle counting needs an undirected graph");
    return LAGR_ERR_INVALID_GRAPH;
  }
  *ntriangles = 0;
  if (G->n == 0 || G->nnz == 0) {
    clear_msg(msg);
    return LAGR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  const TcParams prm = tc_default_params();
  LAGR_TRY(tc_alloc(G, P, prm, s, msg));  // (re)allocating resets u_order: the orientation is rebuilt
  const bool cached = G->u_colidx && G->u_order == method && P->tc_listw;
  LAGR_TRY(tc_launch(G, P, method, prm, nullptr, 1, tc_total_slot(P), !cached, s, msg));
  G->u_order = method;
  LAGR_TRY(fetch_to_host(P->hscal, P->dscal, LAGR_NSCAL * sizeof(int64_t), s, msg));
  if (P->hscal[SC_ERR] != 0) {
    set_msg(msg, "an anchor list overflowed its capacity (an undirected graph that is not symmetric, or "
                 "capacities forced by lagr_debug_tc_capacity); the count is incomplete");
    return LAGR_ERR_INVALID_GRAPH;
  }
  *ntriangles = (uint64_t)P->hscal[SL_TOTAL];
  clear_msg(msg);
  return LAGR_OK;
}

extern "C" int lagr_debug_tc_capacity(int64_t capc, int64_t capwh) {
  if (capc < 0 || capwh < 0) return LAGR_ERR_INVALID_VALUE;
  g_force_capc.store(capc);
  g_force_capwh.store(capwh);
  return LAGR_OK;
}

extern "C" int lagr_tc_edges(uint32_t *c, uint64_t *ntriangles, lagr_graph G, int32_t method, void *stream,
                             char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  if (!c && G->nnz > 0) {
    set_msg(msg, "c is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  if (method != LAGR_TC_AUTO && method != LAGR_TC_SORT && method != LAGR_TC_NOSORT) {
    set_msg(msg, "unknown triangle-count method %d", method);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (G->kind != LAGR_UNDIRECTED) {
    set_msg(msg, "triangle counting needs an undirected graph");
    return LAGR_ERR_INVALID_GRAPH;
  }
  if (ntriangles) *ntriangles = 0;
  const int32_t n = G->n;
  const int64_t nnz = G->nnz;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nnz == 0) {
    clear_msg(msg);
    return LAGR_OK;
  }
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  const TcParams prm = tc_default_params();
  LAGR_TRY(tc_alloc(G, P, prm, s, msg));
  const bool cached = G->u_colidx && G->u_order == method && P->tc_listw;
  if (!cached) {
    LAGR_TRY(tc_launch(G, P, method, prm, nullptr, 1, tc_total_slot(P), true, s, msg, false));
    G->u_order = method;
  }
  const RowPlan &rp = P->pr_at;  // built by tc_alloc
  Temp<int32_t> lw(s), lc(s), lh(s), hsz(s), hoff(s);
  Temp<int64_t> ks(s);
  LAGR_TRY(lw.alloc(n, msg, "warp anchors"));
  LAGR_TRY(lc.alloc(n, msg, "CTA anchors"));
  LAGR_TRY(lh.alloc(n, msg, "long anchors"));
  LAGR_TRY(hsz.alloc(n, msg, "table sizes"));
  LAGR_TRY(hoff.alloc((size_t)n + 1, msg, "table offsets"));
  LAGR_TRY(ks.alloc(KS_NSLOT, msg, "counters"));
  LAGR_CUDA_TRY(cudaMemsetAsync(ks.p, 0, KS_NSLOT * sizeof(int64_t), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)nnz * sizeof(uint32_t), s));
  tc_kept_classify<<<grid_for(n, 256), 256, 0, s>>>(G->u_dplus, n, lw.p, lc.p, lh.p, hsz.p, ks.p);
  LAGR_LAUNCH_CHECK();
  int64_t h[KS_NSLOT];
  LAGR_TRY(fetch_to_host(h, ks.p, sizeof(h), s, msg));
  const int64_t nh = h[KS_NH];
  Temp<int32_t> gkey(s), gpos(s);
  Temp<uint32_t> gcnt(s);
  if (nh > 0) {  // global tables of the longest anchors: one after the other
    LAGR_TRY(exclusive_scan(hsz.p, hoff.p, nh, s, msg));
    int32_t tot = 0;
    const int32_t *src[1] = {hoff.p + nh};
    LAGR_TRY(fetch_i32s(&tot, src, 1, s, msg));
    LAGR_TRY(gkey.alloc(tot, msg, "anchor tables"));
    LAGR_TRY(gpos.alloc(tot, msg, "anchor positions"));
    LAGR_TRY(gcnt.alloc(tot, msg, "anchor counters"));
  }
  const size_t bmbytes = ((size_t)1 << TCC_WIN_LOG) / 8;
  const size_t csmem = (size_t)3 * KEPT_SLOTS_MAX * sizeof(int32_t) + bmbytes;
  const int32_t w0c = n > (1 << TCC_WIN_LOG) ? n - (1 << TCC_WIN_LOG) : 0;
  const int32_t w0w = n > (1 << KEPT_WIN_LOG) ? n - (1 << KEPT_WIN_LOG) : 0;
  LAGR_CUDA_TRY(cudaFuncSetAttribute(tc_kept_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
  if (h[KS_NW] > 0)
    tc_kept_warp<<<resident_ctas((const void *)tc_kept_warp, KEPT_WWARPS * 32, 0), KEPT_WWARPS * 32, 0, s>>>(
        G->rowptr, G->colidx, G->u_dplus, G->u_colidx, P->tc_rank, lw.p, ks.p, c, w0w);
  if (h[KS_NC] > 0)
    tc_kept_cta<<<resident_ctas((const void *)tc_kept_cta, KEPT_THREADS, csmem), KEPT_THREADS, csmem, s>>>(
        G->rowptr, G->colidx, G->u_dplus, G->u_colidx, P->tc_rank, lc.p, ks.p, KS_NC, KS_QC, nullptr, nullptr,
        nullptr, nullptr, c, w0c);
  if (nh > 0)
    tc_kept_cta<<<sm_count(), KEPT_THREADS, bmbytes, s>>>(G->rowptr, G->colidx, G->u_dplus, G->u_colidx,
                                                          P->tc_rank, lh.p, ks.p, KS_NH, KS_QH, gkey.p, gpos.p,
                                                          gcnt.p, hoff.p, c, w0c);
  const int mg = resident_ctas((const void *)tc_kept_mirror, 256, 0);
  tc_kept_mirror<<<mg, 256, 0, s>>>(G->rowptr, G->colidx, P->tc_rank, rp.blk, rp.nblk, c);
  LAGR_LAUNCH_CHECK();
  LAGR_TRY(fetch_to_host(h, ks.p, sizeof(h), s, msg));
  if (ntriangles) *ntriangles = (uint64_t)h[KS_TOTAL];
  clear_msg(msg);
  return LAGR_OK;
}
