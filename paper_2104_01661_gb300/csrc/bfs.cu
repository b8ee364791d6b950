// Parents BFS (Alg. 1 and Alg. 2, Sec. IV-A) and the 64-source bitmap BFS (the ns x n frontier
// of Alg. 3, Sec. IV-B, with ns <= 64).
//
// One level is q'<!s(p),r> = q' any.secondi A (push) or q<!s(p),r> = A' any.secondi q (pull),
// followed by p<s(q)> = q.  Here the two are fused: the kernel that discovers v writes parent[v]
// (the secondi value: the frontier vertex that reached v; `any` keeps whichever claims v first)
// and level[v] directly.  The complemented structural mask !s(p) is a visited bitmap; the
// frontier is a vertex queue for push and a bitmap for pull (the bitmap format of Sec. VI-A).
//
// Push expands 32 frontier vertices per warp with the load-balanced segment walk and claims
// unvisited vertices with atomicOr on the visited bitmap.  Pull gives each unvisited vertex one
// lane that scans its in-neighbours and stops at the first one in the frontier (any monoid).
// Narrow frontiers (the high-diameter regime of the paper's road graph) run many levels inside
// one single-CTA launch with only __syncthreads between levels.  The push/pull choice is
// Beamer's rule: pull when the frontier's edges exceed the unexplored edges / alpha, push again
// when the frontier shrinks below n / beta.  The host takes that choice between phases from
// counters the kernels store into mapped host memory; lagr_bfs_multi interleaves the phases of
// several independent traversals on side streams.
#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace lagr {
namespace {

constexpr int BFS_THREADS = 256;
constexpr int SMALL_THREADS = 1024;
constexpr int64_t SMALL_MAX = 8192;     // frontiers up to this many vertices ...
constexpr int64_t SMALL_EDGES = 16384;  // ... and this many out-edges stay in the single-CTA kernel
constexpr int ALPHA_DO = 14;
constexpr int BETA_DO = 24;

// counters of one BFS call (device int64, mirrored to pinned host memory)
enum BfsSlot {
  B_NQ = 0,      // size of the current frontier
  B_LEV = 1,     // last completed level
  B_PAR = 2,     // which queue buffer holds the frontier (0: qa, 1: qb)
  B_MU = 3,      // unexplored edges
  B_MF = 4,      // edges out of the current frontier
  B_NEXT = 5,    // next-frontier size being built
  B_MNEXT = 6,   // edges out of the next frontier being built
  B_EXIT = 7,    // why the single-CTA kernel returned
  B_NSLOT = 8
};

// the counters, also stored into the caller's pinned host mirror (device-mapped), so that the host
// reads them after a stream synchronisation without a copy
__device__ __forceinline__ void mirror_counters(const int64_t *c, int64_t *hm) {
  for (int i = 0; i < B_NSLOT; i++) hm[i] = c[i];
}

__global__ void bfs_init(int32_t n, int32_t *__restrict__ level, int32_t *__restrict__ parent,
                         uint32_t *__restrict__ visited, int64_t nwords) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (level) level[i] = -1;
    if (parent) parent[i] = -1;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += stride) visited[i] = 0;
}

__global__ void bfs_seed(const int32_t *__restrict__ rowptr, int64_t nnz, int32_t src, int32_t *__restrict__ level,
                         int32_t *__restrict__ parent, uint32_t *__restrict__ visited, int32_t *__restrict__ qa,
                         int64_t *__restrict__ c, int64_t *hm) {
  if (level) level[src] = 0;
  if (parent) parent[src] = src;
  visited[src >> 5] |= 1u << (src & 31);
  qa[0] = src;
  const int64_t d = rowptr[src + 1] - rowptr[src];
  for (int i = 0; i < B_NSLOT; i++) c[i] = 0;
  c[B_NQ] = 1;
  c[B_MF] = d;
  c[B_MU] = nnz - d;
  if (hm) mirror_counters(c, hm);
}

// Claim v for the frontier vertex u at level lev.  Returns true when this thread won v.
__device__ __forceinline__ bool claim(uint32_t *__restrict__ visited, int32_t v) {
  const uint32_t bit = 1u << (v & 31);
  if (visited[v >> 5] & bit) return false;
  return !(atomicOr(&visited[v >> 5], bit) & bit);
}

// One push level of the single-CTA kernel.  Frontier vertices with at most NARROW_DEG edges are
// taken one per thread, whose column and visited loads are all in flight together (a narrow level
// is a chain of dependent loads, so their latency, not bandwidth, is its cost); longer rows are
// listed in big[] and walked afterwards by the warps, 32 edges at a time.  Appends to qout through
// *qcount; adds the out-degree of every discovered vertex to mdeg.
constexpr int NARROW_DEG = 8;
__device__ __forceinline__ void push_level_narrow(const int32_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ colidx, const int32_t *__restrict__ qin,
                                                  int64_t nq, int32_t *__restrict__ qout,
                                                  uint32_t *__restrict__ visited, int32_t *__restrict__ level,
                                                  int32_t *__restrict__ parent, int32_t lev,
                                                  unsigned long long *qcount, unsigned long long &mdeg, int32_t *big,
                                                  int *nbig) {
  for (int64_t i = threadIdx.x; i < nq; i += blockDim.x) {
    const int32_t u = qin[i];
    const int32_t st = rowptr[u];
    int32_t len = rowptr[u + 1] - st;
    if (len > NARROW_DEG) {
      big[atomicAdd(nbig, 1)] = u;
      len = 0;
    }
    int32_t v[NARROW_DEG];
#pragma unroll
    for (int j = 0; j < NARROW_DEG; j++) v[j] = j < len ? colidx[st + j] : -1;
    uint32_t fresh = 0;  // bit j: candidate v[j] exists and is not yet visited
#pragma unroll
    for (int j = 0; j < NARROW_DEG; j++)
      if (v[j] >= 0 && !((visited[v[j] >> 5] >> (v[j] & 31)) & 1u)) fresh |= 1u << j;
    while (fresh) {
      const int j = __ffs(fresh) - 1;
      fresh &= fresh - 1;
      int32_t w = v[0];
#pragma unroll
      for (int q = 1; q < NARROW_DEG; q++)
        if (q == j) w = v[q];
      const int32_t dw = rowptr[w + 1] - rowptr[w];  // issued with the claim below
      if (!(atomicOr(&visited[w >> 5], 1u << (w & 31)) & (1u << (w & 31)))) {
        qout[atomicAdd(qcount, 1ull)] = w;
        if (level) level[w] = lev;
        if (parent) parent[w] = u;
        mdeg += (unsigned long long)dw;
      }
    }
  }
  __syncthreads();
  // the longer rows: warps take 32 of them at a time and spread their edges over the lanes
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int nb = *nbig;
  for (int wb = (threadIdx.x >> 5) * 32; wb < nb; wb += (int)(blockDim.x >> 5) * 32) {
    int32_t u = -1, st = 0, len = 0;
    if (wb + lane < nb) {
      u = big[wb + lane];
      st = rowptr[u];
      len = rowptr[u + 1] - st;
    }
    warp_segments(st, len, u, [&](bool valid, int uu, int, int gidx) {
      bool won = false;
      int32_t w = 0;
      int32_t dw = 0;
      if (valid) {
        w = colidx[gidx];
        won = claim(visited, w);
        if (won) dw = rowptr[w + 1] - rowptr[w];
      }
      const unsigned m = __ballot_sync(LAGR_FULL_MASK, won);
      if (m) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(qcount, (unsigned long long)__popc(m));
        pos = __shfl_sync(LAGR_FULL_MASK, pos, 0);
        if (won) {
          qout[pos + __popc(m & lt)] = w;
          if (level) level[w] = lev;
          if (parent) parent[w] = uu;
          mdeg += (unsigned long long)dw;
        }
      }
    });
  }
}

// One wide push level.  The next frontier is not appended to a queue (one shared counter would
// serialise the whole grid); a vertex claimed here gets its bit in nbits (cleared by the caller),
// and the counts are reduced per warp once, at the end.  The frontier is read from the queue that
// c[B_PAR] selects.
__global__ void __launch_bounds__(BFS_THREADS)
    bfs_push(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const int32_t *__restrict__ qa,
             const int32_t *__restrict__ qb, uint32_t *__restrict__ visited, uint32_t *__restrict__ nbits,
             int32_t *__restrict__ level, int32_t *__restrict__ parent, int64_t *__restrict__ c) {
  const int64_t nq = c[B_NQ];
  const int32_t lev = (int32_t)c[B_LEV] + 1;
  const int32_t *qin = c[B_PAR] ? qb : qa;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long found = 0, mdeg = 0;
  for (int64_t wb = warp0 * 32; wb < nq; wb += nwarps * 32) {
    const int64_t i = wb + lane;
    int32_t u = -1, st = 0, len = 0;
    if (i < nq) {
      u = qin[i];
      st = rowptr[u];
      len = rowptr[u + 1] - st;
    }
    warp_segments(st, len, u, [&](bool valid, int uu, int, int gidx) {
      if (!valid) return;
      const int32_t v = colidx[gidx];
      if (claim(visited, v)) {
        atomicOr(&nbits[v >> 5], 1u << (v & 31));
        if (level) level[v] = lev;
        if (parent) parent[v] = uu;
        found++;
        mdeg += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
      }
    });
  }
  found = warp_sum(found);
  mdeg = warp_sum(mdeg);
  if (lane == 0) {
    if (found) atomicAdd((unsigned long long *)&c[B_NEXT], found);
    if (mdeg) atomicAdd((unsigned long long *)&c[B_MNEXT], mdeg);
  }
}

// Degrees of the frontier vertices (the input of the edge-balanced push's scan).
__global__ void bfs_frontier_degrees(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ qa,
                                     const int32_t *__restrict__ qb, const int64_t *__restrict__ c,
                                     int32_t *__restrict__ fdeg) {
  const int64_t nq = c[B_NQ];
  const int32_t *q = c[B_PAR] ? qb : qa;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = q[i];
    fdeg[i] = rowptr[u + 1] - rowptr[u];
  }
}

constexpr int LB_CHUNK = 2048;  // frontier edges per CTA in the edge-balanced push

// Edge-balanced wide push: CTA b expands the frontier edges [b*LB_CHUNK, (b+1)*LB_CHUNK) of the
// concatenated adjacency lists, whatever vertices they belong to, so one hub's list is shared by
// many CTAs instead of being walked by one warp.  offs = exclusive prefix of the frontier degrees
// (offs[nq] = total edges).  The frontier vertices that the chunk touches are staged in shared
// memory and each edge finds its vertex by a binary search there.  Claimed vertices get their bit
// in nbits (cleared by the caller); counts are reduced once per warp.
__global__ void __launch_bounds__(256)
    bfs_push_lb(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const int32_t *__restrict__ qa,
                const int32_t *__restrict__ qb, const int32_t *__restrict__ offs, uint32_t *__restrict__ visited,
                uint32_t *__restrict__ nbits, int32_t *__restrict__ level, int32_t *__restrict__ parent,
                int64_t *__restrict__ c) {
  __shared__ int32_t s_off[LB_CHUNK + 1];
  __shared__ int32_t s_u[LB_CHUNK + 1];
  __shared__ int32_t s_rs[LB_CHUNK + 1];
  __shared__ int32_t s_i0, s_cnt;
  const int64_t nq = c[B_NQ];
  const int32_t lev = (int32_t)c[B_LEV] + 1;
  const int32_t *q = c[B_PAR] ? qb : qa;
  const int32_t total = offs[nq];
  const int32_t c0 = blockIdx.x * LB_CHUNK;
  if (c0 >= total) return;  // uniform per CTA
  const int32_t c1 = min(c0 + LB_CHUNK, total);
  if (threadIdx.x == 0) {
    // first vertex: the last i with offs[i] <= c0; last vertex: the last i with offs[i] <= c1 - 1
    int32_t lo = 0, hi = (int32_t)nq - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= c0) lo = mid; else hi = mid - 1;
    }
    const int32_t i0 = lo;
    hi = (int32_t)nq - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= c1 - 1) lo = mid; else hi = mid - 1;
    }
    s_i0 = i0;
    s_cnt = lo - i0 + 1;
  }
  __syncthreads();
  const int32_t i0 = s_i0, cnt = s_cnt;
  const bool staged = cnt <= LB_CHUNK;  // vertices of degree 0 could make the range wider
  if (staged) {
    for (int32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int32_t u = q[i0 + t];
      s_off[t] = offs[i0 + t];
      s_u[t] = u;
      s_rs[t] = rowptr[u];
    }
  }
  __syncthreads();
  unsigned long long found = 0, mdeg = 0;
  for (int32_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
    int32_t lo = 0, hi = cnt - 1;  // last t with offs[i0 + t] <= e
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if ((staged ? s_off[mid] : offs[i0 + mid]) <= e) lo = mid; else hi = mid - 1;
    }
    int32_t u, rs, o;
    if (staged) {
      u = s_u[lo];
      rs = s_rs[lo];
      o = s_off[lo];
    } else {
      u = q[i0 + lo];
      rs = rowptr[u];
      o = offs[i0 + lo];
    }
    const int32_t v = colidx[rs + (e - o)];
    if (claim(visited, v)) {
      atomicOr(&nbits[v >> 5], 1u << (v & 31));
      if (level) level[v] = lev;
      if (parent) parent[v] = u;
      found++;
      mdeg += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
    }
  }
  found = warp_sum(found);
  mdeg = warp_sum(mdeg);
  if ((threadIdx.x & 31) == 0) {
    if (found) atomicAdd((unsigned long long *)&c[B_NEXT], found);
    if (mdeg) atomicAdd((unsigned long long *)&c[B_MNEXT], mdeg);
  }
}

// Many narrow push levels in one CTA.  Returns when the frontier is empty, grows past nmax (at most
// SMALL_MAX) vertices or SMALL_EDGES out-edges, the direction rule asks for a pull, or max_level is
// reached.
__global__ void __launch_bounds__(SMALL_THREADS, 1)
    bfs_push_small(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t *__restrict__ qa,
                   int32_t *__restrict__ qb, uint32_t *__restrict__ visited, int32_t *__restrict__ level,
                   int32_t *__restrict__ parent, int64_t *__restrict__ c, int32_t max_level, int allow_pull,
                   int64_t *hm, int64_t nmax = SMALL_MAX) {
  __shared__ unsigned long long s_next, s_mdeg;
  __shared__ int32_t s_big[SMALL_MAX];  // frontier vertices with long rows (the caller keeps nq <= SMALL_MAX)
  __shared__ int s_nbig;
  int64_t nq = c[B_NQ], mu = c[B_MU], mf = c[B_MF];
  int32_t lev = (int32_t)c[B_LEV];
  int par = (int)c[B_PAR];
  int exit_reason = 0;
  bool first = true, growing = false;
  for (;;) {
    if (nq == 0) { exit_reason = 1; break; }
    // the caller hands over only narrow frontiers; a level that widens goes back to the grid
    if (!first && (nq > nmax || mf > SMALL_EDGES)) { exit_reason = 2; break; }
    // the caller chose push for the first level; afterwards pull when a growing frontier's
    // edges outweigh the unexplored edges / alpha
    if (!first && allow_pull && growing && mf > mu / ALPHA_DO) { exit_reason = 3; break; }
    if (lev + 1 > max_level) { exit_reason = 4; break; }
    const int64_t nq_before = nq;
    if (threadIdx.x == 0) {
      s_next = 0;
      s_mdeg = 0;
      s_nbig = 0;
    }
    __syncthreads();
    const int32_t *qin = par ? qb : qa;
    int32_t *qout = par ? qa : qb;
    unsigned long long mdeg = 0;
    push_level_narrow(rowptr, colidx, qin, nq, qout, visited, level, parent, lev + 1, &s_next, mdeg, s_big, &s_nbig);
    mdeg = warp_sum(mdeg);
    if ((threadIdx.x & 31) == 0 && mdeg) atomicAdd(&s_mdeg, mdeg);
    __syncthreads();
    nq = (int64_t)s_next;
    mf = (int64_t)s_mdeg;
    mu -= mf;
    lev += 1;
    par ^= 1;
    growing = nq > nq_before;
    first = false;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c[B_NQ] = nq;
    c[B_LEV] = lev;
    c[B_PAR] = par;
    c[B_MU] = mu;
    c[B_MF] = mf;
    c[B_EXIT] = exit_reason;
    if (hm) mirror_counters(c, hm);
  }
}

// ---- narrow levels on the whole GPU: a cooperative launch with a grid barrier per level --------
//
// The single-CTA kernel above keeps narrow levels cheap but runs each level's chain of dependent
// loads on 1024 threads: on a high-diameter graph (the paper's road graph; the 4096 x 4096 grid
// here, frontiers of up to 4096 vertices over 8191 levels) a level costs the latency of several
// such chains.  bfs_push_coop spreads each level over every CTA of a cooperative launch (all CTAs
// resident at once, so they can wait for each other) and separates the levels with a grid barrier.
// The barrier's wait is bounded: when it runs out the kernel records LAGR_ERR_TIMEOUT and every
// CTA leaves.  The frontier is appended to a queue with one counter per level; three counters in
// rotation let a level reset the counter of the level after next without a second barrier.  The
// exit rule is that of the single-CTA kernel, with wider limits.

constexpr int COOP_THREADS = 256;
constexpr int64_t COOP_MIN = 2048;          // frontiers from this many vertices (hysteresis: down
                                            // to half of it) use the cooperative kernel, below it
                                            // the single-CTA one (a grid barrier costs more than a
                                            // level of a few vertices per thread)
constexpr int64_t COOP_MAX = 1 << 15;       // frontiers up to this many vertices ...
constexpr int64_t COOP_EDGES = 1 << 15;     // ... and out-edges stay in the cooperative kernel (a
                                            // row longer than 8 is one warp's, so this bounds it)
constexpr int COOP_BIG = 512;               // long rows a CTA lists per level (more: walked inline)
constexpr long long COOP_SPIN = 1ll << 24;  // barrier polls before giving up (seconds)

struct CoopState {
  unsigned long long qcount[3], mdeg[3];  // next-frontier size and out-degree sum, per level mod 3
  unsigned int arrive;                    // grid barrier arrivals (monotone)
  int err;                                // LAGR_ERR_TIMEOUT when a barrier wait ran out
};

// returns false when the wait ran out (then st->err is set and every CTA will leave)
__device__ __forceinline__ bool coop_barrier(CoopState *st, unsigned int target) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&st->arrive, 1u);
    int ok = 1;
    long long it = 0;
    while (*(volatile unsigned int *)&st->arrive < target) {
      if (*(volatile int *)&st->err || ++it > COOP_SPIN) {
        ok = 0;
        atomicExch(&st->err, LAGR_ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(COOP_THREADS, 2)
    bfs_push_coop(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t *__restrict__ qa,
                  int32_t *__restrict__ qb, uint32_t *__restrict__ visited, int32_t *__restrict__ level,
                  int32_t *__restrict__ parent, int64_t *__restrict__ c, CoopState *__restrict__ st,
                  int32_t max_level, int allow_pull, int64_t *hm) {
  __shared__ int32_t s_big[COOP_BIG];
  __shared__ int s_nbig;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  int64_t nq = c[B_NQ], mu = c[B_MU], mf = c[B_MF];
  int32_t lev = (int32_t)c[B_LEV];
  int par = (int)c[B_PAR];
  int exit_reason = 0;
  bool first = true, growing = false;
  unsigned int bar = 0;
  for (int it = 0;; it++) {
    if (nq == 0) { exit_reason = 1; break; }
    if (!first && (nq > COOP_MAX || mf > COOP_EDGES)) { exit_reason = 2; break; }
    if (!first && nq < COOP_MIN / 2) { exit_reason = 6; break; }  // narrow again: one CTA does better
    if (!first && allow_pull && growing && mf > mu / ALPHA_DO) { exit_reason = 3; break; }
    if (lev + 1 > max_level) { exit_reason = 4; break; }
    const int nxt = (it + 1) % 3;
    if (gtid == 0) {  // counters of the level after next: last read a level ago
      st->qcount[(it + 2) % 3] = 0;
      st->mdeg[(it + 2) % 3] = 0;
    }
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const int32_t *qin = par ? qb : qa;
    int32_t *qout = par ? qa : qb;
    unsigned long long *qcount = &st->qcount[nxt];
    unsigned long long mdeg = 0;
    const int32_t nlev = lev + 1;
    for (int64_t i = gtid; i < nq; i += gthreads) {
      const int32_t u = qin[i];
      const int32_t rs = rowptr[u];
      int32_t len = rowptr[u + 1] - rs;
      if (len > NARROW_DEG) {
        const int b = atomicAdd(&s_nbig, 1);
        if (b < COOP_BIG) {
          s_big[b] = u;
          len = 0;
        }
      }
      // short rows (and long ones past the CTA's list): this thread claims the neighbours itself
      for (int32_t k = 0; k < len; k++) {
        const int32_t w = colidx[rs + k];
        if (claim(visited, w)) {
          qout[atomicAdd(qcount, 1ull)] = w;
          if (level) level[w] = nlev;
          if (parent) parent[w] = u;
          mdeg += (unsigned long long)(rowptr[w + 1] - rowptr[w]);
        }
      }
    }
    __syncthreads();
    // the CTA's long rows: its warps take 32 at a time, edges spread over the lanes
    const int nb = min(s_nbig, COOP_BIG);
    for (int wb = (threadIdx.x >> 5) * 32; wb < nb; wb += (int)(blockDim.x >> 5) * 32) {
      int32_t u = -1, rs = 0, len = 0;
      if (wb + lane < nb) {
        u = s_big[wb + lane];
        rs = rowptr[u];
        len = rowptr[u + 1] - rs;
      }
      warp_segments(rs, len, u, [&](bool valid, int uu, int, int gidx) {
        bool won = false;
        int32_t w = 0, dw = 0;
        if (valid) {
          w = colidx[gidx];
          won = claim(visited, w);
          if (won) dw = rowptr[w + 1] - rowptr[w];
        }
        const unsigned m = __ballot_sync(LAGR_FULL_MASK, won);
        if (m) {
          unsigned long long pos = 0;
          if (lane == 0) pos = atomicAdd(qcount, (unsigned long long)__popc(m));
          pos = __shfl_sync(LAGR_FULL_MASK, pos, 0);
          if (won) {
            qout[pos + __popc(m & lt)] = w;
            if (level) level[w] = nlev;
            if (parent) parent[w] = uu;
            mdeg += (unsigned long long)dw;
          }
        }
      });
    }
    mdeg = warp_sum(mdeg);
    if (lane == 0 && mdeg) atomicAdd(&st->mdeg[nxt], mdeg);
    bar += gridDim.x;
    if (!coop_barrier(st, bar)) { exit_reason = 5; break; }
    const int64_t nq_before = nq;
    nq = (int64_t)*(volatile unsigned long long *)&st->qcount[nxt];
    mf = (int64_t)*(volatile unsigned long long *)&st->mdeg[nxt];
    mu -= mf;
    lev = nlev;
    par ^= 1;
    growing = nq > nq_before;
    first = false;
  }
  if (gtid == 0) {
    c[B_NQ] = nq;
    c[B_LEV] = lev;
    c[B_PAR] = par;
    c[B_MU] = mu;
    c[B_MF] = mf;
    c[B_EXIT] = exit_reason;
    if (hm) mirror_counters(c, hm);
  }
}

// queue -> frontier bitmap (the bitmap is cleared first by the caller)
__global__ void bfs_q2b(const int32_t *__restrict__ qa, const int32_t *__restrict__ qb, const int64_t *__restrict__ c,
                        uint32_t *__restrict__ fbits) {
  const int64_t nq = c[B_NQ];
  const int32_t *q = c[B_PAR] ? qb : qa;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = q[i];
    atomicOr(&fbits[v >> 5], 1u << (v & 31));
  }
}

// frontier bitmap -> queue qa (order of the words; B_PAR is reset to 0 by the host update)
__global__ void bfs_b2q(const uint32_t *__restrict__ fbits, int64_t nwords, int32_t *__restrict__ qa,
                        unsigned long long *__restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nwords; base += stride) {
    const int64_t w = base + lane;
    uint32_t word = (w < nwords) ? fbits[w] : 0u;
    const int cnt = __popc(word);
    const int incl = warp_inclusive_scan(cnt);
    const int tot = __shfl_sync(LAGR_FULL_MASK, incl, 31);
    unsigned long long p = 0;
    if (lane == 31 && tot) p = atomicAdd(count, (unsigned long long)tot);
    p = __shfl_sync(LAGR_FULL_MASK, p, 31);
    int64_t pos = (int64_t)p + incl - cnt;
    while (word) {
      const int b = __ffs(word) - 1;
      qa[pos++] = (int32_t)(w * 32 + b);
      word &= word - 1;
    }
  }
}

// One pull level: each unvisited vertex scans its in-neighbours (rows of A') for one in the
// frontier.  A warp owns one 32-vertex word of the bitmaps, so it updates them without atomics.
__global__ void __launch_bounds__(BFS_THREADS)
    bfs_pull(const int32_t *__restrict__ at_rowptr, const int32_t *__restrict__ at_colidx,
             const int32_t *__restrict__ rowptr, int32_t n, const uint32_t *__restrict__ fbits,
             uint32_t *__restrict__ nbits, uint32_t *__restrict__ visited, int32_t *__restrict__ level,
             int32_t *__restrict__ parent, int64_t *__restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int32_t lev = (int32_t)c[B_LEV] + 1;
  const int64_t nwords = ((int64_t)n + 31) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long found_n = 0, mdeg = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords; w += warps) {
    const uint32_t vis = visited[w];
    const int64_t v = w * 32 + lane;
    const bool need = v < n && !((vis >> lane) & 1u);
    if (!__any_sync(LAGR_FULL_MASK, need)) {
      if (lane == 0) nbits[w] = 0;
      continue;
    }
    int32_t par = -1, dv = 0;
    if (need) {
      const int32_t b = at_rowptr[v], e = at_rowptr[v + 1];
      dv = e - b;
      // four in-neighbours per round, so that their column and frontier loads overlap
      int32_t k = b;
      for (; k + 3 < e && par < 0; k += 4) {
        const int32_t u0 = at_colidx[k], u1 = at_colidx[k + 1], u2 = at_colidx[k + 2], u3 = at_colidx[k + 3];
        const bool h0 = (fbits[u0 >> 5] >> (u0 & 31)) & 1u, h1 = (fbits[u1 >> 5] >> (u1 & 31)) & 1u;
        const bool h2 = (fbits[u2 >> 5] >> (u2 & 31)) & 1u, h3 = (fbits[u3 >> 5] >> (u3 & 31)) & 1u;
        par = h0 ? u0 : h1 ? u1 : h2 ? u2 : h3 ? u3 : -1;
      }
      for (; k < e && par < 0; k++) {
        const int32_t u = at_colidx[k];
        if ((fbits[u >> 5] >> (u & 31)) & 1u) par = u;
      }
    }
    const unsigned m = __ballot_sync(LAGR_FULL_MASK, par >= 0);
    if (lane == 0) {
      nbits[w] = m;
      if (m) visited[w] = vis | m;
      found_n += __popc(m);
    }
    if (par >= 0) {
      if (level) level[v] = lev;
      if (parent) parent[v] = par;
      // the out-degree (the in-degree read above when A' is A)
      mdeg += (unsigned long long)(at_rowptr == rowptr ? dv : rowptr[v + 1] - rowptr[v]);
    }
  }
  found_n = warp_sum(found_n);
  mdeg = warp_sum(mdeg);
  if (lane == 0) {
    if (found_n) atomicAdd((unsigned long long *)&c[B_NEXT], found_n);
    if (mdeg) atomicAdd((unsigned long long *)&c[B_MNEXT], mdeg);
  }
}

// after a level: the next frontier becomes the current one
__global__ void bfs_advance(int64_t *__restrict__ c, int flip, int64_t *hm) {
  c[B_NQ] = c[B_NEXT];
  c[B_MF] = c[B_MNEXT];
  c[B_MU] -= c[B_MNEXT];
  c[B_LEV] += 1;
  if (flip) c[B_PAR] ^= 1;
  c[B_NEXT] = 0;
  c[B_MNEXT] = 0;
  if (hm) mirror_counters(c, hm);
}

__global__ void bfs_set_par(int64_t *__restrict__ c, int par) { c[B_PAR] = par; }

// ---- 64 sources at once -------------------------------------------------------------------------
//
// Bit s of the 64-bit words front[v] / seen[v] belongs to source s.  A level is either a push over
// the frontier's edges (edge-balanced as above; next bits are OR-ed into acc[v] with a 64-bit
// atomic, and the touched vertices are finalised afterwards) or a pull over all vertices that some
// source has not reached yet (coalesced row blocks; a row's scan stops once every source bit it
// still lacks has been seen among its neighbours).  Either way the level writes level[s][v] for
// every new bit and the list of vertices of the next frontier.

enum Bfs64Slot { S64_NF = 0, S64_MF = 1, S64_NT = 2, S64_NSLOT = 4 };

__global__ void bfs64_init(int32_t n, int32_t k, int32_t *__restrict__ level, unsigned long long *__restrict__ seen,
                           unsigned long long *__restrict__ fa, unsigned long long *__restrict__ fb,
                           unsigned long long *__restrict__ acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    seen[i] = 0;
    fa[i] = 0;
    fb[i] = 0;
    acc[i] = 0;
  }
  const int64_t total = (int64_t)k * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) level[i] = -1;
}

struct Sources64 {
  int32_t v[64];
};

__global__ void bfs64_seed(int32_t n, int32_t k, const Sources64 src, const int32_t *__restrict__ rowptr,
                           int32_t *__restrict__ level, unsigned long long *__restrict__ seen,
                           unsigned long long *__restrict__ front, int32_t *__restrict__ flist,
                           int64_t *__restrict__ cnt) {
  if (threadIdx.x != 0) return;
  int64_t nf = 0, mf = 0;
  for (int s = 0; s < k; s++) {
    const int32_t v = src.v[s];
    if (front[v] == 0) {
      flist[nf++] = v;
      mf += rowptr[v + 1] - rowptr[v];
    }
    seen[v] |= 1ull << s;
    front[v] |= 1ull << s;
    level[(int64_t)s * n + v] = 0;
  }
  for (int i = 0; i < S64_NSLOT; i++) cnt[i] = 0;
  cnt[S64_NF] = nf;
  cnt[S64_MF] = mf;
}

__device__ __forceinline__ void write_levels(int32_t *__restrict__ level, int32_t n, int32_t v, unsigned long long bits,
                                             int32_t lev) {
  while (bits) {
    const int s = __ffsll((long long)bits) - 1;
    level[(int64_t)s * n + v] = lev;
    bits &= bits - 1;
  }
}

// append v to a list through a counter (warp-aggregated over the lanes that append)
__device__ __forceinline__ void list_append(int32_t *__restrict__ list, unsigned long long *counter, int32_t v) {
  const unsigned act = __activemask();
  const int leader = __ffs(act) - 1;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(act));
  base = __shfl_sync(act, base, leader);
  list[base + __popc(act & lanemask_lt())] = v;
}

__global__ void bfs64_fdeg(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ flist, int32_t nf,
                           int32_t *__restrict__ fdeg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x)
    fdeg[i] = rowptr[flist[i] + 1] - rowptr[flist[i]];
}

// push: the frontier's edges [b*LB_CHUNK, (b+1)*LB_CHUNK) per CTA; acc[v] |= front[u] & ~seen[v]
__global__ void __launch_bounds__(256)
    bfs64_push_lb(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                  const int32_t *__restrict__ flist, int32_t nf, const int32_t *__restrict__ offs,
                  const unsigned long long *__restrict__ front, const unsigned long long *__restrict__ seen,
                  unsigned long long *__restrict__ acc, int32_t *__restrict__ touched, int64_t *__restrict__ cnt) {
  __shared__ int32_t s_off[LB_CHUNK + 1];
  __shared__ int32_t s_u[LB_CHUNK + 1];
  __shared__ int32_t s_rs[LB_CHUNK + 1];
  __shared__ int32_t s_i0, s_cnt;
  const int32_t total = offs[nf];
  const int32_t c0 = blockIdx.x * LB_CHUNK;
  if (c0 >= total) return;
  const int32_t c1 = min(c0 + LB_CHUNK, total);
  if (threadIdx.x == 0) {
    int32_t lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= c0) lo = mid; else hi = mid - 1;
    }
    const int32_t i0 = lo;
    hi = nf - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= c1 - 1) lo = mid; else hi = mid - 1;
    }
    s_i0 = i0;
    s_cnt = lo - i0 + 1;
  }
  __syncthreads();
  const int32_t i0 = s_i0, cnt_v = s_cnt;
  const bool staged = cnt_v <= LB_CHUNK;
  if (staged) {
    for (int32_t t = threadIdx.x; t < cnt_v; t += blockDim.x) {
      const int32_t u = flist[i0 + t];
      s_off[t] = offs[i0 + t];
      s_u[t] = u;
      s_rs[t] = rowptr[u];
    }
  }
  __syncthreads();
  for (int32_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
    int32_t lo = 0, hi = cnt_v - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if ((staged ? s_off[mid] : offs[i0 + mid]) <= e) lo = mid; else hi = mid - 1;
    }
    const int32_t u = staged ? s_u[lo] : flist[i0 + lo];
    const int32_t rs = staged ? s_rs[lo] : rowptr[u];
    const int32_t o = staged ? s_off[lo] : offs[i0 + lo];
    const int32_t v = colidx[rs + (e - o)];
    const unsigned long long bits = front[u] & ~seen[v];
    if (bits) {
      const unsigned long long old = atomicOr(&acc[v], bits);
      if (old == 0) list_append(touched, (unsigned long long *)&cnt[S64_NT], v);
    }
  }
}

// after a push: the touched vertices take their new bits
__global__ void bfs64_finish_push(const int32_t *__restrict__ touched, const int64_t *__restrict__ cnt,
                                  const int32_t *__restrict__ rowptr, unsigned long long *__restrict__ acc,
                                  unsigned long long *__restrict__ seen, unsigned long long *__restrict__ fnext,
                                  int32_t *__restrict__ level, int32_t n, int32_t lev, int32_t *__restrict__ nflist,
                                  int64_t *__restrict__ out) {
  const int64_t nt = cnt[S64_NT];
  unsigned long long mdeg = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = touched[t];
    const unsigned long long a = acc[v];
    acc[v] = 0;
    const unsigned long long nw = a & ~seen[v];
    if (nw) {
      seen[v] |= nw;
      fnext[v] = nw;
      write_levels(level, n, v, nw, lev);
      list_append(nflist, (unsigned long long *)&out[S64_NF], v);
      mdeg += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
    }
  }
  mdeg = warp_sum(mdeg);
  if ((threadIdx.x & 31) == 0 && mdeg) atomicAdd((unsigned long long *)&out[S64_MF], mdeg);
}

// pull over the row blocks: each vertex still missing some source bit ORs its neighbours' frontier
// words, stopping once the bits it lacks are all covered.  Short rows: a thread each; longer rows:
// a warp each; rows longer than ROW_HEAVY: a trailing CTA each.
__global__ void __launch_bounds__(256)
    bfs64_pull_rows(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                    const int32_t *__restrict__ blk, int32_t nblk, const int32_t *__restrict__ heavy, int32_t nheavy,
                    unsigned long long kmask, const unsigned long long *__restrict__ front,
                    unsigned long long *__restrict__ seen, unsigned long long *__restrict__ fnext,
                    int32_t *__restrict__ level, int32_t n, int32_t lev, int32_t *__restrict__ nflist,
                    int64_t *__restrict__ out) {
  __shared__ int32_t longrows[ROW_UNITS / 33 + 2];
  __shared__ int n_long;
  __shared__ unsigned long long s_acc;
  __shared__ int s_done;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long mdeg = 0;
  auto settle = [&](int32_t v, unsigned long long sv, unsigned long long acc) {
    const unsigned long long nw = acc & ~sv;
    if (nw) {
      seen[v] = sv | nw;
      fnext[v] = nw;
      write_levels(level, n, v, nw, lev);
      list_append(nflist, (unsigned long long *)&out[S64_NF], v);
      mdeg += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
    }
  };
  if ((int32_t)blockIdx.x >= nblk) {
    for (int32_t h = blockIdx.x - nblk; h < nheavy; h += gridDim.x - nblk) {
      const int32_t v = heavy[h];
      const unsigned long long sv = seen[v];
      if (sv == kmask) continue;  // uniform: every thread reads the same word
      if (threadIdx.x == 0) {
        s_acc = 0;
        s_done = 0;
      }
      __syncthreads();
      const int32_t b = rowptr[v], e = rowptr[v + 1];
      for (int32_t base = b; base < e; base += blockDim.x) {
        const int32_t k2 = base + threadIdx.x;
        unsigned long long x = k2 < e ? __ldg(&front[colidx[k2]]) : 0ull;
        const unsigned lo = __reduce_or_sync(LAGR_FULL_MASK, (unsigned)x);
        const unsigned hi = __reduce_or_sync(LAGR_FULL_MASK, (unsigned)(x >> 32));
        if (lane == 0 && (lo | hi)) atomicOr(&s_acc, ((unsigned long long)hi << 32) | lo);
        __syncthreads();
        if (threadIdx.x == 0 && ((s_acc | sv) == kmask)) s_done = 1;
        __syncthreads();
        if (s_done) break;
      }
      if (threadIdx.x == 0) settle(v, sv, s_acc);
      __syncthreads();
    }
  } else {
    if (threadIdx.x == 0) n_long = 0;
    __syncthreads();
    const int32_t r0 = blk[blockIdx.x], r1 = blk[blockIdx.x + 1];
    for (int32_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
      const int32_t b = rowptr[v], e = rowptr[v + 1];
      if (e - b > 32) {
        if (e - b <= ROW_HEAVY) longrows[atomicAdd(&n_long, 1)] = v;
        continue;
      }
      const unsigned long long sv = seen[v];
      if (sv == kmask) continue;
      unsigned long long acc = 0;
      for (int32_t q = b; q < e; q++) {
        acc |= __ldg(&front[colidx[q]]);
        if ((acc | sv) == kmask) break;
      }
      settle(v, sv, acc);
    }
    __syncthreads();
    for (int q = warp; q < n_long; q += 8) {
      const int32_t v = longrows[q];
      const unsigned long long sv = seen[v];
      if (sv == kmask) continue;
      const int32_t b = rowptr[v], e = rowptr[v + 1];
      unsigned long long acc = 0;
      for (int32_t base = b; base < e; base += 32) {
        const int32_t k2 = base + lane;
        const unsigned long long x = k2 < e ? __ldg(&front[colidx[k2]]) : 0ull;
        const unsigned lo = __reduce_or_sync(LAGR_FULL_MASK, (unsigned)x);
        const unsigned hi = __reduce_or_sync(LAGR_FULL_MASK, (unsigned)(x >> 32));
        acc |= ((unsigned long long)hi << 32) | lo;
        if ((acc | sv) == kmask) break;
      }
      if (lane == 0) settle(v, sv, acc);
    }
  }
  mdeg = warp_sum(mdeg);
  if (lane == 0 && mdeg) atomicAdd((unsigned long long *)&out[S64_MF], mdeg);
}

// the old frontier's words go back to zero, so the buffer can hold the level after next
__global__ void bfs64_clear(const int32_t *__restrict__ flist, int32_t nf, unsigned long long *__restrict__ front) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x)
    front[flist[i]] = 0;
}

}  // namespace
}  // namespace lagr

using namespace lagr;

namespace lagr {
namespace {

// the device can launch cooperative kernels (queried once per device)
bool coop_supported() {
  static int cached[64];  // 0 unknown, 1 yes, 2 no
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) {
    cudaGetLastError();
    return false;
  }
  if (!cached[d]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, d) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    cached[d] = v ? 1 : 2;
  }
  return cached[d] == 1;
}

// One direction-optimising parents BFS (Alg. 1 / 2) as a host-side state machine on its own stream.
// launch() takes the counters of the last phase from the mapped host mirror h (the phase's last
// kernel stores them there), applies the direction rule and enqueues the next phase: several
// narrow push levels in one CTA, one wide push level, or one pull level.  After the stream has been
// synchronised, settle() does the phase's bookkeeping.  Several runs interleave their phases on
// several streams, so one synchronisation serves them all (lagr_bfs_multi).
struct BfsRun {
  lagr_graph G = nullptr;
  int32_t src = 0;
  int32_t *level = nullptr, *parent = nullptr;
  bool push_only = false, pull_only = false;
  cudaStream_t s = nullptr;
  int64_t *h = nullptr, *hd = nullptr;  // B_NSLOT counters: host view, device view
  Temp<uint32_t> visited, fbits, nbits;
  Temp<int32_t> qa, qb, fdeg, offs;
  Temp<int64_t> cnt;
  Temp<CoopState> cst;  // the cooperative kernel's counters and barrier (coop runs only)
  bool coop = false;    // narrow levels on the whole GPU (a run that has the GPU to itself)
  int rep = 0;  // frontier representation: 0 = queue (push), 1 = bitmap fbits (pull)
  int pushes = 0, pulls = 0;
  int32_t last_lev = 0;  // deepest level that discovered a vertex
  bool pull = false;     // direction of the previous level
  int64_t prev_nq = 0;   // frontier size before the last level
  bool done = false;
  int phase = 0;         // what the last launch enqueued: 1 narrow push, 2 wide push, 3 pull
  int32_t lev0 = 0;      // the level count before it

  explicit BfsRun(cudaStream_t st)
      : s(st), visited(st), fbits(st), nbits(st), qa(st), qb(st), fdeg(st), offs(st), cnt(st), cst(st) {}

  int start(char *msg) {
    const int32_t n = G->n;
    const int64_t nwords = ((int64_t)n + 31) / 32;
    LAGR_TRY(visited.alloc(nwords, msg, "visited bitmap"));
    LAGR_TRY(fbits.alloc(nwords, msg, "frontier bitmap"));
    LAGR_TRY(nbits.alloc(nwords, msg, "next frontier bitmap"));
    LAGR_TRY(qa.alloc(n, msg, "frontier queue"));
    LAGR_TRY(qb.alloc(n, msg, "frontier queue"));
    LAGR_TRY(fdeg.alloc(n, msg, "frontier degrees"));
    LAGR_TRY(offs.alloc((size_t)n + 1, msg, "frontier edge offsets"));
    LAGR_TRY(cnt.alloc(B_NSLOT, msg, "BFS counters"));
    if (coop) LAGR_TRY(cst.alloc(1, msg, "cooperative BFS state"));
    bfs_init<<<grid_for(n, 256), 256, 0, s>>>(n, level, parent, visited.p, nwords);
    bfs_seed<<<1, 1, 0, s>>>(G->rowptr, G->nnz, src, level, parent, visited.p, qa.p, cnt.p, hd);
    LAGR_LAUNCH_CHECK();
    return LAGR_OK;
  }

  int launch(char *msg) {
    const int32_t n = G->n;
    const int64_t nwords = ((int64_t)n + 31) / 32;
    const int64_t nq = h[B_NQ], mf = h[B_MF], mu = h[B_MU];
    const int32_t lev = (int32_t)h[B_LEV];
    lev0 = lev;
    if (nq == 0) {
      done = true;
      return LAGR_OK;
    }
    if (lev + 1 > n) {
      set_msg(msg, "BFS exceeded n levels");
      return LAGR_ERR_TIMEOUT;
    }
    // direction of the next level (Beamer's rule: pull once a growing frontier's edges exceed the
    // unexplored edges / alpha; push again once the frontier falls below n / beta)
    if (push_only) pull = false;
    else if (pull_only) pull = true;
    else if (!pull) pull = nq > prev_nq && mf > mu / ALPHA_DO;
    else pull = !(nq < (int64_t)n / BETA_DO);
    prev_nq = nq;
    if (!pull) {
      if (rep == 1) {  // bitmap -> queue qa
        LAGR_CUDA_TRY(cudaMemsetAsync(cnt.p + B_NEXT, 0, sizeof(int64_t), s));
        bfs_b2q<<<grid_for(nwords, 256), 256, 0, s>>>(fbits.p, nwords, qa.p, (unsigned long long *)(cnt.p + B_NEXT));
        bfs_set_par<<<1, 1, 0, s>>>(cnt.p, 0);
        LAGR_LAUNCH_CHECK();
        LAGR_CUDA_TRY(cudaMemsetAsync(cnt.p + B_NEXT, 0, sizeof(int64_t), s));
        rep = 0;
      }
      if (coop && nq >= COOP_MIN && nq <= COOP_MAX && mf <= COOP_EDGES) {
        // narrow levels on every SM: a cooperative launch (all CTAs resident), one grid barrier
        // per level, until the frontier widens past the cooperative limits or asks for a pull
        LAGR_CUDA_TRY(cudaMemsetAsync(cst.p, 0, sizeof(CoopState), s));
        const int res = resident_ctas((const void *)bfs_push_coop, COOP_THREADS, 0);
        const int grid = res < sm_count() ? res : sm_count();  // 38 to 304 CTAs measured within 5 %
        const int32_t *rp = G->rowptr, *ci = G->colidx;
        int32_t *qap = qa.p, *qbp = qb.p, *lv = level, *pa = parent;
        uint32_t *vis = visited.p;
        int64_t *cn = cnt.p, *hm = hd;
        CoopState *stp = cst.p;
        int32_t maxl = n;
        int allow = push_only ? 0 : 1;
        void *args[] = {&rp, &ci, &qap, &qbp, &vis, &lv, &pa, &cn, &stp, &maxl, &allow, &hm};
        {
          KTimer kt(TK_BFS_SMALL, s);
          LAGR_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)bfs_push_coop, dim3(grid), dim3(COOP_THREADS), args,
                                                    0, s));
        }
        note_launch();
        phase = 1;
      } else if (nq <= SMALL_MAX && mf <= SMALL_EDGES) {
        // several narrow levels in one CTA; it stops when the frontier empties, widens, or the
        // direction rule asks for a pull (the same rule as above, so it runs at least one level)
        {
          KTimer kt(TK_BFS_SMALL, s);
          bfs_push_small<<<1, SMALL_THREADS, 0, s>>>(G->rowptr, G->colidx, qa.p, qb.p, visited.p, level, parent,
                                                     cnt.p, n, push_only ? 0 : 1, hd, coop ? COOP_MIN : SMALL_MAX);
        }
        LAGR_LAUNCH_CHECK();
        phase = 1;
      } else {
        // wide push, balanced over the frontier's edges: degrees, their prefix, one CTA per
        // LB_CHUNK edges; the next frontier comes back as the bitmap nbits
        bfs_frontier_degrees<<<grid_for(nq, 256), 256, 0, s>>>(G->rowptr, qa.p, qb.p, cnt.p, fdeg.p);
        LAGR_LAUNCH_CHECK();
        LAGR_TRY(exclusive_scan(fdeg.p, offs.p, nq, s, msg));
        LAGR_CUDA_TRY(cudaMemsetAsync(nbits.p, 0, nwords * sizeof(uint32_t), s));
        const int64_t nchunks = (mf + LB_CHUNK - 1) / LB_CHUNK;
        {
          KTimer kt(TK_BFS_LB, s);
          bfs_push_lb<<<(unsigned)(nchunks > 0 ? nchunks : 1), 256, 0, s>>>(G->rowptr, G->colidx, qa.p, qb.p, offs.p,
                                                                           visited.p, nbits.p, level, parent, cnt.p);
        }
        bfs_advance<<<1, 1, 0, s>>>(cnt.p, 0, hd);
        LAGR_LAUNCH_CHECK();
        std::swap(fbits.p, nbits.p);
        rep = 1;
        phase = 2;
      }
      return LAGR_OK;
    }
    // pull level
    if (rep == 0) {  // queue -> bitmap
      LAGR_CUDA_TRY(cudaMemsetAsync(fbits.p, 0, nwords * sizeof(uint32_t), s));
      bfs_q2b<<<grid_for(nq, 256), 256, 0, s>>>(qa.p, qb.p, cnt.p, fbits.p);
      LAGR_LAUNCH_CHECK();
      rep = 1;
    }
    {
      KTimer kt(TK_BFS_PULL, s);
      bfs_pull<<<grid_for(nwords * 32, BFS_THREADS), BFS_THREADS, 0, s>>>(G->at_rowptr, G->at_colidx, G->rowptr, n,
                                                                          fbits.p, nbits.p, visited.p, level, parent,
                                                                          cnt.p);
    }
    bfs_advance<<<1, 1, 0, s>>>(cnt.p, 0, hd);
    LAGR_LAUNCH_CHECK();
    std::swap(fbits.p, nbits.p);
    phase = 3;
    return LAGR_OK;
  }

  int settle(char *msg) {
    if (phase == 1) {
      const int32_t levs = (int32_t)h[B_LEV] - lev0;
      if (h[B_EXIT] == 4) {
        set_msg(msg, "BFS exceeded n levels");
        return LAGR_ERR_TIMEOUT;
      }
      if (h[B_EXIT] == 5) {
        set_msg(msg, "a grid barrier of the cooperative BFS kernel ran out of time");
        return LAGR_ERR_TIMEOUT;
      }
      if (levs <= 0) {
        set_msg(msg, "internal: narrow-frontier kernel made no progress");
        return LAGR_ERR_TIMEOUT;
      }
      pushes += levs;
      last_lev = (h[B_NQ] > 0) ? (int32_t)h[B_LEV] : (int32_t)h[B_LEV] - 1;
    } else {
      if (phase == 2) pushes++;
      else pulls++;
      if (h[B_NQ] > 0) last_lev = (int32_t)h[B_LEV];
    }
    phase = 0;
    return LAGR_OK;
  }
};

int check_bfs_flags(int32_t flags, char *msg) {
  if (flags & ~(LAGR_BFS_PUSH_ONLY | LAGR_BFS_PULL_ONLY) ||
      (flags & (LAGR_BFS_PUSH_ONLY | LAGR_BFS_PULL_ONLY)) == (LAGR_BFS_PUSH_ONLY | LAGR_BFS_PULL_ONLY)) {
    set_msg(msg, "bad BFS flags 0x%x", flags);
    return LAGR_ERR_INVALID_VALUE;
  }
  return LAGR_OK;
}

// The library's side streams for interleaved runs (per device, created once, non-blocking)
constexpr int BFS_STREAMS = 8;
std::mutex g_bfs_stream_mu;
cudaStream_t g_bfs_streams[64][BFS_STREAMS];

int bfs_streams(cudaStream_t **out, char *msg) {
  int d = 0;
  LAGR_CUDA_TRY(cudaGetDevice(&d));
  if (d < 0 || d >= 64) {
    set_msg(msg, "device %d out of range", d);
    return LAGR_ERR_INVALID_VALUE;
  }
  std::lock_guard<std::mutex> lk(g_bfs_stream_mu);
  for (int i = 0; i < BFS_STREAMS; i++)
    if (!g_bfs_streams[d][i]) LAGR_CUDA_TRY(cudaStreamCreateWithFlags(&g_bfs_streams[d][i], cudaStreamNonBlocking));
  *out = g_bfs_streams[d];
  return LAGR_OK;
}

// the mapped host mirrors of k runs: B_NSLOT counters each, LAGR_NHOST / B_NSLOT runs per block
struct Mirrors {
  std::vector<HostBlock> blocks;
  ~Mirrors() {
    for (const HostBlock &b : blocks) host_block_put(b);
  }
  int get(int k, char *msg) {
    constexpr int per = LAGR_NHOST / B_NSLOT;
    for (int i = 0; i < (k + per - 1) / per; i++) {
      HostBlock b;
      if (!host_block_get(&b)) {
        set_msg(msg, "out of pinned host memory");
        return LAGR_ERR_OUT_OF_MEMORY;
      }
      blocks.push_back(b);
    }
    return LAGR_OK;
  }
  int64_t *host(int t) const { return blocks[t / (LAGR_NHOST / B_NSLOT)].h + (t % (LAGR_NHOST / B_NSLOT)) * B_NSLOT; }
  int64_t *dev(int t) const { return blocks[t / (LAGR_NHOST / B_NSLOT)].d + (t % (LAGR_NHOST / B_NSLOT)) * B_NSLOT; }
};

}  // namespace
}  // namespace lagr

extern "C" int lagr_bfs(int32_t *level, int32_t *parent, int32_t *depth, lagr_graph G, int32_t src, int32_t flags,
                        void *stream, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  if (src < 0 || src >= G->n) {
    set_msg(msg, "source %d out of range [0, %d)", src, G->n);
    return LAGR_ERR_INVALID_VALUE;
  }
  LAGR_TRY(check_bfs_flags(flags, msg));
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  if (!(flags & LAGR_BFS_PUSH_ONLY)) LAGR_TRY(lagr_property_AT(G, s, msg));
  Mirrors mir;
  LAGR_TRY(mir.get(1, msg));
  BfsRun r(s);
  r.G = G;
  r.src = src;
  r.level = level;
  r.parent = parent;
  r.push_only = flags & LAGR_BFS_PUSH_ONLY;
  r.pull_only = flags & LAGR_BFS_PULL_ONLY;
  r.coop = coop_supported();
  r.h = mir.host(0);
  r.hd = mir.dev(0);
  LAGR_TRY(r.start(msg));
  for (;;) {
    LAGR_CUDA_TRY(cudaStreamSynchronize(s));
    if (r.phase) LAGR_TRY(r.settle(msg));
    LAGR_TRY(r.launch(msg));
    if (r.done) break;
  }
  G->last_levels = r.last_lev + 1;
  G->last_push_levels = r.pushes;
  G->last_pull_levels = r.pulls;
  if (depth) *depth = r.last_lev + 1;
  clear_msg(msg);
  return LAGR_OK;
}

extern "C" int lagr_bfs_multi(int32_t *level, int32_t *parent, int32_t *depth, lagr_graph G, const int32_t *src,
                              int32_t k, int32_t flags, void *stream, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  if (!src) {
    set_msg(msg, "src is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  if (k < 1 || k > LAGR_BFS_MULTI_MAX) {
    set_msg(msg, "k must be in [1, %d], got %d", LAGR_BFS_MULTI_MAX, k);
    return LAGR_ERR_INVALID_VALUE;
  }
  for (int i = 0; i < k; i++)
    if (src[i] < 0 || src[i] >= G->n) {
      set_msg(msg, "source %d (index %d) out of range", src[i], i);
      return LAGR_ERR_INVALID_VALUE;
    }
  LAGR_TRY(check_bfs_flags(flags, msg));
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  if (!(flags & LAGR_BFS_PUSH_ONLY)) LAGR_TRY(lagr_property_AT(G, s, msg));
  cudaStream_t *side = nullptr;
  LAGR_TRY(bfs_streams(&side, msg));
  const int ns = k < BFS_STREAMS ? k : BFS_STREAMS;
  Mirrors mir;
  LAGR_TRY(mir.get(k, msg));
  // the side streams start after the work queued on the caller's stream, which waits for them at
  // the end.  On an error return the join first waits for the side streams, so that no kernel
  // still writes a host mirror when the mirrors go back to the pool.
  cudaEvent_t ev[BFS_STREAMS + 1] = {};
  for (int i = 0; i <= ns; i++) LAGR_CUDA_TRY(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
  struct Join {
    cudaEvent_t *ev;
    cudaStream_t s, *side;
    int ns;
    ~Join() {
      for (int i = 0; i < ns; i++) {
        cudaStreamSynchronize(side[i]);
        cudaEventRecord(ev[i + 1], side[i]);
        cudaStreamWaitEvent(s, ev[i + 1], 0);
      }
      for (int i = 0; i <= ns; i++) cudaEventDestroy(ev[i]);
    }
  };
  LAGR_CUDA_TRY(cudaEventRecord(ev[0], s));
  for (int i = 0; i < ns; i++) LAGR_CUDA_TRY(cudaStreamWaitEvent(side[i], ev[0], 0));
  const int64_t n = G->n;
  std::vector<std::unique_ptr<BfsRun>> runs;
  {
    Join join{ev, s, side, ns};
    for (int t = 0; t < k; t++) {
      runs.emplace_back(new BfsRun(side[t % ns]));
      BfsRun &r = *runs.back();
      r.G = G;
      r.src = src[t];
      r.level = level ? level + (int64_t)t * n : nullptr;
      r.parent = parent ? parent + (int64_t)t * n : nullptr;
      r.push_only = flags & LAGR_BFS_PUSH_ONLY;
      r.pull_only = flags & LAGR_BFS_PULL_ONLY;
      r.h = mir.host(t);
      r.hd = mir.dev(t);
      LAGR_TRY(r.start(msg));
    }
    for (;;) {
      for (int i = 0; i < ns; i++) LAGR_CUDA_TRY(cudaStreamSynchronize(side[i]));
      bool active = false;
      for (auto &rp : runs) {
        if (rp->done) continue;
        if (rp->phase) LAGR_TRY(rp->settle(msg));
        LAGR_TRY(rp->launch(msg));
        active = active || !rp->done;
      }
      if (!active) break;
    }
    for (int t = 0; t < k; t++)
      if (depth) depth[t] = runs[t]->last_lev + 1;
    const BfsRun &last = *runs.back();
    G->last_levels = last.last_lev + 1;
    G->last_push_levels = last.pushes;
    G->last_pull_levels = last.pulls;
    runs.clear();  // the work space is freed on the side streams before the join
  }
  clear_msg(msg);
  return LAGR_OK;
}

extern "C" int lagr_bfs_batch64(int32_t *level, lagr_graph G, const int32_t *src, int32_t k, void *stream,
                                char *msg) {
  if (!level || !src) {
    set_msg(msg, "level/src is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(check_graph_arg(G, msg));
  if (k < 1 || k > 64) {
    set_msg(msg, "k must be in [1, 64], got %d", k);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (G->kind != LAGR_UNDIRECTED) {
    set_msg(msg, "the 64-source BFS needs an undirected graph");
    return LAGR_ERR_INVALID_GRAPH;
  }
  for (int i = 0; i < k; i++)
    if (src[i] < 0 || src[i] >= G->n) {
      set_msg(msg, "source %d (index %d) out of range", src[i], i);
      return LAGR_ERR_INVALID_VALUE;
    }
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  LAGR_TRY(lagr_property_AT(G, s, msg));
  LAGR_TRY(row_plan(&P->pr_at, G->rowptr, G->n, s, msg));
  const RowPlan &rp = P->pr_at;
  const int32_t n = G->n;
  Temp<unsigned long long> seen(s), fa(s), fb(s), acc(s);
  Temp<int32_t> la(s), lb(s), touched(s), fdeg(s), offs(s);
  Temp<int64_t> cnt(s);
  LAGR_TRY(seen.alloc(n, msg, "seen words"));
  LAGR_TRY(fa.alloc(n, msg, "frontier words"));
  LAGR_TRY(fb.alloc(n, msg, "frontier words"));
  LAGR_TRY(acc.alloc(n, msg, "push words"));
  LAGR_TRY(la.alloc(n, msg, "frontier list"));
  LAGR_TRY(lb.alloc(n, msg, "frontier list"));
  LAGR_TRY(touched.alloc(n, msg, "touched list"));
  LAGR_TRY(fdeg.alloc(n, msg, "frontier degrees"));
  LAGR_TRY(offs.alloc((size_t)n + 1, msg, "frontier offsets"));
  LAGR_TRY(cnt.alloc(2 * S64_NSLOT, msg, "counters"));
  // the sources travel as a kernel argument (no copy)
  Sources64 sv;
  for (int i = 0; i < 64; i++) sv.v[i] = i < k ? src[i] : 0;
  const unsigned long long kmask = (k == 64) ? ~0ull : ((1ull << k) - 1);
  bfs64_init<<<grid_for((int64_t)k * n, 256), 256, 0, s>>>(n, k, level, seen.p, fa.p, fb.p, acc.p);
  bfs64_seed<<<1, 32, 0, s>>>(n, k, sv, G->rowptr, level, seen.p, fa.p, la.p, cnt.p);
  LAGR_LAUNCH_CHECK();
  unsigned long long *front = fa.p, *fnext = fb.p;
  int32_t *flist = la.p, *nflist = lb.p;
  int64_t *cur = cnt.p, *nxt = cnt.p + S64_NSLOT;  // counters of this level / the next
  LAGR_TRY(fetch_to_host(P->hscal, cur, S64_NSLOT * sizeof(int64_t), s, msg));
  int64_t nf = P->hscal[S64_NF], mf = P->hscal[S64_MF];
  int32_t lev = 0;
  const int nhb = rp.nheavy < sm_count() ? rp.nheavy : sm_count();
  while (nf > 0) {
    lev++;
    if (lev > n) {
      set_msg(msg, "BFS exceeded n levels");
      return LAGR_ERR_TIMEOUT;
    }
    LAGR_CUDA_TRY(cudaMemsetAsync(nxt, 0, S64_NSLOT * sizeof(int64_t), s));
    if (mf * ALPHA_DO < G->nnz) {
      // push over the frontier's edges
      bfs64_fdeg<<<grid_for(nf, 256), 256, 0, s>>>(G->rowptr, flist, (int32_t)nf, fdeg.p);
      LAGR_LAUNCH_CHECK();
      LAGR_TRY(exclusive_scan(fdeg.p, offs.p, nf, s, msg));
      LAGR_CUDA_TRY(cudaMemsetAsync(cur + S64_NT, 0, sizeof(int64_t), s));
      const int64_t nchunks = (mf + LB_CHUNK - 1) / LB_CHUNK;
      if (nchunks > 0)
        bfs64_push_lb<<<(unsigned)nchunks, 256, 0, s>>>(G->rowptr, G->colidx, flist, (int32_t)nf, offs.p, front,
                                                        seen.p, acc.p, touched.p, cur);
      bfs64_finish_push<<<grid_for(n, 256), 256, 0, s>>>(touched.p, cur, G->rowptr, acc.p, seen.p, fnext, level, n,
                                                         lev, nflist, nxt);
    } else {
      bfs64_pull_rows<<<rp.nblk + nhb, 256, 0, s>>>(G->rowptr, G->colidx, rp.blk, rp.nblk, rp.heavy, rp.nheavy, kmask,
                                                    front, seen.p, fnext, level, n, lev, nflist, nxt);
    }
    bfs64_clear<<<grid_for(nf, 256), 256, 0, s>>>(flist, (int32_t)nf, front);
    LAGR_LAUNCH_CHECK();
    LAGR_TRY(fetch_to_host(P->hscal, nxt, S64_NSLOT * sizeof(int64_t), s, msg));
    nf = P->hscal[S64_NF];
    mf = P->hscal[S64_MF];
    std::swap(front, fnext);
    std::swap(flist, nflist);
    std::swap(cur, nxt);
  }
  G->last_levels = lev;
  clear_msg(msg);
  return LAGR_OK;
}

// ---- BFS without any device allocation -----------------------------------------------------------
//
// Some callers cannot allocate device memory at all: a process whose device memory is handed out
// up front by another framework and may not grow, code that runs while the allocator must not be
// touched (a host thread racing other work on the same context, a latency-critical loop that must
// not block in cudaMalloc/cudaFree), or a runtime with no allocator behind it.  For them
// lagr_bfs_noalloc keeps its whole work space (visited and frontier bitmaps, the two vertex
// queues and the level counters) in one fixed array compiled into this file, so the caller only
// provides the graph and the outputs.
//
// The array is a file-scope __device__ variable: a GPU holds its LAGR_BFS_NOALLOC_MAX_N-sized copy
// (about 17 MB) from the moment this file's device code is loaded on it (with CUDA's lazy module
// loading, at the first use of one of its kernels on that device) until the process exits.  Host
// code cannot use the variable's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress while that device is current and remembers it; make that
// first call before capturing a stream.  Every call on a device shares the one array and leaves its contents
// behind; each call clears what it needs at the start, and calls whose GPU work overlaps (two
// streams, or two host threads) race on the array and must be serialised by the caller.

namespace lagr {
namespace {

constexpr int64_t NA_WORDS = LAGR_BFS_NOALLOC_MAX_N / 32;
constexpr size_t NA_BITMAP_BYTES = (size_t)NA_WORDS * sizeof(uint32_t);
constexpr size_t NA_QUEUE_BYTES = (size_t)LAGR_BFS_NOALLOC_MAX_N * sizeof(int32_t);
// layout: visited | frontier bitmap | next bitmap | queue a | queue b | counters
constexpr size_t NA_OFF_VISITED = 0;
constexpr size_t NA_OFF_FBITS = NA_OFF_VISITED + NA_BITMAP_BYTES;
constexpr size_t NA_OFF_NBITS = NA_OFF_FBITS + NA_BITMAP_BYTES;
constexpr size_t NA_OFF_QA = NA_OFF_NBITS + NA_BITMAP_BYTES;
constexpr size_t NA_OFF_QB = NA_OFF_QA + NA_QUEUE_BYTES;
constexpr size_t NA_OFF_CNT = NA_OFF_QB + NA_QUEUE_BYTES;
constexpr size_t NA_BYTES = NA_OFF_CNT + B_NSLOT * sizeof(int64_t);
static_assert(NA_OFF_CNT % 8 == 0, "counter alignment");

static __device__ __align__(256) unsigned char g_bfs_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 256;
// device address of the array, per device (atomic: host threads may make their first calls at once;
// they look up and store the same address)
static std::atomic<unsigned char *> g_na_ptr[NA_MAX_DEVICES];

int noalloc_scratch(unsigned char **out, char *msg) {
  int dev = 0;
  LAGR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) {
    set_msg(msg, "device ordinal %d out of range", dev);
    return LAGR_ERR_INVALID_VALUE;
  }
  unsigned char *p = g_na_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *q = nullptr;
    LAGR_CUDA_TRY(cudaGetSymbolAddress(&q, g_bfs_noalloc_scratch));
    p = static_cast<unsigned char *>(q);
    g_na_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return LAGR_OK;
}

}  // namespace
}  // namespace lagr

extern "C" int lagr_bfs_noalloc(int32_t *level, int32_t *parent, int32_t *depth, int32_t n, int64_t nnz,
                                const int32_t *rowptr, const int32_t *colidx, int32_t src, void *stream,
                                char *msg) {
  if (n < 1 || nnz < 0) {
    set_msg(msg, "need n >= 1 and nnz >= 0 (n=%d, nnz=%lld)", n, (long long)nnz);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (n > LAGR_BFS_NOALLOC_MAX_N || nnz >= ((int64_t)1 << 31)) {
    set_msg(msg, "lagr_bfs_noalloc handles at most %d vertices and < 2^31 entries (n=%d, nnz=%lld); use lagr_bfs",
            LAGR_BFS_NOALLOC_MAX_N, n, (long long)nnz);
    return LAGR_ERR_TOO_LARGE;
  }
  if (!rowptr || (nnz > 0 && !colidx)) {
    set_msg(msg, "rowptr/colidx is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  if (src < 0 || src >= n) {
    set_msg(msg, "source %d out of range [0, %d)", src, n);
    return LAGR_ERR_INVALID_VALUE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *base = nullptr;
  LAGR_TRY(noalloc_scratch(&base, msg));
  uint32_t *visited = reinterpret_cast<uint32_t *>(base + NA_OFF_VISITED);
  uint32_t *fbits = reinterpret_cast<uint32_t *>(base + NA_OFF_FBITS);
  uint32_t *nbits = reinterpret_cast<uint32_t *>(base + NA_OFF_NBITS);
  int32_t *qa = reinterpret_cast<int32_t *>(base + NA_OFF_QA);
  int32_t *qb = reinterpret_cast<int32_t *>(base + NA_OFF_QB);
  int64_t *cnt = reinterpret_cast<int64_t *>(base + NA_OFF_CNT);
  const int64_t nwords = ((int64_t)n + 31) / 32;

  // bfs_init clears the visited words and the outputs, bfs_seed resets every counter
  bfs_init<<<grid_for(n, 256), 256, 0, s>>>(n, level, parent, visited, nwords);
  bfs_seed<<<1, 1, 0, s>>>(rowptr, nnz, src, level, parent, visited, qa, cnt, nullptr);
  LAGR_LAUNCH_CHECK();
  int64_t h[B_NSLOT];
  auto sync_counters = [&]() -> int {
    LAGR_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    LAGR_CUDA_TRY(cudaStreamSynchronize(s));
    return LAGR_OK;
  };
  LAGR_TRY(sync_counters());
  int rep = 0;  // 0: frontier in a queue, 1: in fbits
  bool pull = false;
  int64_t prev_nq = 0;
  int32_t last_lev = 0;
  for (;;) {
    const int64_t nq = h[B_NQ], mf = h[B_MF], mu = h[B_MU];
    const int32_t lev = (int32_t)h[B_LEV];
    if (nq == 0) break;
    if (lev + 1 > n) {
      set_msg(msg, "BFS exceeded n levels");
      return LAGR_ERR_TIMEOUT;
    }
    if (!pull) pull = nq > prev_nq && mf > mu / ALPHA_DO;
    else pull = !(nq < (int64_t)n / BETA_DO);
    prev_nq = nq;
    if (!pull) {
      if (rep == 1) {
        LAGR_CUDA_TRY(cudaMemsetAsync(cnt + B_NEXT, 0, sizeof(int64_t), s));
        bfs_b2q<<<grid_for(nwords, 256), 256, 0, s>>>(fbits, nwords, qa, (unsigned long long *)(cnt + B_NEXT));
        bfs_set_par<<<1, 1, 0, s>>>(cnt, 0);
        LAGR_LAUNCH_CHECK();
        LAGR_CUDA_TRY(cudaMemsetAsync(cnt + B_NEXT, 0, sizeof(int64_t), s));
        rep = 0;
      }
      if (nq <= SMALL_MAX && mf <= SMALL_EDGES) {
        bfs_push_small<<<1, SMALL_THREADS, 0, s>>>(rowptr, colidx, qa, qb, visited, level, parent, cnt, n, 1,
                                                   nullptr);
        LAGR_LAUNCH_CHECK();
        LAGR_TRY(sync_counters());
        if (h[B_EXIT] == 4 || (int32_t)h[B_LEV] <= lev) {
          set_msg(msg, "BFS exceeded n levels");
          return LAGR_ERR_TIMEOUT;
        }
        last_lev = (h[B_NQ] > 0) ? (int32_t)h[B_LEV] : (int32_t)h[B_LEV] - 1;
      } else {
        LAGR_CUDA_TRY(cudaMemsetAsync(nbits, 0, nwords * sizeof(uint32_t), s));
        bfs_push<<<grid_for(nq, BFS_THREADS), BFS_THREADS, 0, s>>>(rowptr, colidx, qa, qb, visited, nbits, level,
                                                                   parent, cnt);
        bfs_advance<<<1, 1, 0, s>>>(cnt, 0, nullptr);
        LAGR_LAUNCH_CHECK();
        uint32_t *t = fbits;
        fbits = nbits;
        nbits = t;
        rep = 1;
        LAGR_TRY(sync_counters());
        if (h[B_NQ] > 0) last_lev = (int32_t)h[B_LEV];
      }
      continue;
    }
    if (rep == 0) {
      LAGR_CUDA_TRY(cudaMemsetAsync(fbits, 0, nwords * sizeof(uint32_t), s));
      bfs_q2b<<<grid_for(nq, 256), 256, 0, s>>>(qa, qb, cnt, fbits);
      LAGR_LAUNCH_CHECK();
      rep = 1;
    }
    // the graph is undirected, so A' = A: the pull scans the rows of A
    bfs_pull<<<grid_for(nwords * 32, BFS_THREADS), BFS_THREADS, 0, s>>>(rowptr, colidx, rowptr, n, fbits, nbits,
                                                                        visited, level, parent, cnt);
    bfs_advance<<<1, 1, 0, s>>>(cnt, 0, nullptr);
    LAGR_LAUNCH_CHECK();
    uint32_t *t = fbits;
    fbits = nbits;
    nbits = t;
    LAGR_TRY(sync_counters());
    if (h[B_NQ] > 0) last_lev = (int32_t)h[B_LEV];
  }
  if (depth) *depth = last_lev + 1;
  clear_msg(msg);
  return LAGR_OK;
}
