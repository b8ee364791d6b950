// Batched betweenness centrality (Alg. 3, Sec. IV-B) in float64, up to 64 sources at once.
//
// Alg. 3 keeps ns x n matrices: P (shortest-path counts), the frontier F, the per-level patterns
// S[d], and in the backtrack B (one plus the accumulated dependencies) and W.  Here the ns rows are
// interleaved per vertex (row-major n x ns: the ns values of a vertex are contiguous) and the
// pattern of a frontier is a 64-bit source mask per vertex, as in the 64-source BFS:
//
//  - BFS phase, direction-optimised (push or pull per level, as Sec. IV-B adds it to BC; the pull
//    is taken when it reads under half the edges of the push, see the host loop).  The frontier of level d is a list of
//    (vertex, mask) pairs.  One push step,
//    F<!s(P), replace> = F plus.first A fused with P += F, walks the list's edges (edge-balanced:
//    a hub's row is spread over many warps): for an edge v -> w the sources m = mask(v) & ~seen(w)
//    that reach w for the first time add P(v) into P(w) (float64 atomics; the counts are integers
//    below 2^53, so their sums are exact and do not depend on the order) and set m in w's mask for
//    the next level.  A finishing pass turns the touched vertices' masks into the next list and
//    adds them to seen.  The lists of all levels are kept: they are the patterns S[d].  A pull step
//    computes the same product from the unreached side (bc_fwd_pull, over the rows of A').
//  - Backtrack.  For each level d from the deepest down to 2: W = B ./ P on the pattern of level
//    d, then W<s(S[d-1])> = W plus.first A' as a pull over the rows of level d-1 (each such vertex
//    u sums W(l) over its out-neighbours l that are on level d for the same source: one warp
//    reduction per source and chunk), then B += W .* P on level d-1.
//  - centrality(j) = sum over the sources of B(k, j) - 1.
// The backtrack starts at the deepest level, so every level's dependencies reach the level above
// (the loop bounds of the printed algorithm would skip the deepest level; see the design notes).
#include <algorithm>
#include <vector>

#include "frontier.cuh"

namespace lagr {
namespace {

constexpr int BC_THREADS = 256;
enum BcSlot { BC_NNEXT = 0, BC_NCAND = 1, BC_MU = 2, BC_MF = 3, BC_NSLOT = 4 };
constexpr int BC_PULL_MARGIN = 2;  // pull when the unreached vertices' edges are under half the frontier's

struct BcSources {
  int32_t v[64];
};

// P(s_k, k) = 1, seen(s_k) has bit k, and the distinct sources with their masks form level 0
__global__ void bc_seed(int32_t ns, const BcSources src, int32_t *__restrict__ lvert,
                        unsigned long long *__restrict__ lmask, unsigned long long *__restrict__ seen,
                        double *__restrict__ sigma, int64_t *__restrict__ cnt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t nl = 0;
  for (int32_t k = 0; k < ns; k++) {
    const int32_t v = src.v[k];
    sigma[(int64_t)v * ns + k] = 1.0;
    const unsigned long long bit = 1ull << k;
    int64_t j = 0;
    while (j < nl && lvert[j] != v) j++;
    if (j == nl) {
      lvert[nl] = v;
      lmask[nl] = 0;
      nl++;
    }
    lmask[j] |= bit;
    seen[v] |= bit;
  }
  cnt[BC_NNEXT] = nl;
}

// One push step of the BFS phase from the level list (lvert, lmask)[0 .. nent) (chunk plan off):
// new (vertex, source) pairs get their path counts and their bits in nmask; a vertex touched for
// the first time is appended to nvert.
__global__ void __launch_bounds__(BC_THREADS)
    bc_push(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t ns,
            const int32_t *__restrict__ lvert, const unsigned long long *__restrict__ lmask, int32_t nent,
            const int32_t *__restrict__ off, const unsigned long long *__restrict__ seen,
            unsigned long long *__restrict__ nmask, double *__restrict__ sigma, int32_t *__restrict__ nvert,
            int64_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = nent > 0 ? off[nent] : 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int32_t i = fx_entry_of(off, nent, (int32_t)c);
    const int32_t v = lvert[i];
    const unsigned long long mv = lmask[i];
    const int32_t b = rowptr[v] + ((int32_t)c - off[i]) * FX_CHUNK;
    const int32_t e = min(rowptr[v + 1], b + FX_CHUNK);
    const double *sv = sigma + (int64_t)v * ns;
    for (int32_t k = b + lane; k < e; k += 32) {
      const int32_t w = __ldg(&colidx[k]);
      unsigned long long m = mv & ~seen[w];
      if (!m) continue;
      const unsigned long long old = atomicOr(&nmask[w], m);
      if (old == 0) nvert[atomicAdd((unsigned long long *)&cnt[BC_NNEXT], 1ull)] = w;
      double *sw = sigma + (int64_t)w * ns;
      while (m) {
        const int q = __ffsll((long long)m) - 1;
        m &= m - 1;
        atomicAdd(&sw[q], sv[q]);
      }
    }
  }
}

// The direction rule's counts and the pull's candidates: the vertices some source has not reached
// (listed in cand), the edges of those vertices (mu) and the out-edges of the level's list (mf).
__global__ void bc_census(int32_t n, unsigned long long full, const unsigned long long *__restrict__ seen,
                          const int32_t *__restrict__ rowptr, const int32_t *__restrict__ lvert, int32_t nent,
                          int32_t *__restrict__ cand, int64_t *__restrict__ cnt) {
  unsigned long long mu = 0, mf = 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = b + threadIdx.x;
    const bool need = w < n && (full & ~seen[w]) != 0;
    if (need) mu += (unsigned long long)(rowptr[w + 1] - rowptr[w]);
    const unsigned bal = __ballot_sync(LAGR_FULL_MASK, need);
    unsigned long long pos = 0;
    if (lane == 0 && bal) pos = atomicAdd((unsigned long long *)&cnt[BC_NCAND], (unsigned long long)__popc(bal));
    pos = __shfl_sync(LAGR_FULL_MASK, pos, 0);
    if (need) cand[pos + __popc(bal & lt)] = (int32_t)w;
  }
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lvert[j];
    mf += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
  }
  mu = warp_sum(mu);
  mf = warp_sum(mf);
  if (lane == 0) {
    if (mu) atomicAdd((unsigned long long *)&cnt[BC_MU], mu);
    if (mf) atomicAdd((unsigned long long *)&cnt[BC_MF], mf);
  }
}

__global__ void bc_scatter_masks(const int32_t *__restrict__ lvert, const unsigned long long *__restrict__ lmask,
                                 int32_t nent, unsigned long long *__restrict__ dmask) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent; j += (int64_t)gridDim.x * blockDim.x)
    dmask[lvert[j]] = lmask[j];
}

// One pull step of the BFS phase, F<!s(P), replace> = F plus.first A computed from the side of the
// vertices not yet reached (the direction optimisation the paper adds to BC as Alg. 2 adds it to
// Alg. 1): every candidate w sums P(v) over its in-neighbours v (rows of A') that are on the
// level's frontier for a source w still lacks (fmask: the level's masks, dense).  At most NS
// sources keep per-lane sums over the chunk; NS = 0 reduces per 32 edges for any ns.  A chunk adds
// its sums with one float64 atomic per source (the counts are integers: exact in any order) and
// sets the sources it reached in nmask; the first to set any appends w to the next list.
template <int NS>
__global__ void __launch_bounds__(BC_THREADS)
    bc_fwd_pull(const int32_t *__restrict__ at_rowptr, const int32_t *__restrict__ at_colidx, int32_t ns,
                unsigned long long full, const int32_t *__restrict__ cand, int32_t nent,
                const int32_t *__restrict__ off, const unsigned long long *__restrict__ seen,
                const unsigned long long *__restrict__ fmask, unsigned long long *__restrict__ nmask,
                double *__restrict__ sigma, int32_t *__restrict__ nvert, int64_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = nent > 0 ? off[nent] : 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int32_t i = fx_entry_of(off, nent, (int32_t)c);
    const int32_t w = cand[i];
    const unsigned long long need = full & ~seen[w];
    const int32_t b = at_rowptr[w] + ((int32_t)c - off[i]) * FX_CHUNK;
    const int32_t e = min(at_rowptr[w + 1], b + FX_CHUNK);
    double *sw = sigma + (int64_t)w * ns;
    unsigned long long got = 0;  // sources with a term in this chunk (every lane)
    if (NS > 0) {
      double a[NS > 0 ? NS : 1];
#pragma unroll
      for (int q = 0; q < (NS > 0 ? NS : 1); q++) a[q] = 0.0;
      unsigned long long touched = 0;
      for (int32_t k = b + lane; k < e; k += 32) {
        const int32_t v = __ldg(&at_colidx[k]);
        const unsigned long long mm = fmask[v] & need;
        touched |= mm;
#pragma unroll
        for (int q = 0; q < (NS > 0 ? NS : 1); q++)
          if ((mm >> q) & 1ull) a[q] += sigma[(int64_t)v * ns + q];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) touched |= __shfl_xor_sync(LAGR_FULL_MASK, touched, o);
      got = touched;
#pragma unroll
      for (int q = 0; q < (NS > 0 ? NS : 1); q++) {
        if (!((got >> q) & 1ull)) continue;
        double t = a[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(LAGR_FULL_MASK, t, o);
        if (lane == 0) atomicAdd(&sw[q], t);
      }
    } else {
      for (int32_t base = b; base < e; base += 32) {
        const int32_t k = base + lane;
        int32_t v = 0;
        unsigned long long mm = 0;
        if (k < e) {
          v = __ldg(&at_colidx[k]);
          mm = fmask[v] & need;
        }
        unsigned long long any = mm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(LAGR_FULL_MASK, any, o);
        got |= any;
        while (any) {
          const int q = __ffsll((long long)any) - 1;
          any &= any - 1;
          double t = ((mm >> q) & 1ull) ? sigma[(int64_t)v * ns + q] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(LAGR_FULL_MASK, t, o);
          if (lane == 0) atomicAdd(&sw[q], t);
        }
      }
    }
    if (lane == 0 && got) {
      const unsigned long long old = atomicOr(&nmask[w], got);
      if (old == 0) nvert[atomicAdd((unsigned long long *)&cnt[BC_NNEXT], 1ull)] = w;
    }
  }
}

// the next level's list: masks out of nmask (cleared), added to seen
__global__ void bc_push_finish(const int32_t *__restrict__ nvert, int32_t nn, unsigned long long *__restrict__ nmask,
                               unsigned long long *__restrict__ nlmask, unsigned long long *__restrict__ seen) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = nvert[j];
    const unsigned long long m = nmask[w];
    nmask[w] = 0;
    nlmask[j] = m;
    seen[w] |= m;
  }
}

// W = B ./ P on the pattern of one level; that level's masks into the dense dmask
__global__ void bc_level_w(int32_t ns, const int32_t *__restrict__ lvert, const unsigned long long *__restrict__ lmask,
                           int32_t nent, const double *__restrict__ B, const double *__restrict__ sigma,
                           double *__restrict__ W, unsigned long long *__restrict__ dmask) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lvert[j];
    unsigned long long m = lmask[j];
    dmask[v] = m;
    while (m) {
      const int q = __ffsll((long long)m) - 1;
      m &= m - 1;
      const int64_t x = (int64_t)v * ns + q;
      W[x] = B[x] / sigma[x];
    }
  }
}

// W<s(S[d-1])> = W plus.first A': every vertex u of level d-1 (for the sources of its mask) sums W
// over its out-neighbours on level d for the same source; one warp per chunk of u's row, one warp
// reduction per source, partial sums added into acc
__global__ void __launch_bounds__(BC_THREADS)
    bc_pull(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t ns,
            const int32_t *__restrict__ lvert, const unsigned long long *__restrict__ lmask, int32_t nent,
            const int32_t *__restrict__ off, const unsigned long long *__restrict__ dmask,
            const double *__restrict__ W, double *__restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = nent > 0 ? off[nent] : 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int32_t i = fx_entry_of(off, nent, (int32_t)c);
    const int32_t u = lvert[i];
    const unsigned long long mu = lmask[i];
    const int32_t b = rowptr[u] + ((int32_t)c - off[i]) * FX_CHUNK;
    const int32_t e = min(rowptr[u + 1], b + FX_CHUNK);
    for (int32_t base = b; base < e; base += 32) {
      const int32_t k = base + lane;
      int32_t l = 0;
      unsigned long long mm = 0;
      if (k < e) {
        l = __ldg(&colidx[k]);
        mm = mu & dmask[l];
      }
      unsigned long long any = mm;  // the sources some lane has a term for (OR over the warp)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(LAGR_FULL_MASK, any, o);
      while (any) {
        const int q = __ffsll((long long)any) - 1;
        any &= any - 1;
        double t = ((mm >> q) & 1ull) ? W[(int64_t)l * ns + q] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(LAGR_FULL_MASK, t, o);
        if (lane == 0) atomicAdd(&acc[(int64_t)u * ns + q], t);
      }
    }
  }
}

// The same pull for at most NS sources: each lane keeps one running sum per source over the chunk's
// edges in registers, and the warp reduces each source once per chunk instead of once per 32 edges.
template <int NS>
__global__ void __launch_bounds__(BC_THREADS)
    bc_pull_few(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t ns,
                const int32_t *__restrict__ lvert, const unsigned long long *__restrict__ lmask, int32_t nent,
                const int32_t *__restrict__ off, const unsigned long long *__restrict__ dmask,
                const double *__restrict__ W, double *__restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = nent > 0 ? off[nent] : 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int32_t i = fx_entry_of(off, nent, (int32_t)c);
    const int32_t u = lvert[i];
    const unsigned long long mu = lmask[i];
    const int32_t b = rowptr[u] + ((int32_t)c - off[i]) * FX_CHUNK;
    const int32_t e = min(rowptr[u + 1], b + FX_CHUNK);
    double a[NS];
#pragma unroll
    for (int q = 0; q < NS; q++) a[q] = 0.0;
    unsigned touched = 0;  // the sources this lane has a term for
    for (int32_t k = b + lane; k < e; k += 32) {
      const int32_t l = __ldg(&colidx[k]);
      const unsigned mm = (unsigned)(mu & dmask[l]);
      touched |= mm;
#pragma unroll
      for (int q = 0; q < NS; q++)
        if ((mm >> q) & 1u) a[q] += W[(int64_t)l * ns + q];
    }
    const unsigned any = __reduce_or_sync(LAGR_FULL_MASK, touched);
#pragma unroll
    for (int q = 0; q < NS; q++) {
      if (!((any >> q) & 1u)) continue;
      double t = a[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(LAGR_FULL_MASK, t, o);
      if (lane == 0) atomicAdd(&acc[(int64_t)u * ns + q], t);
    }
  }
}

// B += W .* P on level d-1 (W there is the pulled sum in acc, cleared here); level d's dense masks
// are cleared by the caller's second call with clear_only
__global__ void bc_level_apply(int32_t ns, const int32_t *__restrict__ lvert,
                               const unsigned long long *__restrict__ lmask, int32_t nent,
                               const double *__restrict__ sigma, double *__restrict__ acc, double *__restrict__ B) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = lvert[j];
    unsigned long long m = lmask[j];
    while (m) {
      const int q = __ffsll((long long)m) - 1;
      m &= m - 1;
      const int64_t x = (int64_t)u * ns + q;
      B[x] += acc[x] * sigma[x];
      acc[x] = 0.0;
    }
  }
}

__global__ void bc_clear_masks(const int32_t *__restrict__ lvert, int32_t nent, unsigned long long *__restrict__ dmask) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nent; j += (int64_t)gridDim.x * blockDim.x)
    dmask[lvert[j]] = 0;
}

__global__ void bc_fill(int64_t len, double v, double *__restrict__ a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// centrality(j) = -ns + sum_k B(j, k)
__global__ void bc_reduce(int32_t n, int32_t ns, const double *__restrict__ B, double *__restrict__ centrality) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double c = -(double)ns;
    for (int32_t k = 0; k < ns; k++) c += B[j * ns + k];
    centrality[j] = c;
  }
}

}  // namespace
}  // namespace lagr

using namespace lagr;

extern "C" int lagr_betweenness(double *centrality, int32_t *levels, lagr_graph G, const int32_t *src, int32_t ns,
                                void *stream, char *msg) {
  if (!centrality || !src) {
    set_msg(msg, "centrality or src is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  LAGR_TRY(check_graph_arg(G, msg));
  if (ns < 1 || ns > 64) {
    set_msg(msg, "need 1 <= ns <= 64 sources, got %d", ns);
    return LAGR_ERR_INVALID_VALUE;
  }
  const int32_t n = G->n;
  for (int32_t k = 0; k < ns; k++)
    if (src[k] < 0 || src[k] >= n) {
      set_msg(msg, "source %d (%d) out of range [0, %d)", k, src[k], n);
      return LAGR_ERR_INVALID_VALUE;
    }
  if (levels) *levels = 0;
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  const int64_t N = (int64_t)n * ns;
  Temp<double> sigma(s), B(s), W(s), acc(s);
  Temp<unsigned long long> seen(s), nmask(s), dmask(s);
  Temp<int64_t> cnt(s);
  LAGR_TRY(sigma.alloc(N, msg, "path counts"));
  LAGR_TRY(B.alloc(N, msg, "dependencies"));
  LAGR_TRY(W.alloc(N, msg, "backtrack values"));
  LAGR_TRY(acc.alloc(N, msg, "backtrack sums"));
  LAGR_TRY(seen.alloc(n, msg, "reached masks"));
  LAGR_TRY(nmask.alloc(n, msg, "next masks"));
  LAGR_TRY(dmask.alloc(n, msg, "level masks"));
  LAGR_TRY(cnt.alloc(BC_NSLOT, msg, "counters"));
  Temp<int32_t> cand(s);
  LAGR_TRY(cand.alloc(n, msg, "pull candidates"));
  LAGR_TRY(lagr_property_AT(G, s, msg));  // the pull reads in-neighbours (A' aliases A when undirected)
  // the level lists (vertex, mask), all levels one after the other; grown when a level may not fit
  int64_t cap = (int64_t)n * (ns < 4 ? ns : 4) + 64;
  Temp<int32_t> lv(s);
  Temp<unsigned long long> lm(s);
  LAGR_TRY(lv.alloc(cap, msg, "level lists"));
  LAGR_TRY(lm.alloc(cap, msg, "level masks"));
  FxSpace fx;
  struct FxGuard {
    FxSpace *f;
    cudaStream_t s;
    ~FxGuard() { fx_free(f, s); }
  } fxg{&fx, s};
  LAGR_TRY(fx_alloc(&fx, n, s, msg));

  LAGR_CUDA_TRY(cudaMemsetAsync(sigma.p, 0, N * sizeof(double), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(acc.p, 0, N * sizeof(double), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(seen.p, 0, (size_t)n * sizeof(unsigned long long), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(nmask.p, 0, (size_t)n * sizeof(unsigned long long), s));
  LAGR_CUDA_TRY(cudaMemsetAsync(dmask.p, 0, (size_t)n * sizeof(unsigned long long), s));
  bc_fill<<<grid_for(N, BC_THREADS), BC_THREADS, 0, s>>>(N, 1.0, B.p);
  BcSources sv;  // the sources travel as a kernel argument (no copy)
  for (int32_t k = 0; k < 64; k++) sv.v[k] = k < ns ? src[k] : 0;
  bc_seed<<<1, 32, 0, s>>>(ns, sv, lv.p, lm.p, seen.p, sigma.p, cnt.p);
  LAGR_LAUNCH_CHECK();
  int64_t h[BC_NSLOT];
  LAGR_TRY(fetch_to_host(h, cnt.p, sizeof(h), s, msg));
  std::vector<int64_t> start = {0, h[BC_NNEXT]};  // level d's list is [start[d], start[d+1])
  const int grid = resident_ctas((const void *)bc_push, BC_THREADS, 0);
  const int fgrid4 = resident_ctas((const void *)bc_fwd_pull<4>, BC_THREADS, 0);
  const int fgrid8 = resident_ctas((const void *)bc_fwd_pull<8>, BC_THREADS, 0);
  const int fgrid0 = resident_ctas((const void *)bc_fwd_pull<0>, BC_THREADS, 0);
  const unsigned long long full = ns == 64 ? ~0ull : ((1ull << ns) - 1);
  int pulls = 0, pushes = 0;  // BFS-phase steps by direction (the last one finds no new vertex)
  bool pull = false;
  const int pgrid = resident_ctas((const void *)bc_pull, BC_THREADS, 0);
  const int pgrid4 = resident_ctas((const void *)bc_pull_few<4>, BC_THREADS, 0);
  const int pgrid8 = resident_ctas((const void *)bc_pull_few<8>, BC_THREADS, 0);
  // BFS phase
  for (int32_t d = 0;; d++) {
    if (d > n) {
      set_msg(msg, "BFS phase exceeded n levels");
      return LAGR_ERR_TIMEOUT;
    }
    const int64_t s0 = start[d], nent = start[d + 1] - start[d];
    if (start[d + 1] + n > cap) {  // room for a full next level
      const int64_t ncap = std::max<int64_t>(2 * cap, start[d + 1] + n);
      Temp<int32_t> lv2(s);
      Temp<unsigned long long> lm2(s);
      LAGR_TRY(lv2.alloc(ncap, msg, "level lists"));
      LAGR_TRY(lm2.alloc(ncap, msg, "level masks"));
      LAGR_CUDA_TRY(cudaMemcpyAsync(lv2.p, lv.p, start[d + 1] * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      LAGR_CUDA_TRY(cudaMemcpyAsync(lm2.p, lm.p, start[d + 1] * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                    s));
      std::swap(lv.p, lv2.p);
      std::swap(lm.p, lm2.p);
      cap = ncap;
    }
    // direction of the step (Beamer's rule over the sources' union): pull once the frontier's
    // out-edges exceed the edges of the vertices still unreached by some source / alpha
    LAGR_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, BC_NSLOT * sizeof(int64_t), s));
    bc_census<<<grid_for(n, BC_THREADS), BC_THREADS, 0, s>>>(n, full, seen.p, G->rowptr, lv.p + s0, (int32_t)nent,
                                                             cand.p, cnt.p);
    LAGR_LAUNCH_CHECK();
    LAGR_TRY(fetch_to_host(h, cnt.p, sizeof(h), s, msg));
    const int64_t ncand = h[BC_NCAND];
    // Pull when it reads fewer edges than the push by a margin: the pull walks every edge of the
    // vertices some source has not reached (mu) with a few float64 sums per chunk, the push every
    // out-edge of the frontier (mf) with an atomic per new (vertex, source) pair.  (Beamer's rule,
    // mf > mu / 14 with its hysteresis, chose pulls that measured slower than the push on R-MAT:
    // 13.1 vs 12.0 ms for 4 sources at scale 22, 169 vs 118 ms for 64.)  Past 8 sources the pull
    // reduces per 32 edges and per source and loses to the push (123 vs 118 ms for 64): push only.
    pull = ns <= 8 && ncand > 0 && BC_PULL_MARGIN * h[BC_MU] < h[BC_MF];
    if (pull) {
      bc_scatter_masks<<<grid_for(nent, BC_THREADS), BC_THREADS, 0, s>>>(lv.p + s0, lm.p + s0, (int32_t)nent,
                                                                        dmask.p);
      LAGR_TRY(fx_plan(&fx, cand.p, (int32_t)ncand, G->at_rowptr, s, msg));
      if (ns <= 4)
        bc_fwd_pull<4><<<fgrid4, BC_THREADS, 0, s>>>(G->at_rowptr, G->at_colidx, ns, full, cand.p, (int32_t)ncand,
                                                     fx.off, seen.p, dmask.p, nmask.p, sigma.p, lv.p + start[d + 1],
                                                     cnt.p);
      else if (ns <= 8)
        bc_fwd_pull<8><<<fgrid8, BC_THREADS, 0, s>>>(G->at_rowptr, G->at_colidx, ns, full, cand.p, (int32_t)ncand,
                                                     fx.off, seen.p, dmask.p, nmask.p, sigma.p, lv.p + start[d + 1],
                                                     cnt.p);
      else
        bc_fwd_pull<0><<<fgrid0, BC_THREADS, 0, s>>>(G->at_rowptr, G->at_colidx, ns, full, cand.p, (int32_t)ncand,
                                                     fx.off, seen.p, dmask.p, nmask.p, sigma.p, lv.p + start[d + 1],
                                                     cnt.p);
      bc_clear_masks<<<grid_for(nent, BC_THREADS), BC_THREADS, 0, s>>>(lv.p + s0, (int32_t)nent, dmask.p);
      pulls++;
    } else {
      pushes++;
      LAGR_TRY(fx_plan(&fx, lv.p + s0, (int32_t)nent, G->rowptr, s, msg));
      bc_push<<<grid, BC_THREADS, 0, s>>>(G->rowptr, G->colidx, ns, lv.p + s0, lm.p + s0, (int32_t)nent, fx.off,
                                          seen.p, nmask.p, sigma.p, lv.p + start[d + 1], cnt.p);
    }
    LAGR_LAUNCH_CHECK();
    LAGR_TRY(fetch_to_host(h, cnt.p, sizeof(h), s, msg));
    const int64_t nn = h[BC_NNEXT];
    if (nn == 0) break;
    bc_push_finish<<<grid_for(nn, BC_THREADS), BC_THREADS, 0, s>>>(lv.p + start[d + 1], (int32_t)nn, nmask.p,
                                                                  lm.p + start[d + 1], seen.p);
    LAGR_LAUNCH_CHECK();
    start.push_back(start[d + 1] + nn);
  }
  const int32_t D = (int32_t)start.size() - 2;  // the deepest level (level 0: the sources)
  // backtrack: level d into level d - 1, from the deepest level up to level 2 -> 1
  for (int32_t d = D; d >= 2; d--) {
    const int64_t sd = start[d], nd = start[d + 1] - start[d];
    const int64_t su = start[d - 1], nu = start[d] - start[d - 1];
    bc_level_w<<<grid_for(nd, BC_THREADS), BC_THREADS, 0, s>>>(ns, lv.p + sd, lm.p + sd, (int32_t)nd, B.p,
                                                               sigma.p, W.p, dmask.p);
    LAGR_TRY(fx_plan(&fx, lv.p + su, (int32_t)nu, G->rowptr, s, msg));
    if (ns <= 4)
      bc_pull_few<4><<<pgrid4, BC_THREADS, 0, s>>>(G->rowptr, G->colidx, ns, lv.p + su, lm.p + su, (int32_t)nu,
                                                   fx.off, dmask.p, W.p, acc.p);
    else if (ns <= 8)
      bc_pull_few<8><<<pgrid8, BC_THREADS, 0, s>>>(G->rowptr, G->colidx, ns, lv.p + su, lm.p + su, (int32_t)nu,
                                                   fx.off, dmask.p, W.p, acc.p);
    else
      bc_pull<<<pgrid, BC_THREADS, 0, s>>>(G->rowptr, G->colidx, ns, lv.p + su, lm.p + su, (int32_t)nu, fx.off,
                                           dmask.p, W.p, acc.p);
    bc_level_apply<<<grid_for(nu, BC_THREADS), BC_THREADS, 0, s>>>(ns, lv.p + su, lm.p + su, (int32_t)nu, sigma.p,
                                                                   acc.p, B.p);
    bc_clear_masks<<<grid_for(nd, BC_THREADS), BC_THREADS, 0, s>>>(lv.p + sd, (int32_t)nd, dmask.p);
    LAGR_LAUNCH_CHECK();
  }
  bc_reduce<<<grid_for(n, BC_THREADS), BC_THREADS, 0, s>>>(n, ns, B.p, centrality);
  LAGR_LAUNCH_CHECK();
  LAGR_CUDA_TRY(cudaStreamSynchronize(s));
  if (levels) *levels = D;
  G->last_levels = D + 1;
  G->last_pull_levels = pulls;
  G->last_push_levels = pushes;
  clear_msg(msg);
  return LAGR_OK;
}
