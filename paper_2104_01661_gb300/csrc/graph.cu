// The graph object and its cached properties (Sec. II-A), the allocator hook and the message
// convention (Sec. II-D), CheckGraph / Property_AT / Property_RowDegree (Sec. V utilities).
#include <cstdlib>
#include <cstring>

#include <atomic>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace lagr {

// ---- messages ---------------------------------------------------------------------------------

void set_msg(char *msg, const char *fmt, ...) {
  if (!msg) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, LAGR_MSG_LEN, fmt, ap);
  va_end(ap);
}

// ---- launch counter -------------------------------------------------------------------------------
// The library is linked with --wrap=__cudaLaunchKernel, so every <<<...>>> launch in these files
// passes through here first (the runtime entry point is declared in CUDA's crt headers).

static unsigned long long g_launches = 0;

void note_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }

}  // namespace lagr

extern "C" cudaError_t __real___cudaLaunchKernel(cudaKernel_t kernel, dim3 grid, dim3 block, void **args,
                                                 size_t smem, cudaStream_t stream);
extern "C" cudaError_t __wrap___cudaLaunchKernel(cudaKernel_t kernel, dim3 grid, dim3 block, void **args,
                                                 size_t smem, cudaStream_t stream) {
  __atomic_fetch_add(&lagr::g_launches, 1ull, __ATOMIC_RELAXED);
  return __real___cudaLaunchKernel(kernel, grid, block, args, smem, stream);
}

namespace lagr {

// ---- launch geometry -----------------------------------------------------------------------------

constexpr int GEOM_DEVICES = 64;
static std::atomic<int> g_nsm[GEOM_DEVICES];

int sm_count() {
  int d = 0, nsm = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    d = -1;
  }
  if (d >= 0 && d < GEOM_DEVICES && (nsm = g_nsm[d].load(std::memory_order_relaxed)) > 0) return nsm;
  if (d < 0 || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    return 1;  // no device answered: a one-CTA-per-wave grid is still a valid grid
  }
  if (d < GEOM_DEVICES) g_nsm[d].store(nsm, std::memory_order_relaxed);
  return nsm;
}

static std::mutex g_occ_mu;
struct OccKey {
  const void *k;
  int threads, dev;
  size_t smem;
  int ctas;
};
static std::vector<OccKey> g_occ;

int resident_ctas(const void *kernel, int threads, size_t smem) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (const OccKey &o : g_occ)
      if (o.k == kernel && o.threads == threads && o.smem == smem && o.dev == d) return o.ctas;
  }
  const int nsm = sm_count();
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int ctas = per_sm * nsm;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ.push_back(OccKey{kernel, threads, d, smem, ctas});
  return ctas;
}

int grid_for(int64_t work, int threads, int waves) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)waves * sm_count();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---- allocator hook -----------------------------------------------------------------------------

static lagr_alloc_fn g_alloc = nullptr;
static lagr_free_fn g_free = nullptr;
static void *g_ctx = nullptr;

// The default allocator takes device memory from a pool of the library's own (one per device) that
// keeps what is freed instead of handing it back at the next synchronisation, as a pool with the
// default release threshold does: the entry points synchronise often (BFS levels, PageRank checks),
// and re-mapping the work space of every call would cost more than the work on small graphs.
// lagr_release_memory trims the pools.
constexpr int MAX_DEVICES = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[MAX_DEVICES] = {};

static cudaMemPool_t lib_pool() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[d]) {
    cudaMemPoolProps pr;
    memset(&pr, 0, sizeof(pr));
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = d;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    g_pool[d] = pool;
  }
  return g_pool[d];
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc) return g_alloc(bytes, (void *)s, g_ctx);
  void *p = nullptr;
  cudaMemPool_t pool = lib_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of a failed allocation
    return nullptr;
  }
  return p;
}

// Pinned host mirrors of the device scalars (LAGR_NHOST int64 each, with their device-mapped
// addresses), recycled between graphs and calls: allocating and freeing pinned memory per graph
// costs a device-wide synchronisation in the free.
static std::mutex g_host_mu;
static std::vector<HostBlock> g_host_free;

bool host_block_get(HostBlock *b) {
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    if (!g_host_free.empty()) {
      *b = g_host_free.back();
      g_host_free.pop_back();
      return true;
    }
  }
  int64_t *h = nullptr;
  void *d = nullptr;
  if (cudaHostAlloc((void **)&h, LAGR_NHOST * sizeof(int64_t), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    return false;
  }
  *b = HostBlock{h, (int64_t *)d};
  return true;
}

void host_block_put(HostBlock b) {
  std::lock_guard<std::mutex> lk(g_host_mu);
  g_host_free.push_back(b);
}

struct FetchList {
  const int32_t *p[8];
};

__global__ void fetch_words_kernel(const uint32_t *__restrict__ src, int nwords, uint32_t *dst) {
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = src[i];
}

__global__ void fetch_list_kernel(FetchList l, int count, int32_t *dst) {
  if ((int)threadIdx.x < count) dst[threadIdx.x] = *l.p[threadIdx.x];
}

int fetch_to_host(void *dst, const void *dsrc, size_t bytes, cudaStream_t s, char *msg) {
  if (bytes % 4 != 0 || bytes > LAGR_NHOST * sizeof(int64_t)) {
    set_msg(msg, "internal: fetch of %zu bytes", bytes);
    return LAGR_ERR_INVALID_VALUE;
  }
  HostBlock b;
  if (!host_block_get(&b)) {
    set_msg(msg, "out of pinned host memory");
    return LAGR_ERR_OUT_OF_MEMORY;
  }
  fetch_words_kernel<<<1, 32, 0, s>>>((const uint32_t *)dsrc, (int)(bytes / 4), (uint32_t *)b.d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_msg(msg, "CUDA error: %s", cudaGetErrorString(e));
    return LAGR_ERR_CUDA;  // the block may still be written: it is not recycled
  }
  memcpy(dst, b.h, bytes);
  host_block_put(b);
  return LAGR_OK;
}

int fetch_i32s(int32_t *dst, const int32_t *const *srcs, int count, cudaStream_t s, char *msg) {
  if (count < 1 || count > 8) {
    set_msg(msg, "internal: fetch of %d scalars", count);
    return LAGR_ERR_INVALID_VALUE;
  }
  HostBlock b;
  if (!host_block_get(&b)) {
    set_msg(msg, "out of pinned host memory");
    return LAGR_ERR_OUT_OF_MEMORY;
  }
  FetchList l;
  for (int i = 0; i < 8; i++) l.p[i] = i < count ? srcs[i] : nullptr;
  fetch_list_kernel<<<1, 32, 0, s>>>(l, count, (int32_t *)b.d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_msg(msg, "CUDA error: %s", cudaGetErrorString(e));
    return LAGR_ERR_CUDA;
  }
  memcpy(dst, b.h, (size_t)count * sizeof(int32_t));
  host_block_put(b);
  return LAGR_OK;
}

void dev_free(void *p, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, (void *)s, g_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// ---- private state ------------------------------------------------------------------------------

int priv_get(lagr_graph G, cudaStream_t s, char *msg, Priv **out) {
  Priv *P = static_cast<Priv *>(G->priv);
  if (!P) {
    P = new Priv();
    G->priv = P;
  }
  if (!P->dscal) {
    LAGR_TRY(alloc_n(&P->dscal, LAGR_NSCAL, s, msg, "device scalars"));
    LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal, 0, LAGR_NSCAL * sizeof(int64_t), s));
  }
  if (!P->hscal) {
    HostBlock b;
    if (!host_block_get(&b)) {
      set_msg(msg, "out of pinned host memory (%d bytes)", (int)(LAGR_NHOST * sizeof(int64_t)));
      return LAGR_ERR_OUT_OF_MEMORY;
    }
    P->hscal = b.h;
    P->hscal_dev = b.d;
  }
  *out = P;
  return LAGR_OK;
}

static void free_tc_cache(Priv *P, cudaStream_t s) {
  dev_free(P->tc_listw, s);
  dev_free(P->tc_listwh, s);
  dev_free(P->tc_listc, s);
  dev_free(P->tc_rank, s);
  dev_free(P->tc_sortbuf, s);
  dev_free(P->tc_radix, s);
  dev_free(P->tc_radix_scan, s);
  P->tc_listwh = nullptr;
  P->tc_capwh = 0;
  P->tc_rank = P->tc_sortbuf = P->tc_radix = nullptr;
  P->tc_radix_scan = nullptr;
  P->tc_listw = nullptr;
  P->tc_listc = nullptr;
  P->tc_capc = 0;
}

void priv_release(lagr_graph G, cudaStream_t s) {
  Priv *P = static_cast<Priv *>(G->priv);
  if (!P) return;
  free_tc_cache(P, s);
  for (RowPlan *rp : {&P->pr_at, &P->pr_a, &P->pr_fwd, &P->pr_adj}) {
    dev_free(rp->blk, s);
    dev_free(rp->heavy, s);
    dev_free(rp->hc_off, s);
    dev_free(rp->hc_row, s);
    dev_free(rp->hblk, s);
  }
  dev_free(P->dscal, s);
  if (P->hscal) {
    // every reader of hscal synchronises first; this covers a call that returned early
    if (cudaStreamSynchronize(s) == cudaSuccess) host_block_put(HostBlock{P->hscal, P->hscal_dev});
    else cudaGetLastError();
  }
  delete P;
  G->priv = nullptr;
}

int check_graph_arg(lagr_graph G, char *msg) {
  if (!G) {
    set_msg(msg, "graph is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  if (G->n > 0 && !G->rowptr) {
    set_msg(msg, "graph has no row pointers");
    return LAGR_ERR_NULL_POINTER;
  }
  if (G->nnz > 0 && !G->colidx) {
    set_msg(msg, "graph has no column indices");
    return LAGR_ERR_NULL_POINTER;
  }
  return LAGR_OK;
}

// ---- CheckGraph kernels -----------------------------------------------------------------------

namespace {

enum CheckBits {
  BAD_ROWPTR0 = 1,
  BAD_MONOTONE = 2,
  BAD_LAST = 4,
  BAD_RANGE = 8,
  BAD_ORDER = 16,
  BAD_SYMMETRY = 32
};

__global__ void check_rowptr(const int32_t *__restrict__ rowptr, int32_t n, int64_t nnz, int64_t *__restrict__ flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (rowptr[i + 1] < rowptr[i]) atomicOr((unsigned long long *)&flags[0], BAD_MONOTONE);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rowptr[0] != 0) atomicOr((unsigned long long *)&flags[0], BAD_ROWPTR0);
    if ((int64_t)rowptr[n] != nnz) atomicOr((unsigned long long *)&flags[0], BAD_LAST);
  }
}

// one warp per row: range, strict order, self-loop count
__global__ void check_rows(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int32_t n,
                           int64_t *__restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bad = 0, diag = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    for (int32_t k = b + lane; k < e; k += 32) {
      const int32_t j = colidx[k];
      if (j < 0 || j >= n) bad |= BAD_RANGE;
      if (k + 1 < e && colidx[k + 1] <= j) bad |= BAD_ORDER;
      if (j == i) diag++;
    }
  }
  if (bad) atomicOr((unsigned long long *)&flags[0], bad);
  diag = warp_sum(diag);
  if (lane == 0 && diag) atomicAdd((unsigned long long *)&flags[1], diag);
}

__global__ void compare_arrays(const int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t len,
                               int64_t *__restrict__ flags) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x)
    if (a[k] != b[k]) {
      atomicOr((unsigned long long *)&flags[0], BAD_SYMMETRY);
      return;
    }
}

__global__ void row_degree_kernel(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    deg[i] = rowptr[i + 1] - rowptr[i];
}

}  // namespace

}  // namespace lagr

using namespace lagr;

// ---- opt-in kernel timing -----------------------------------------------------------------------

namespace lagr {
static const char *const kTimedNames[TK_COUNT] = {"pr_gather",      "tc_count_cta", "tc_count_warp",
                                                  "bfs_push_small", "bfs_push_lb",  "bfs_pull"};
struct TimedPair {
  int k;
  cudaEvent_t a, b;
};
static std::mutex g_tmu;
static int g_timing = 0;
static std::vector<TimedPair> g_pending;
static double g_tms[TK_COUNT];
static int64_t g_tcount[TK_COUNT];

KTimer::KTimer(TimedKernel k_, cudaStream_t s_) : k(k_), s(s_) {
  if (!__atomic_load_n(&g_timing, __ATOMIC_RELAXED)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
      cudaEventRecord(a, s) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    a = b = nullptr;
  }
}

KTimer::~KTimer() {
  if (!a) return;
  if (cudaEventRecord(b, s) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return;
  }
  std::lock_guard<std::mutex> lk(g_tmu);
  g_pending.push_back(TimedPair{(int)k, a, b});
}

// fold the recorded pairs into the totals (waits for them)
static int timing_collect() {
  std::lock_guard<std::mutex> lk(g_tmu);
  int rc = LAGR_OK;
  for (const TimedPair &p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_tms[p.k] += ms;
      g_tcount[p.k] += 1;
    } else {
      cudaGetLastError();
      rc = LAGR_ERR_CUDA;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
  return rc;
}
}  // namespace lagr

extern "C" {

const char *lagr_version(void) { return "lagr-gb300 0.1 (sm_103a)"; }

uint64_t lagr_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }


int lagr_timing_enable(int on) {
  __atomic_store_n(&lagr::g_timing, on ? 1 : 0, __ATOMIC_RELAXED);
  return LAGR_OK;
}

int lagr_timing_reset(void) {
  const int rc = lagr::timing_collect();
  std::lock_guard<std::mutex> lk(lagr::g_tmu);
  for (int k = 0; k < lagr::TK_COUNT; k++) {
    lagr::g_tms[k] = 0.0;
    lagr::g_tcount[k] = 0;
  }
  return rc;
}

int lagr_timing_read(const char *kernel, double *ms, int64_t *launches) {
  if (!kernel || !ms || !launches) return LAGR_ERR_NULL_POINTER;
  int k = 0;
  while (k < lagr::TK_COUNT && strcmp(kernel, lagr::kTimedNames[k]) != 0) k++;
  if (k == lagr::TK_COUNT) return LAGR_ERR_INVALID_VALUE;
  const int rc = lagr::timing_collect();
  std::lock_guard<std::mutex> lk(lagr::g_tmu);
  *ms = lagr::g_tms[k];
  *launches = lagr::g_tcount[k];
  return rc;
}

int lagr_set_allocator(lagr_alloc_fn alloc, lagr_free_fn free_, void *ctx) {
  if ((alloc == nullptr) != (free_ == nullptr)) return LAGR_ERR_NULL_POINTER;
  g_alloc = alloc;
  g_free = free_;
  g_ctx = ctx;
  return LAGR_OK;
}

int lagr_release_memory(uint64_t keep_bytes, char *msg) {
  set_msg(msg, "");
  int rc = LAGR_OK;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < MAX_DEVICES; d++)
      if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], (size_t)keep_bytes) != cudaSuccess) {
        set_msg(msg, "cudaMemPoolTrimTo failed on device %d: %s", d, cudaGetErrorString(cudaGetLastError()));
        rc = LAGR_ERR_CUDA;
      }
  }
  std::vector<HostBlock> held;
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    held.swap(g_host_free);
  }
  for (const HostBlock &b : held) cudaFreeHost(b.h);
  return rc;
}

int lagr_graph_new(lagr_graph *G, int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                   const float *val, int32_t kind, char *msg) {
  if (!G) {
    set_msg(msg, "G is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  *G = nullptr;
  if (n < 0 || nnz < 0) {
    set_msg(msg, "negative size (n=%d, nnz=%lld)", n, (long long)nnz);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (nnz >= ((int64_t)1 << 31) || n == INT32_MAX) {
    set_msg(msg, "graph too large for int32 indices (n=%d, nnz=%lld)", n, (long long)nnz);
    return LAGR_ERR_TOO_LARGE;
  }
  if (kind != LAGR_UNDIRECTED && kind != LAGR_DIRECTED) {
    set_msg(msg, "unknown graph kind %d", kind);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (!rowptr || (nnz > 0 && !colidx)) {
    set_msg(msg, "rowptr/colidx is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  lagr_graph g = static_cast<lagr_graph>(calloc(1, sizeof(lagr_graph_struct)));
  if (!g) {
    set_msg(msg, "out of host memory");
    return LAGR_ERR_OUT_OF_MEMORY;
  }
  g->n = n;
  g->nnz = nnz;
  g->kind = kind;
  g->rowptr = rowptr;
  g->colidx = colidx;
  g->val = val;
  g->a_pattern_is_symmetric = (kind == LAGR_UNDIRECTED) ? 1 : -1;
  g->ndiag = -1;
  g->u_order = -1;
  g->last_levels = g->last_push_levels = g->last_pull_levels = g->last_iters = -1;
  g->last_resid = -1.0;
  *G = g;
  clear_msg(msg);
  return LAGR_OK;
}

int lagr_delete_properties(lagr_graph G, void *stream, char *msg) {
  if (!G) {
    set_msg(msg, "graph is NULL");
    return LAGR_ERR_NULL_POINTER;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (G->at_owned) {
    dev_free(G->at_rowptr, s);
    dev_free(G->at_colidx, s);
    dev_free(G->at_val, s);
  }
  G->at_rowptr = G->at_colidx = nullptr;
  G->at_val = nullptr;
  G->at_owned = 0;
  dev_free(G->row_degree, s);
  G->row_degree = nullptr;
  dev_free(G->u_dplus, s);
  dev_free(G->u_colidx, s);
  G->u_dplus = G->u_colidx = nullptr;
  G->u_order = -1;
  G->ndiag = -1;
  priv_release(G, s);
  clear_msg(msg);
  return LAGR_OK;
}

int lagr_graph_free(lagr_graph *G, void *stream, char *msg) {
  if (!G || !*G) {
    clear_msg(msg);
    return LAGR_OK;
  }
  int st = lagr_delete_properties(*G, stream, msg);
  free(*G);
  *G = nullptr;
  return st;
}

int lagr_property_row_degree(lagr_graph G, void *stream, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  cudaStream_t s = (cudaStream_t)stream;
  if (!G->row_degree) {
    int32_t *d = nullptr;
    LAGR_TRY(alloc_n(&d, (size_t)G->n + 1, s, msg, "row degree"));
    if (G->n > 0) row_degree_kernel<<<grid_for(G->n, 256), 256, 0, s>>>(G->rowptr, G->n, d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      dev_free(d, s);
      set_msg(msg, "row degree: %s", cudaGetErrorString(e));
      return LAGR_ERR_CUDA;
    }
    G->row_degree = d;
  }
  clear_msg(msg);
  return LAGR_OK;
}

int lagr_property_AT(lagr_graph G, void *stream, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  cudaStream_t s = (cudaStream_t)stream;
  if (G->at_rowptr) {
    clear_msg(msg);
    return LAGR_OK;
  }
  if (G->kind == LAGR_UNDIRECTED) {
    G->at_rowptr = const_cast<int32_t *>(G->rowptr);
    G->at_colidx = const_cast<int32_t *>(G->colidx);
    G->at_val = const_cast<float *>(G->val);
    G->at_owned = 0;
    clear_msg(msg);
    return LAGR_OK;
  }
  int32_t *rp = nullptr, *ci = nullptr;
  float *v = nullptr;
  int st = alloc_n(&rp, (size_t)G->n + 1, s, msg, "A' row pointers");
  if (st == LAGR_OK) st = alloc_n(&ci, (size_t)G->nnz, s, msg, "A' column indices");
  if (st == LAGR_OK && G->val) st = alloc_n(&v, (size_t)G->nnz, s, msg, "A' values");
  if (st == LAGR_OK) st = transpose_csr(G->n, G->nnz, G->rowptr, G->colidx, G->val, rp, ci, v, s, msg);
  if (st < 0) {
    dev_free(rp, s);
    dev_free(ci, s);
    dev_free(v, s);
    return st;
  }
  G->at_rowptr = rp;
  G->at_colidx = ci;
  G->at_val = v;
  G->at_owned = 1;
  clear_msg(msg);
  return LAGR_OK;
}

int lagr_graph_check(lagr_graph G, void *stream, char *msg) {
  LAGR_TRY(check_graph_arg(G, msg));
  cudaStream_t s = (cudaStream_t)stream;
  Priv *P = nullptr;
  LAGR_TRY(priv_get(G, s, msg, &P));
  const int32_t n = G->n;
  LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal, 0, 2 * sizeof(int64_t), s));
  check_rowptr<<<grid_for(n, 256), 256, 0, s>>>(G->rowptr, n, G->nnz, P->dscal);
  LAGR_LAUNCH_CHECK();
  LAGR_TRY(fetch_to_host(P->hscal, P->dscal, 2 * sizeof(int64_t), s, msg));
  int64_t bad = P->hscal[0];
  if (bad) {
    set_msg(msg, "invalid row pointers:%s%s%s", (bad & BAD_ROWPTR0) ? " rowptr[0] != 0" : "",
            (bad & BAD_MONOTONE) ? " decreasing" : "", (bad & BAD_LAST) ? " rowptr[n] != nnz" : "");
    return LAGR_ERR_INVALID_GRAPH;
  }
  if (n > 0) check_rows<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(G->rowptr, G->colidx, n, P->dscal);
  LAGR_LAUNCH_CHECK();
  LAGR_TRY(fetch_to_host(P->hscal, P->dscal, 2 * sizeof(int64_t), s, msg));
  bad = P->hscal[0];
  G->ndiag = P->hscal[1];
  if (bad) {
    set_msg(msg, "invalid column indices:%s%s", (bad & BAD_RANGE) ? " out of range" : "",
            (bad & BAD_ORDER) ? " row not strictly increasing (unsorted or duplicate)" : "");
    return LAGR_ERR_INVALID_GRAPH;
  }
  // symmetry: A == A' entry for entry (both have sorted rows)
  {
    Temp<int32_t> rp(s), ci(s);
    LAGR_TRY(rp.alloc((size_t)n + 1, msg, "check transpose"));
    LAGR_TRY(ci.alloc((size_t)G->nnz, msg, "check transpose"));
    LAGR_TRY(transpose_csr(n, G->nnz, G->rowptr, G->colidx, nullptr, rp.p, ci.p, nullptr, s, msg));
    LAGR_CUDA_TRY(cudaMemsetAsync(P->dscal, 0, sizeof(int64_t), s));
    compare_arrays<<<grid_for(n + 1, 256), 256, 0, s>>>(G->rowptr, rp.p, (int64_t)n + 1, P->dscal);
    if (G->nnz > 0) compare_arrays<<<grid_for(G->nnz, 256), 256, 0, s>>>(G->colidx, ci.p, G->nnz, P->dscal);
    LAGR_LAUNCH_CHECK();
    LAGR_TRY(fetch_to_host(P->hscal, P->dscal, sizeof(int64_t), s, msg));
  }
  const int symmetric = P->hscal[0] == 0;
  G->a_pattern_is_symmetric = symmetric;
  if (G->kind == LAGR_UNDIRECTED && !symmetric) {
    set_msg(msg, "graph is marked undirected but A != A'");
    return LAGR_ERR_INVALID_GRAPH;
  }
  clear_msg(msg);
  return LAGR_OK;
}

}  // extern "C"
