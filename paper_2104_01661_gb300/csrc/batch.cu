// Many graphs in one launch.  A batch of g undirected graphs concatenated block-diagonally is one
// graph whose edges never cross members, so the triangle-count kernels and the PageRank iteration
// run over all members at once: triangles are accumulated per member (the member of an anchor
// vertex comes from a binary search of the vertex offsets), and PageRank uses a teleport vector
// that gives every vertex of member i the weight 1/n_i, which is Alg. 4 run on each member.
//
// The plan allocates everything once, autotunes the triangle kernels' work partition (neighbour
// chunk per CTA item and the warp/CTA anchor threshold) by timing candidates with CUDA events,
// caches the choice in a small JSON file keyed by GPU name and batch shape, and captures the whole
// pass -- orientation, anchor classification, counting, `iters` PageRank iterations -- in one
// CUDA graph that lagr_batch_run replays.  This is the paper's per-call overhead lesson (the
// high-diameter road graph, Sec. VI-B) applied to many small graphs: one graph launch instead of
// thousands of calls.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

struct lagr_batch_struct {
  int32_t g = 0, N = 0;
  int64_t nnz = 0;
  float damping = 0.85f;
  int32_t iters = 0;
  lagr_graph G = nullptr;
  lagr::Priv *P = nullptr;
  int32_t *voff = nullptr;  // device [g+1]
  float *vvec = nullptr;    // device [N], 1/n_member
  lagr::PrPlan *pr = nullptr;
  lagr::TcParams prm{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t *cap_ntri = nullptr;
  float *cap_rank = nullptr;
};

namespace lagr {
namespace {

__global__ void batch_teleport(const int32_t *__restrict__ voff, int32_t g, int32_t N, float *__restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = g - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (voff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    v[i] = 1.0f / (float)(voff[lo + 1] - voff[lo]);
  }
}

std::string tune_key(const lagr_batch_struct *B) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|g=%d|N=%d|nnz=%lld", prop.name, B->g, B->N, (long long)B->nnz);
  for (char *c = buf; *c; c++)
    if (*c == '"' || *c == '\\') *c = '_';
  return std::string(buf);
}

// cache format: one JSON object, one entry per line:  "key": {"chunk": C, "wmax": W, "ms": T},
bool tune_lookup(const char *path, const std::string &key, TcParams *out) {
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  const std::string want = "\"" + key + "\"";
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char *p = strstr(line, want.c_str());
    if (!p) continue;
    int chunk = 0, wmax = 0;
    const char *c = strstr(p, "\"chunk\":");
    const char *w = strstr(p, "\"wmax\":");
    if (c && w && sscanf(c, "\"chunk\": %d", &chunk) == 1 && sscanf(w, "\"wmax\": %d", &wmax) == 1 && chunk >= 32 &&
        wmax >= 1) {
      out->chunk = chunk;
      out->wmax = wmax;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_store(const char *path, const std::string &key, TcParams prm, float ms) {
  if (!path) return;
  std::vector<std::string> keep;
  if (FILE *f = fopen(path, "r")) {
    char line[1024];
    const std::string want = "\"" + key + "\"";
    while (fgets(line, sizeof(line), f)) {
      std::string l(line);
      if (l.find("\": {") == std::string::npos || l.find(want) != std::string::npos) continue;
      while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
      keep.push_back(l);
    }
    fclose(f);
  }
  char buf[1024];
  snprintf(buf, sizeof(buf), "\"%s\": {\"chunk\": %d, \"wmax\": %d, \"ms\": %.4f}", key.c_str(), prm.chunk, prm.wmax,
           (double)ms);
  keep.push_back(buf);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fputs("{\n", f);
  for (size_t i = 0; i < keep.size(); i++) fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
  fputs("}\n", f);
  fclose(f);
  rename(tmp.c_str(), path);
}

// time one full triangle pass (orientation + classification + counting) with `prm`
int time_tc(lagr_batch_struct *B, TcParams prm, unsigned long long *counts, cudaStream_t s, float *ms, char *msg) {
  cudaEvent_t e0, e1;
  LAGR_CUDA_TRY(cudaEventCreate(&e0));
  LAGR_CUDA_TRY(cudaEventCreate(&e1));
  int st = tc_launch(B->G, B->P, LAGR_TC_SORT, prm, B->voff, B->g, counts, true, s, msg);  // warm-up
  if (st == LAGR_OK) {
    cudaEventRecord(e0, s);
    st = tc_launch(B->G, B->P, LAGR_TC_SORT, prm, B->voff, B->g, counts, true, s, msg);
    cudaEventRecord(e1, s);
  }
  if (st == LAGR_OK) {
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e != cudaSuccess) {
      set_msg(msg, "autotune timing: %s", cudaGetErrorString(e));
      st = LAGR_ERR_CUDA;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace
}  // namespace lagr

using namespace lagr;

extern "C" {

int lagr_batch_free(lagr_batch *B, void *stream, char *msg) {
  if (!B || !*B) {
    clear_msg(msg);
    return LAGR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  lagr_batch_struct *b = *B;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  pr_plan_destroy(b->pr, s);
  dev_free(b->voff, s);
  dev_free(b->vvec, s);
  int st = lagr_graph_free(&b->G, stream, msg);
  delete b;
  *B = nullptr;
  return st;
}

int lagr_batch_plan(lagr_batch *B, int32_t g, const int32_t *voff, int32_t N, int64_t nnz, const int32_t *rowptr,
                    const int32_t *colidx, float damping, int32_t iters, int32_t tile, const char *tune_cache,
                    void *stream, char *msg) {
  if (!B || !voff || !rowptr || (nnz > 0 && !colidx)) {
    set_msg(msg, "NULL argument");
    return LAGR_ERR_NULL_POINTER;
  }
  *B = nullptr;
  if (g < 1 || N < 1 || nnz < 0 || iters < 0 || tile < 0 || !(damping > 0.0f && damping < 1.0f)) {
    set_msg(msg, "bad batch arguments (g=%d N=%d nnz=%lld iters=%d tile=%d)", g, N, (long long)nnz, iters, tile);
    return LAGR_ERR_INVALID_VALUE;
  }
  if (voff[0] != 0 || voff[g] != N) {
    set_msg(msg, "voff must start at 0 and end at N");
    return LAGR_ERR_INVALID_VALUE;
  }
  for (int32_t i = 0; i < g; i++)
    if (voff[i + 1] <= voff[i]) {
      set_msg(msg, "member %d is empty or voff decreases", i);
      return LAGR_ERR_INVALID_VALUE;
    }
  cudaStream_t s = (cudaStream_t)stream;
  lagr_batch_struct *b = new lagr_batch_struct();
  b->g = g;
  b->N = N;
  b->nnz = nnz;
  b->damping = damping;
  b->iters = iters;
  auto fail = [&](int st) {
    lagr_batch_free(&b, stream, nullptr);
    return st;
  };
  int st = lagr_graph_new(&b->G, N, nnz, rowptr, colidx, nullptr, LAGR_UNDIRECTED, msg);
  if (st < 0) return fail(st);
  st = priv_get(b->G, s, msg, &b->P);
  if (st < 0) return fail(st);
  st = alloc_n(&b->voff, (size_t)g + 1, s, msg, "member offsets");
  if (st < 0) return fail(st);
  st = alloc_n(&b->vvec, (size_t)N, s, msg, "member teleport");
  if (st < 0) return fail(st);
  {
    // stage voff through pinned memory so the copy stays stream-ordered and asynchronous
    int32_t *h = nullptr;
    if (cudaMallocHost(&h, ((size_t)g + 1) * sizeof(int32_t)) != cudaSuccess) {
      set_msg(msg, "pinned staging buffer");
      return fail(LAGR_ERR_OUT_OF_MEMORY);
    }
    memcpy(h, voff, ((size_t)g + 1) * sizeof(int32_t));
    cudaError_t e = cudaMemcpyAsync(b->voff, h, ((size_t)g + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeHost(h);
    if (e != cudaSuccess) {
      set_msg(msg, "member offsets: %s", cudaGetErrorString(e));
      return fail(LAGR_ERR_CUDA);
    }
  }
  batch_teleport<<<8 * sm_count(), 256, 0, s>>>(b->voff, g, N, b->vvec);
  if (cudaGetLastError() != cudaSuccess) {
    set_msg(msg, "batch teleport launch failed");
    return fail(LAGR_ERR_CUDA);
  }
  st = pr_plan_create(&b->pr, b->G, b->P, damping, b->vvec, s, msg);
  if (st < 0) return fail(st);

  // work partition: explicit tile, cached choice, or autotune
  TcParams prm = tc_default_params();
  const std::string key = tune_key(b);
  if (tile > 0) {
    prm.chunk = tile < 32 ? 32 : tile;
  } else if (!tune_lookup(tune_cache, key, &prm)) {
    const int chunks[] = {256, 512, 1024, 2048, 4096};
    const int wmaxes[] = {32, 128, 256};
    // allocate for the candidate with the most CTA items first
    st = tc_alloc(b->G, b->P, TcParams{chunks[0], wmaxes[0]}, s, msg);
    if (st < 0) return fail(st);
    unsigned long long *counts = nullptr;
    st = alloc_n(&counts, (size_t)g, s, msg, "autotune counts");
    if (st < 0) return fail(st);
    float best = 1e30f;
    for (int c : chunks)
      for (int w : wmaxes) {
        float ms = 0.0f;
        st = time_tc(b, TcParams{c, w}, counts, s, &ms, msg);
        if (st < 0) {
          dev_free(counts, s);
          return fail(st);
        }
        if (ms < best) {
          best = ms;
          prm = TcParams{c, w};
        }
      }
    dev_free(counts, s);
    tune_store(tune_cache, key, prm, best);
  }
  st = tc_alloc(b->G, b->P, prm, s, msg);
  if (st < 0) return fail(st);
  b->prm = prm;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_msg(msg, "batch plan synchronisation failed");
    return fail(LAGR_ERR_CUDA);
  }
  *B = b;
  clear_msg(msg);
  return LAGR_OK;
}

int lagr_batch_tile(int32_t *tile, lagr_batch B) {
  if (!tile || !B) return LAGR_ERR_NULL_POINTER;
  *tile = B->prm.chunk;
  return LAGR_OK;
}

int lagr_batch_run(uint64_t *ntri, float *rank, lagr_batch B, void *stream, char *msg) {
  if (!ntri || !rank || !B) {
    set_msg(msg, "NULL argument");
    return LAGR_ERR_NULL_POINTER;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!B->exec || B->cap_ntri != ntri || B->cap_rank != rank) {
    // (re)capture the whole pass with these output buffers
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    cudaStream_t cs = s;
    bool own = false;
    if (cs == nullptr) {  // the legacy stream cannot be captured
      LAGR_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    LAGR_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = tc_launch(B->G, B->P, LAGR_TC_SORT, B->prm, B->voff, B->g, (unsigned long long *)ntri, true, cs, msg);
    if (st == LAGR_OK) st = pr_plan_enqueue(B->pr, rank, B->vvec, B->iters, cs, msg);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (own) cudaStreamDestroy(cs);
    if (st < 0) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) {
      set_msg(msg, "capture of the batch pass failed: %s", cudaGetErrorString(e));
      return LAGR_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      set_msg(msg, "instantiating the batch graph failed: %s", cudaGetErrorString(e));
      return LAGR_ERR_CUDA;
    }
    B->graph = graph;
    B->cap_ntri = ntri;
    B->cap_rank = rank;
  }
  LAGR_CUDA_TRY(cudaGraphLaunch(B->exec, s));
  clear_msg(msg);
  return LAGR_OK;
}

}  // extern "C"
