/*
 * Seeded synthetic graph generators.
 *
 * These produce the INPUTS of the masked semiring products (R-MAT stand-ins
 * for the Kronecker graphs of the paper's Table IV, Erdos-Renyi stand-ins for
 * its uniform-random graph, and a 2D 4-neighbour grid for its high-diameter
 * road graph).  They hold none of the method's arithmetic: no triangle
 * counting, no traversal, no ranking.  Both the CUDA path's tests/benchmarks
 * and the CPU oracle consume what these functions emit.
 *
 * Random numbers: splitmix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used in counter mode: draw k
 * of a stream with seed s is mix(s + (k+1) * GAMMA).  Every draw is therefore
 * addressable without replaying the stream, so results are identical however
 * the work is split.
 *
 * Output format: CSR with int32 row pointers and int32 column indices, rows
 * sorted ascending, no duplicate entries.  Self-loops are removed when asked.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* k-th draw of the counter-mode stream `seed`. */
static inline uint64_t draw(uint64_t seed, uint64_t k) { return mix64(seed + (k + 1) * GAMMA); }

/* uniform double in [0, 1) from the top 53 bits */
static inline double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

uint64_t gen_splitmix64_draw(uint64_t seed, uint64_t k) { return draw(seed, k); }

/*
 * R-MAT edge list (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of the
 * `nedges` edges descends `scale` levels of the adjacency matrix, picking the
 * quadrant (0,0) with probability a, (0,1) with b, (1,0) with c, (1,1) with
 * d = 1-a-b-c.  No noise and no label scrambling, so vertex 0 is the top hub.
 * Level l of edge e uses draw e*scale + l of the stream.
 */
void gen_rmat_edges(int scale, int64_t nedges, double a, double b, double c, uint64_t seed,
                    int32_t *src, int32_t *dst) {
  const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nedges; e++) {
    uint32_t r = 0, q = 0;
    for (int l = 0; l < scale; l++) {
      double u = unit(draw(seed, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
      uint32_t rb, cb;
      if (u < a) { rb = 0; cb = 0; }
      else if (u < ab) { rb = 0; cb = 1; }
      else if (u < abc) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      r = (r << 1) | rb;
      q = (q << 1) | cb;
    }
    src[e] = (int32_t)r;
    dst[e] = (int32_t)q;
  }
}

/* uniform integer in [0, n) by multiply-shift on the top 32 bits (n < 2^32) */
static inline uint32_t below(uint64_t x, uint32_t n) { return (uint32_t)(((x >> 32) * (uint64_t)n) >> 32); }

/* Erdos-Renyi style edge list: both endpoints uniform in [0, n). */
void gen_uniform_edges(int32_t n, int64_t nedges, uint64_t seed, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nedges; e++) {
    src[e] = (int32_t)below(draw(seed, 2 * (uint64_t)e), (uint32_t)n);
    dst[e] = (int32_t)below(draw(seed, 2 * (uint64_t)e + 1), (uint32_t)n);
  }
}

static void isort(int32_t *x, int64_t len) {
  for (int64_t i = 1; i < len; i++) {
    int32_t v = x[i];
    int64_t j = i - 1;
    while (j >= 0 && x[j] > v) { x[j + 1] = x[j]; j--; }
    x[j + 1] = v;
  }
}

static int cmp_i32(const void *p, const void *q) {
  int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
  return (a > b) - (a < b);
}

/*
 * Edge list -> CSR.  symmetric != 0 also inserts (dst,src) for every edge;
 * drop_self != 0 removes (v,v).  Rows are sorted and duplicates removed, so
 * the result does not depend on the order in which entries were scattered.
 * rowptr has n+1 entries; colidx must hold (symmetric ? 2 : 1) * nedges
 * entries.  Returns the number of stored entries (<= that capacity), or -1
 * when an endpoint is out of range or the count does not fit int32.
 */
int64_t gen_edges_to_csr(int32_t n, int64_t nedges, const int32_t *src, const int32_t *dst,
                         int symmetric, int drop_self, int32_t *rowptr, int32_t *colidx) {
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
  for (int64_t e = 0; e < nedges; e++) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) { bad = 1; continue; }
    if (drop_self && u == v) continue;
#pragma omp atomic
    cnt[u + 1]++;
    if (symmetric && u != v) {
#pragma omp atomic
      cnt[v + 1]++;
    }
  }
  if (bad) { free(cnt); return -1; }
  for (int32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
  if (cnt[n] > INT32_MAX) { free(cnt); return -1; }
  int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!pos) { free(cnt); return -1; }
  memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nedges; e++) {
    int32_t u = src[e], v = dst[e];
    if (drop_self && u == v) continue;
    int64_t k;
#pragma omp atomic capture
    k = pos[u]++;
    colidx[k] = v;
    if (symmetric && u != v) {
#pragma omp atomic capture
      k = pos[v]++;
      colidx[k] = u;
    }
  }
  free(pos);
  /* sort each row and squeeze out duplicates in place; row i keeps its slot */
  int64_t *kept = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!kept) { free(cnt); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t i = 0; i < n; i++) {
    int64_t b = cnt[i], len = cnt[i + 1] - b;
    int32_t *row = colidx + b;
    if (len < 32) isort(row, len); else qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t out = 0;
    for (int64_t k = 0; k < len; k++) {
      if (out > 0 && row[out - 1] == row[k]) continue;
      row[out++] = row[k];
    }
    kept[i] = out;
  }
  /* compact rows to the front (serial: rows only move left) */
  int64_t out = 0;
  rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int64_t b = cnt[i];
    if (out != b) memmove(colidx + out, colidx + b, (size_t)kept[i] * sizeof(int32_t));
    out += kept[i];
    rowptr[i + 1] = (int32_t)out;
  }
  free(kept);
  free(cnt);
  return out;
}

/* rows x cols grid, vertex id r*cols + c, edges to the 4 neighbours (sorted). */
int64_t gen_grid_csr(int32_t rows, int32_t cols, int32_t *rowptr, int32_t *colidx) {
  int64_t k = 0;
  rowptr[0] = 0;
  for (int32_t r = 0; r < rows; r++) {
    for (int32_t c = 0; c < cols; c++) {
      int64_t v = (int64_t)r * cols + c;
      if (r > 0) colidx[k++] = (int32_t)(v - cols);
      if (c > 0) colidx[k++] = (int32_t)(v - 1);
      if (c + 1 < cols) colidx[k++] = (int32_t)(v + 1);
      if (r + 1 < rows) colidx[k++] = (int32_t)(v + cols);
      rowptr[v + 1] = (int32_t)k;
    }
  }
  return k;
}

/* count values in (0, 1]: 1 - u with u uniform in [0, 1) */
void gen_uniform_open0(int64_t count, uint64_t seed, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; i++) out[i] = 1.0 - unit(draw(seed, (uint64_t)i));
}

/* standard normals by Box-Muller on pairs of draws (2i, 2i+1) */
void gen_normal(int64_t count, uint64_t seed, double *out) {
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; i++) {
    double u1 = 1.0 - unit(draw(seed, 2 * (uint64_t)i));   /* (0, 1] so log is finite */
    double u2 = unit(draw(seed, 2 * (uint64_t)i + 1));
    out[i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
  }
}

/*
 * k distinct vertices uniform in [0, n) with at least one stored entry in
 * their row, by rejection.  Returns the number found (< k only if the graph
 * has fewer than k such vertices or the draws run out).
 */
int32_t gen_sources(int32_t n, const int32_t *rowptr, int32_t k, uint64_t seed, int32_t *out) {
  int32_t found = 0;
  for (uint64_t t = 0; found < k && t < (uint64_t)64 * (uint64_t)n + 1024; t++) {
    int32_t v = (int32_t)below(draw(seed, t), (uint32_t)n);
    if (rowptr[v + 1] == rowptr[v]) continue;
    int dup = 0;
    for (int32_t j = 0; j < found; j++) if (out[j] == v) { dup = 1; break; }
    if (!dup) out[found++] = v;
  }
  return found;
}

/*
 * Symmetric edge weights uniform in (0, 1], stored as float32: the entry (i, j)
 * of a CSR gets the value of the unordered pair {min(i,j), max(i,j)}, draw
 * min * n + max of the stream, so A(i,j) = A(j,i) on a symmetric pattern.
 */
void gen_pair_weights(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, float *out) {
#pragma omp parallel for schedule(dynamic, 4096)
  for (int32_t i = 0; i < n; i++) {
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
      int32_t j = colidx[e];
      uint64_t a = (uint64_t)(i < j ? i : j), b = (uint64_t)(i < j ? j : i);
      out[e] = (float)(1.0 - unit(draw(seed, a * (uint64_t)n + b)));
    }
  }
}
