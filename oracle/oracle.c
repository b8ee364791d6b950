/*
 * ORACLE -- test infrastructure, not part of the product.
 *
 * A plain, slow, single-threaded C99 restatement of what the masked semiring
 * products of LAGraph (Mattson et al., "LAGraph: Linear Algebra, Network
 * Analysis Libraries, and the Study of Graph Algorithms", 2021) compute:
 *
 *   oracle_tc                 Triangle counting, Alg. 6 (Sec. IV-E): optional
 *                             ascending degree sort, L = tril(A,-1),
 *                             U = triu(A,1), C<s(L)> = L plus.pair U',
 *                             t = sum(C).
 *   oracle_bfs                Parents BFS, Alg. 1 (Sec. IV-A): the frontier q
 *                             and parent vector p as sparse vectors, one
 *                             any.secondi vxm per level under the complemented
 *                             structural mask of p, then p<s(q)> = q.
 *   oracle_pagerank           PageRank as specified in GAP, Alg. 4
 *                             (Sec. IV-C), in float64, plus the
 *                             dangling-redistribution variant the paper
 *                             mentions (Graphalytics form).
 *   oracle_pagerank_weighted  the same iteration over plus.times with a
 *                             row-stochastic weight matrix W and a teleport
 *                             vector v.
 *   oracle_pagerank_adjoint   the transposed fixed point of the weighted
 *                             iteration and the edge / teleport gradients of a
 *                             linear loss (implicit differentiation; the paper
 *                             has no adjoint, this follows the derivation
 *                             written beside the function).
 *   oracle_tc_edges           Alg. 6 with C<s(L)> kept: the value of C at
 *                             every stored entry of L.
 *   oracle_fastsv             Connected components, Alg. 7 (Sec. IV-F).
 *   oracle_sssp_delta         Single-source shortest paths, Alg. 5 (Sec.
 *                             IV-D), delta-stepping in float32.
 *   oracle_bc                 Batched betweenness centrality, Alg. 3 (Sec.
 *                             IV-B), float64 path counts and dependencies.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * call this file.  It shares no code with the CUDA library: no headers, no
 * helpers, no tables.  Inputs are host CSR arrays (int32 row pointers and
 * column indices, rows sorted, no duplicates) as emitted by the seeded
 * generators.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <time.h>

/* ------------------------------------------------------------------------- */
/* small helpers                                                             */
/* ------------------------------------------------------------------------- */

static int cmp_int32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* degree pairs (degree, vertex) for the ascending degree sort; ties by vertex */
typedef struct { int64_t deg; int32_t v; } degv;
static int cmp_degv(const void *a, const void *b) {
  const degv *x = (const degv *)a, *y = (const degv *)b;
  if (x->deg != y->deg) return (x->deg > y->deg) - (x->deg < y->deg);
  return (x->v > y->v) - (x->v < y->v);
}

static int cmp_int64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------- */
/* Triangle counting, Alg. 6                                                  */
/* ------------------------------------------------------------------------- */

/*
 * Degree statistics of the first step of Alg. 6.  The paper samples them; the
 * oracle takes the exact mean and the lower-middle median of all n degrees.
 * Returns 1 when mean > 4 * median (the condition under which Alg. 6 sorts).
 */
int oracle_tc_wants_sort(int32_t n, const int32_t *rowptr, double *mean_out, int64_t *median_out) {
  if (n <= 0) { if (mean_out) *mean_out = 0; if (median_out) *median_out = 0; return 0; }
  int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  double sum = 0;
  for (int32_t i = 0; i < n; i++) { deg[i] = rowptr[i + 1] - rowptr[i]; sum += (double)deg[i]; }
  qsort(deg, (size_t)n, sizeof(int64_t), cmp_int64);
  int64_t median = deg[(n - 1) / 2];
  double mean = sum / (double)n;
  free(deg);
  if (mean_out) *mean_out = mean;
  if (median_out) *median_out = median;
  return mean > 4.0 * (double)median;
}

/*
 * method: 0 = as Alg. 6 (sort only when mean > 4*median), 1 = always sort,
 * 2 = never sort.  Returns the number of triangles, or UINT64_MAX on an
 * allocation failure.
 */
uint64_t oracle_tc_sample(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method, int32_t stride,
                          int64_t *l_entries, double *count_seconds);

uint64_t oracle_tc(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method) {
  return oracle_tc_sample(n, rowptr, colidx, method, 1, NULL, NULL);
}

static double now_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/*
 * The same computation restricted to the mask rows i = 0, stride, 2*stride, ... of L (in the
 * possibly degree-sorted labelling): a bounded sample of the work for timing.  stride = 1 is the
 * whole count.  *l_entries receives the number of mask entries (i,j) visited and *count_seconds
 * the time of the masked product alone (either may be NULL).
 */
static uint64_t tc_core(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method, int32_t stride,
                        int64_t *l_entries, double *count_seconds, uint32_t *c_out);

uint64_t oracle_tc_sample(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method, int32_t stride,
                          int64_t *l_entries, double *count_seconds) {
  return tc_core(n, rowptr, colidx, method, stride, l_entries, count_seconds, NULL);
}

/*
 * The same product with C kept (the unfused form of Alg. 6): c_out[e] for every
 * stored entry e = (i,j) of the given CSR is C(p^-1(i), p^-1(j)) -- the value of
 * C<s(L)> = L plus.pair U' at that entry in the relabelled graph -- when the
 * entry lies in L (its row comes after its column in the degree order), and 0
 * otherwise.  The sum of c_out is t, which is returned (UINT64_MAX on an
 * allocation failure).
 */
uint64_t oracle_tc_edges(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method, uint32_t *c_out) {
  return tc_core(n, rowptr, colidx, method, 1, NULL, NULL, c_out);
}

static uint64_t tc_core(int32_t n, const int32_t *rowptr, const int32_t *colidx, int method, int32_t stride,
                        int64_t *l_entries, double *count_seconds, uint32_t *c_out) {
  int64_t nnz = rowptr[n];
  if (stride < 1) stride = 1;
  int sort = (method == 1) || (method == 0 && oracle_tc_wants_sort(n, rowptr, NULL, NULL));

  /* A = A(p,p) when sorting: new vertex i is old vertex p[i] (p is the identity otherwise). */
  int32_t *Ap = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *Ai = (int32_t *)malloc(((size_t)nnz + 1) * sizeof(int32_t));
  int32_t *p = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!Ap || !Ai || !p) { free(Ap); free(Ai); free(p); return UINT64_MAX; }
  for (int32_t i = 0; i < n; i++) p[i] = i;
  if (sort) {
    degv *dv = (degv *)malloc(((size_t)n + 1) * sizeof(degv));
    int32_t *pinv = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) { dv[i].deg = rowptr[i + 1] - rowptr[i]; dv[i].v = i; }
    qsort(dv, (size_t)n, sizeof(degv), cmp_degv);           /* p[i] = dv[i].v */
    for (int32_t i = 0; i < n; i++) { pinv[dv[i].v] = i; p[i] = dv[i].v; }
    Ap[0] = 0;
    for (int32_t i = 0; i < n; i++) {
      int32_t old = dv[i].v;
      int32_t len = rowptr[old + 1] - rowptr[old];
      for (int32_t k = 0; k < len; k++) Ai[Ap[i] + k] = pinv[colidx[rowptr[old] + k]];
      qsort(Ai + Ap[i], (size_t)len, sizeof(int32_t), cmp_int32);
      Ap[i + 1] = Ap[i] + len;
    }
    free(dv);
    free(pinv);
  } else {
    memcpy(Ap, rowptr, ((size_t)n + 1) * sizeof(int32_t));
    memcpy(Ai, colidx, (size_t)nnz * sizeof(int32_t));
  }
  if (c_out) memset(c_out, 0, (size_t)nnz * sizeof(uint32_t));

  /* L = tril(A,-1) and U = triu(A,1), both held by row */
  int32_t *Lp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *Up = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *Li = (int32_t *)malloc(((size_t)nnz + 1) * sizeof(int32_t));
  int32_t *Ui = (int32_t *)malloc(((size_t)nnz + 1) * sizeof(int32_t));
  Lp[0] = 0; Up[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t nl = Lp[i], nu = Up[i];
    for (int32_t k = Ap[i]; k < Ap[i + 1]; k++) {
      int32_t j = Ai[k];
      if (j < i) Li[nl++] = j;
      else if (j > i) Ui[nu++] = j;
    }
    Lp[i + 1] = nl;
    Up[i + 1] = nu;
  }

  /*
   * C<s(L)> = L plus.pair U' : for every entry (i,j) of L,
   * C(i,j) = sum_k pair(L(i,k), U'(k,j)) = |{k : L(i,k) and U(j,k) present}|,
   * a merge of row i of L with row j of U.  Then t = sum over C.
   */
  uint64_t t = 0;
  int64_t visited = 0;
  double t0 = now_seconds();
  for (int32_t i = 0; i < n; i += stride) {
    visited += Lp[i + 1] - Lp[i];
    for (int32_t q = Lp[i]; q < Lp[i + 1]; q++) {
      int32_t j = Li[q];
      int32_t a = Lp[i], ae = Lp[i + 1], b = Up[j], be = Up[j + 1];
      uint64_t cij = 0;
      while (a < ae && b < be) {
        if (Li[a] < Ui[b]) a++;
        else if (Li[a] > Ui[b]) b++;
        else { cij++; a++; b++; }
      }
      t += cij;
      if (c_out) {
        /* the entry (p[i], p[j]) of the given CSR: binary search of p[j] in row p[i] */
        int32_t lo = rowptr[p[i]], hi = rowptr[p[i] + 1];
        while (lo < hi) {
          int32_t mid = lo + (hi - lo) / 2;
          if (colidx[mid] < p[j]) lo = mid + 1; else hi = mid;
        }
        c_out[lo] = (uint32_t)cij;
      }
    }
  }
  if (count_seconds) *count_seconds = now_seconds() - t0;
  if (l_entries) *l_entries = visited;
  free(Ap); free(Ai); free(Lp); free(Up); free(Li); free(Ui); free(p);
  return t;
}

/* ------------------------------------------------------------------------- */
/* Parents BFS, Alg. 1                                                        */
/* ------------------------------------------------------------------------- */

/*
 * level[v] = the loop counter at which v enters q (0 for the source, -1 when
 * never reached), parent[v] = the value q(v) had then (the secondi operator
 * yields the index k of the frontier entry that reached v; the any monoid may
 * keep any of them -- this oracle keeps the one of smallest k, scanning q in
 * index order).  parent[src] = src.  Returns the number of levels (the
 * largest level + 1), or -1 on a bad source / allocation failure.
 * Push uses the rows of A (q' A), so for a directed graph the search follows
 * out-edges.
 */
int32_t oracle_bfs(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t src,
                   int32_t *level, int32_t *parent) {
  if (src < 0 || src >= n) return -1;
  /* sparse vectors: pattern list + dense value/presence arrays */
  int32_t *q_idx = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *q_new = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *q_val = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  unsigned char *in_qnew = (unsigned char *)calloc((size_t)n + 1, 1);
  unsigned char *p_has = (unsigned char *)calloc((size_t)n + 1, 1);
  if (!q_idx || !q_new || !q_val || !in_qnew || !p_has) {
    free(q_idx); free(q_new); free(q_val); free(in_qnew); free(p_has);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) { level[v] = -1; parent[v] = -1; }

  /* p(src) = src ; q(src) = src */
  parent[src] = src; p_has[src] = 1; level[src] = 0;
  int32_t nq = 1;
  q_idx[0] = src; q_val[src] = src;
  int32_t depth = 1;

  for (int32_t lev = 1; lev <= n - 1; lev++) {
    /* q'<!s(p), replace> = q' any.secondi A */
    int32_t nn = 0;
    for (int32_t a = 0; a < nq; a++) {
      int32_t k = q_idx[a];                     /* q(k) present; secondi -> k */
      for (int32_t e = rowptr[k]; e < rowptr[k + 1]; e++) {
        int32_t j = colidx[e];
        if (p_has[j]) continue;                 /* complemented structural mask */
        if (in_qnew[j]) continue;               /* any: keep the first k */
        in_qnew[j] = 1;
        q_new[nn++] = j;
        q_val[j] = k;
      }
    }
    /* replace: the old q is dropped; the new q holds the pattern q_new */
    qsort(q_new, (size_t)nn, sizeof(int32_t), cmp_int32);
    for (int32_t a = 0; a < nn; a++) {
      int32_t j = q_new[a];
      in_qnew[j] = 0;
      /* p<s(q)> = q */
      parent[j] = q_val[j];
      p_has[j] = 1;
      level[j] = lev;
    }
    memcpy(q_idx, q_new, (size_t)nn * sizeof(int32_t));
    nq = nn;
    if (nq == 0) break;
    depth = lev + 1;
  }
  free(q_idx); free(q_new); free(q_val); free(in_qnew); free(p_has);
  return depth;
}

/* ------------------------------------------------------------------------- */
/* PageRank, Alg. 4 (GAP form) and the dangling-redistribution variant       */
/* ------------------------------------------------------------------------- */

/*
 * Unweighted PageRank over plus.second (edge values are ignored).
 *   teleport = (1-alpha)/n ; r = 1/n ; d_out = row degree ; d = d_out / alpha
 *   repeat: t <- r ; w = t ./ d (only where d_out > 0) ; r = teleport ;
 *           r += A' plus.second w ; t = |t - r| ; stop when sum(t) < tol
 * dangling != 0 adds alpha * (sum of t over rows with d_out = 0) / n to every
 * r(i) (the Graphalytics-style fix; the paper names it without a formula).
 * Writes r[n]; returns the number of iterations done (itermax when the
 * tolerance was never met); *resid_out gets the last sum(t).
 */
int32_t oracle_pagerank(int32_t n, const int32_t *rowptr, const int32_t *colidx, double damping,
                        double tol, int32_t itermax, int dangling, double *r, double *resid_out) {
  if (n <= 0) { if (resid_out) *resid_out = 0.0; return 0; }
  double alpha = damping;
  double *t = (double *)malloc(((size_t)n + 1) * sizeof(double));
  double *w = (double *)malloc(((size_t)n + 1) * sizeof(double));
  double *d = (double *)malloc(((size_t)n + 1) * sizeof(double));
  unsigned char *has_d = (unsigned char *)malloc((size_t)n + 1);
  if (!t || !w || !d || !has_d) { free(t); free(w); free(d); free(has_d); return -1; }
  double teleport = (1.0 - alpha) / (double)n;
  for (int32_t i = 0; i < n; i++) r[i] = 1.0 / (double)n;
  for (int32_t i = 0; i < n; i++) {
    int64_t dout = rowptr[i + 1] - rowptr[i];
    has_d[i] = dout > 0;
    d[i] = has_d[i] ? (double)dout / alpha : 0.0;
  }
  int32_t k = 0;
  double resid = INFINITY;
  for (k = 1; k <= itermax; k++) {
    /* swap t and r: t is now the prior rank */
    memcpy(t, r, (size_t)n * sizeof(double));
    /* w = t ./ d on the pattern of d */
    for (int32_t j = 0; j < n; j++) w[j] = has_d[j] ? t[j] / d[j] : 0.0;
    double dang = 0.0;
    if (dangling) {
      for (int32_t j = 0; j < n; j++) if (!has_d[j]) dang += t[j];
      dang = alpha * dang / (double)n;
    }
    for (int32_t i = 0; i < n; i++) r[i] = teleport + dang;
    /* r += A' plus.second w : r(i) += w(j) for every entry A(j,i), j ascending */
    for (int32_t j = 0; j < n; j++) {
      if (!has_d[j]) continue;
      for (int32_t e = rowptr[j]; e < rowptr[j + 1]; e++) r[colidx[e]] += w[j];
    }
    /* t -= r ; t = abs(t) ; sum */
    resid = 0.0;
    for (int32_t i = 0; i < n; i++) resid += fabs(t[i] - r[i]);
    if (resid < tol) break;
  }
  if (k > itermax) k = itermax;
  if (resid_out) *resid_out = resid;
  free(t); free(w); free(d); free(has_d);
  return k;
}

/*
 * Weighted PageRank over plus.times with a row-stochastic W (row i holds the
 * out-edges of i, val = W(i,j)) and a teleport distribution v (NULL means
 * uniform 1/n):
 *   r = 1/n ; repeat: t <- r ;
 *     r(j) = (1-alpha) v(j) + alpha * sum_i W(i,j) t(i)
 *            [ + alpha * (sum of t over rows with no entry) * v(j)  if dangling ]
 *     stop when sum |t - r| < tol.
 * With W(i,j) = 1/d_out(i) and uniform v this is Alg. 4.
 */
int32_t oracle_pagerank_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                                 const double *val, const double *v, double damping, double tol,
                                 int32_t itermax, int dangling, double *r, double *resid_out) {
  if (n <= 0) { if (resid_out) *resid_out = 0.0; return 0; }
  double alpha = damping;
  double *t = (double *)malloc(((size_t)n + 1) * sizeof(double));
  if (!t) return -1;
  for (int32_t i = 0; i < n; i++) r[i] = 1.0 / (double)n;
  int32_t k;
  double resid = INFINITY;
  for (k = 1; k <= itermax; k++) {
    memcpy(t, r, (size_t)n * sizeof(double));
    double dang = 0.0;
    if (dangling)
      for (int32_t i = 0; i < n; i++) if (rowptr[i + 1] == rowptr[i]) dang += t[i];
    for (int32_t j = 0; j < n; j++) {
      double vj = v ? v[j] : 1.0 / (double)n;
      r[j] = (1.0 - alpha) * vj + alpha * dang * vj;
    }
    for (int32_t i = 0; i < n; i++)
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) r[colidx[e]] += alpha * val[e] * t[i];
    resid = 0.0;
    for (int32_t i = 0; i < n; i++) resid += fabs(t[i] - r[i]);
    if (resid < tol) break;
  }
  if (k > itermax) k = itermax;
  if (resid_out) *resid_out = resid;
  free(t);
  return k;
}

/*
 * Adjoint of the weighted fixed point r = F(r, W, v) with
 *   F_j = (1-alpha) v_j + alpha sum_i W_ij r_i + alpha delta v_j,
 *   delta = sum of r over dangling rows (only when `dangling`),
 * for the loss L = sum_j c_j r_j.  By implicit differentiation,
 *   lambda = c + (dF/dr)' lambda, i.e.
 *   lambda_i = c_i + alpha sum_j W_ij lambda_j + alpha [i dangling] (v . lambda),
 * iterated from lambda = c until the L1 change is below tol (or itermax).
 * Then   dL/dW_ij = alpha r_i lambda_j   for every stored (i,j), CSR order,
 *        dL/dv_j  = ((1-alpha) + alpha delta) lambda_j.
 * r must be the forward fixed point.  Any output pointer may be NULL.
 * Returns the number of adjoint iterations.
 */
int32_t oracle_pagerank_adjoint(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                                const double *val, const double *v, const double *r,
                                const double *c, double damping, double tol, int32_t itermax,
                                int dangling, double *dW, double *dv, double *lambda_out) {
  double alpha = damping;
  double *lam = (double *)malloc(((size_t)n + 1) * sizeof(double));
  double *nxt = (double *)malloc(((size_t)n + 1) * sizeof(double));
  if (!lam || !nxt) { free(lam); free(nxt); return -1; }
  for (int32_t i = 0; i < n; i++) lam[i] = c[i];
  int32_t k;
  for (k = 1; k <= itermax; k++) {
    double vl = 0.0;
    if (dangling)
      for (int32_t j = 0; j < n; j++) vl += (v ? v[j] : 1.0 / (double)n) * lam[j];
    double change = 0.0;
    for (int32_t i = 0; i < n; i++) {
      double s = 0.0;
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) s += val[e] * lam[colidx[e]];
      double x = c[i] + alpha * s;
      if (dangling && rowptr[i + 1] == rowptr[i]) x += alpha * vl;
      nxt[i] = x;
      change += fabs(x - lam[i]);
    }
    memcpy(lam, nxt, (size_t)n * sizeof(double));
    if (change < tol) break;
  }
  if (k > itermax) k = itermax;
  double delta = 0.0;
  if (dangling)
    for (int32_t i = 0; i < n; i++) if (rowptr[i + 1] == rowptr[i]) delta += r[i];
  if (dW)
    for (int32_t i = 0; i < n; i++)
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) dW[e] = alpha * r[i] * lam[colidx[e]];
  if (dv)
    for (int32_t j = 0; j < n; j++) dv[j] = ((1.0 - alpha) + alpha * delta) * lam[j];
  if (lambda_out) memcpy(lambda_out, lam, (size_t)n * sizeof(double));
  free(lam);
  free(nxt);
  return k;
}

/* ------------------------------------------------------------------------- */
/* Connected components, Alg. 7 (FastSV)                                      */
/* ------------------------------------------------------------------------- */

/*
 * The forest of parent pointers starts as n singleton trees (f = identity).
 * Each round, in the paper's order:
 *   Step 1 (stochastic hooking): mngf <min>= A min.second gf, i.e.
 *     mngf(u) = min(mngf(u), min over the entries A(u,v) of gf(v)); then the
 *     assignment f(x) <min>= mngf with x the parent list extracted from f:
 *     f(x(k)) = min(f(x(k)), mngf(k)) for every k (duplicates of x all apply);
 *   Step 2 (aggressive hooking): f = min(f, mngf) elementwise;
 *   Step 3 (shortcutting): f = min(f, gf) elementwise;
 *   Step 4 (grandparents): x = f; gf = f(x), i.e. gf(k) = f(f(k));
 *   Step 5 (termination): sum = #{k : dup(k) != gf(k)}; dup = gf;
 * until sum == 0.  gf, dup and mngf start as copies of f.  On an undirected
 * graph f(u) ends as the smallest vertex id of u's component.
 * Writes f[n]; returns the number of rounds, or -1 on an allocation failure.
 */
int32_t oracle_fastsv(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *f) {
  if (n <= 0) return 0;
  int32_t *gf = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *dup = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *mngf = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *x = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!gf || !dup || !mngf || !x) { free(gf); free(dup); free(mngf); free(x); return -1; }
  for (int32_t u = 0; u < n; u++) f[u] = u;
  for (int32_t u = 0; u < n; u++) { gf[u] = f[u]; dup[u] = gf[u]; mngf[u] = gf[u]; x[u] = f[u]; }
  int32_t rounds = 0;
  int64_t sum;
  do {
    rounds++;
    /* Step 1: mngf <min>= A min.second gf, then f(x) <min>= mngf */
    for (int32_t u = 0; u < n; u++)
      for (int32_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
        int32_t v = colidx[e];
        if (gf[v] < mngf[u]) mngf[u] = gf[v];
      }
    for (int32_t k = 0; k < n; k++)
      if (mngf[k] < f[x[k]]) f[x[k]] = mngf[k];
    /* Step 2: f = f min mngf */
    for (int32_t u = 0; u < n; u++)
      if (mngf[u] < f[u]) f[u] = mngf[u];
    /* Step 3: f = f min gf */
    for (int32_t u = 0; u < n; u++)
      if (gf[u] < f[u]) f[u] = gf[u];
    /* Step 4: {i, x} = f ; gf = f(x) */
    for (int32_t k = 0; k < n; k++) x[k] = f[k];
    for (int32_t k = 0; k < n; k++) gf[k] = f[x[k]];
    /* Step 5: diff = (dup != gf) ; sum = +reduce(diff) ; dup = gf */
    sum = 0;
    for (int32_t k = 0; k < n; k++) sum += dup[k] != gf[k];
    memcpy(dup, gf, (size_t)n * sizeof(int32_t));
  } while (sum != 0);
  free(gf); free(dup); free(mngf); free(x);
  return rounds;
}

/* ------------------------------------------------------------------------- */
/* Single-source shortest paths, Alg. 5 (delta-stepping), float32             */
/* ------------------------------------------------------------------------- */

/*
 * The arithmetic is float32, the type of t and the edge values in Alg. 5: a
 * relaxation is the float32 sum t(u) + A(u,v) rounded to nearest.  t is a
 * sparse vector (an unreached vertex has no entry; reported as +inf).
 *   A_L = the entries with 0 < A <= delta, A_H = the entries with A > delta;
 *   t(s) = 0; i = 0;
 *   while some entry of t has t >= i delta:
 *     tB = the entries of t with i delta <= t < (i+1) delta; e = empty;
 *     while tB has entries:
 *       tReq = A_L' min.plus (t .* tB)   (t restricted to the pattern of tB)
 *       e = e + the pattern of tB
 *       tB = the entries of tReq with i delta <= tReq < (i+1) delta and tReq < t
 *       t = t min tReq                   (eWiseAdd: min where both exist)
 *     tReq = A_H' min.plus (t .* e); t = t min tReq; i = i + 1
 * The bucket bounds i delta are formed in float64.  Writes t[n]; returns the
 * number of buckets processed, or -1 on a bad source, delta or allocation.
 */
int32_t oracle_sssp_delta(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *w,
                          int32_t src, float delta, float *t) {
  if (src < 0 || src >= n || !(delta > 0.0f)) return -1;
  unsigned char *has_t = (unsigned char *)calloc((size_t)n, 1);
  unsigned char *inB = (unsigned char *)calloc((size_t)n, 1);
  unsigned char *inE = (unsigned char *)calloc((size_t)n, 1);
  unsigned char *hasR = (unsigned char *)calloc((size_t)n, 1);
  float *req = (float *)malloc((size_t)n * sizeof(float));
  if (!has_t || !inB || !inE || !hasR || !req) {
    free(has_t); free(inB); free(inE); free(hasR); free(req);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) t[v] = INFINITY;
  t[src] = 0.0f;
  has_t[src] = 1;
  int32_t buckets = 0;
  for (int64_t i = 0;; i++) {
    const double lo = (double)i * (double)delta, hi = (double)(i + 1) * (double)delta;
    int any = 0;
    for (int32_t v = 0; v < n && !any; v++) any = has_t[v] && (double)t[v] >= lo;
    if (!any) break;
    buckets++;
    int64_t nb = 0;
    for (int32_t v = 0; v < n; v++) {
      inB[v] = has_t[v] && (double)t[v] >= lo && (double)t[v] < hi;
      nb += inB[v];
      inE[v] = 0;
    }
    while (nb > 0) {
      /* tReq = A_L' min.plus (t .* tB) */
      memset(hasR, 0, (size_t)n);
      for (int32_t u = 0; u < n; u++) {
        if (!inB[u]) continue;
        for (int32_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
          const float a = w[e];
          if (!(a > 0.0f && a <= delta)) continue;
          const int32_t v = colidx[e];
          const float cand = t[u] + a;
          if (!hasR[v] || cand < req[v]) { req[v] = cand; hasR[v] = 1; }
        }
      }
      /* e = e + s(tB) */
      for (int32_t u = 0; u < n; u++) if (inB[u]) inE[u] = 1;
      /* tB = tReq in bucket i that improves t; then t = t min tReq */
      nb = 0;
      for (int32_t v = 0; v < n; v++) {
        const int improves = hasR[v] && (!has_t[v] || req[v] < t[v]);
        inB[v] = improves && (double)req[v] >= lo && (double)req[v] < hi;
        nb += inB[v];
        if (improves) { t[v] = req[v]; has_t[v] = 1; }
      }
    }
    /* tReq = A_H' min.plus (t .* e) ; t = t min tReq */
    memset(hasR, 0, (size_t)n);
    for (int32_t u = 0; u < n; u++) {
      if (!inE[u]) continue;
      for (int32_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
        const float a = w[e];
        if (!(a > delta)) continue;
        const int32_t v = colidx[e];
        const float cand = t[u] + a;
        if (!hasR[v] || cand < req[v]) { req[v] = cand; hasR[v] = 1; }
      }
    }
    for (int32_t v = 0; v < n; v++)
      if (hasR[v] && (!has_t[v] || req[v] < t[v])) { t[v] = req[v]; has_t[v] = 1; }
  }
  free(has_t); free(inB); free(inE); free(hasR); free(req);
  return buckets;
}

/* ------------------------------------------------------------------------- */
/* Batched betweenness centrality, Alg. 3 (float64)                           */
/* ------------------------------------------------------------------------- */

/*
 * ns sources s_1..s_ns (row k of the ns x n matrices belongs to s_k).
 *   P(k, s_k) = 1;  F<!s(P)> = P plus.first A          (the first frontier)
 *   BFS phase, d = 0, 1, ...:  S[d] = s(F);  P += F;
 *     F<!s(P), replace> = F plus.first A;  stop when F has no entry.
 *   Backtrack phase: B(:) = 1;  for i = D down to 1 (D the last BFS level):
 *     W<s(S[i]), replace> = B ./ P;  W<s(S[i-1]), replace> = W plus.first A';
 *     B += W .* P (on the pattern of W).
 *   centrality(j) = sum_k (B(k, j) - 1).
 * plus.first keeps the left operand: (F plus.first A)(k,j) = sum of F(k,i)
 * over the entries A(i,j); (W plus.first A')(k,j) = sum of W(k,l) over the
 * entries A(j,l).  Sparse matrices are dense value arrays with presence flags.
 * Writes centrality[n]; returns the number of BFS levels (D + 1), or -1 on a
 * bad source or an allocation failure.
 */
int32_t oracle_bc(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t ns, const int32_t *src,
                  double *centrality) {
  if (n <= 0 || ns <= 0) { for (int32_t j = 0; j < n; j++) centrality[j] = 0.0; return 0; }
  for (int32_t k = 0; k < ns; k++) if (src[k] < 0 || src[k] >= n) return -1;
  const size_t N = (size_t)ns * (size_t)n;
  double *P = (double *)calloc(N, sizeof(double));
  double *F = (double *)calloc(N, sizeof(double));
  double *Fn = (double *)calloc(N, sizeof(double));
  double *B = (double *)malloc(N * sizeof(double));
  double *W = (double *)calloc(N, sizeof(double));
  double *Wn = (double *)calloc(N, sizeof(double));
  unsigned char *hasP = (unsigned char *)calloc(N, 1);
  unsigned char *hasF = (unsigned char *)calloc(N, 1);
  unsigned char *hasFn = (unsigned char *)calloc(N, 1);
  unsigned char *hasW = (unsigned char *)calloc(N, 1);
  unsigned char *hasWn = (unsigned char *)calloc(N, 1);
  int32_t *lev = (int32_t *)malloc(N * sizeof(int32_t));  /* lev(k,j) = d where (k,j) is in S[d] */
  int rc = 0;
  if (!P || !F || !Fn || !B || !W || !Wn || !hasP || !hasF || !hasFn || !hasW || !hasWn || !lev) { rc = -1; goto done; }
  for (size_t q = 0; q < N; q++) lev[q] = -1;
  /* P(k, s_k) = 1 */
  for (int32_t k = 0; k < ns; k++) { P[(size_t)k * n + src[k]] = 1.0; hasP[(size_t)k * n + src[k]] = 1; }
  /* F<!s(P)> = P plus.first A */
  for (int32_t k = 0; k < ns; k++) {
    const size_t r = (size_t)k * n;
    for (int32_t i = 0; i < n; i++) {
      if (!hasP[r + i]) continue;
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        const int32_t j = colidx[e];
        if (hasP[r + j]) continue;
        F[r + j] += P[r + i];
        hasF[r + j] = 1;
      }
    }
  }
  int32_t d = 0;
  int64_t nvF = 0;
  for (size_t q = 0; q < N; q++) nvF += hasF[q];
  if (nvF == 0) { rc = 0; d = -1; }
  else {
    for (d = 0; d < n; d++) {
      /* S[d] = s(F); P += F */
      for (size_t q = 0; q < N; q++) {
        if (!hasF[q]) continue;
        lev[q] = d;
        P[q] += F[q];
        hasP[q] = 1;
      }
      /* F<!s(P), replace> = F plus.first A */
      memset(hasFn, 0, N);
      for (size_t q = 0; q < N; q++) Fn[q] = 0.0;
      for (int32_t k = 0; k < ns; k++) {
        const size_t r = (size_t)k * n;
        for (int32_t i = 0; i < n; i++) {
          if (!hasF[r + i]) continue;
          for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            const int32_t j = colidx[e];
            if (hasP[r + j]) continue;
            Fn[r + j] += F[r + i];
            hasFn[r + j] = 1;
          }
        }
      }
      nvF = 0;
      for (size_t q = 0; q < N; q++) { F[q] = Fn[q]; hasF[q] = hasFn[q]; nvF += hasF[q]; }
      if (nvF == 0) break;
    }
  }
  /* backtrack: B(:) = 1 */
  for (size_t q = 0; q < N; q++) B[q] = 1.0;
  for (int32_t i = d; i >= 1; i--) {
    /* W<s(S[i]), replace> = B ./ P */
    for (size_t q = 0; q < N; q++) {
      hasW[q] = lev[q] == i;
      W[q] = hasW[q] ? B[q] / P[q] : 0.0;
    }
    /* W<s(S[i-1]), replace> = W plus.first A' */
    for (int32_t k = 0; k < ns; k++) {
      const size_t r = (size_t)k * n;
      for (int32_t j = 0; j < n; j++) {
        hasWn[r + j] = 0;
        Wn[r + j] = 0.0;
        if (lev[r + j] != i - 1) continue;
        for (int32_t e = rowptr[j]; e < rowptr[j + 1]; e++) {
          const int32_t l = colidx[e];
          if (!hasW[r + l]) continue;
          Wn[r + j] += W[r + l];
          hasWn[r + j] = 1;
        }
      }
    }
    /* B += W .* P */
    for (size_t q = 0; q < N; q++)
      if (hasWn[q]) B[q] += Wn[q] * P[q];
  }
  /* centrality = -ns + sum_k B(k, :) */
  for (int32_t j = 0; j < n; j++) {
    double c = -(double)ns;
    for (int32_t k = 0; k < ns; k++) c += B[(size_t)k * n + j];
    centrality[j] = c;
  }
  rc = d + 1;
done:
  free(P); free(F); free(Fn); free(B); free(W); free(Wn);
  free(hasP); free(hasF); free(hasFn); free(hasW); free(hasWn); free(lev);
  return rc;
}
