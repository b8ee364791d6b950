"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to a closed form, a brute-force count, a
library routine (numpy/scipy/torch dense linear algebra, scipy's unweighted
shortest paths) or an invariant of the mathematics, so that a dropped term, a
wrong sign/index or a transposed operand in ``oracle/oracle.c`` fails here.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(g):
    A = np.zeros((g.n, g.n), dtype=np.float64)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    A[rows, g.colidx] = 1.0 if g.val is None else g.val
    return A


def permuted(g, perm):
    """The same graph with vertex v renamed perm[v]."""
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    return gen.from_edges(g.n, perm[rows], perm[g.colidx], symmetric=not g.directed)


# ----------------------------------------------------------------------------------------------
# Triangle counting (Alg. 6)
# ----------------------------------------------------------------------------------------------

def brute_triangles(g):
    """O(n^3) count of vertex triples {a<b<c} with all three edges present."""
    A = dense(g) != 0
    t = 0
    for a, b, c in itertools.combinations(range(g.n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            t += 1
    return t


def brute_triangles_np(g):
    """Same count, vectorised per (a,b) pair, for n up to a few hundred."""
    A = (dense(g) != 0).astype(np.int64)
    t = 0
    for a in range(g.n):
        for b in np.nonzero(A[a, a + 1:])[0] + a + 1:
            t += int((A[a, b + 1:] & A[b, b + 1:]).sum())
    return t


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_complete_graph(method):
    for n in [1, 2, 3, 4, 5, 7, 12, 33]:
        assert oracle.tc(gen.complete(n), method) == math.comb(n, 3)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_triangle_free_families(method):
    assert oracle.tc(gen.grid(30, 17), method) == 0          # bipartite
    assert oracle.tc(gen.star(40), method) == 0
    assert oracle.tc(gen.binary_tree(63), method) == 0
    assert oracle.tc(gen.complete_bipartite(7, 9), method) == 0
    assert oracle.tc(gen.cycle(10), method) == 0
    assert oracle.tc(gen.path(5), method) == 0


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_wheel(method):
    # hub + k-cycle: one triangle per rim edge for k >= 4; W_3 is K_4
    for k in [4, 5, 6, 11, 50]:
        assert oracle.tc(gen.wheel(k), method) == k
    assert oracle.tc(gen.wheel(3), method) == 4


def test_tc_brute_force_small():
    for seed in range(8):
        g = gen.random_graph(24, 0.35, seed=100 + seed)
        bf = brute_triangles(g)
        for m in (0, 1, 2):
            assert oracle.tc(g, m) == bf


def test_tc_brute_force_medium():
    g = gen.random_graph(160, 0.12, seed=7)
    assert oracle.tc(g) == brute_triangles_np(g)


def test_tc_trace_cube():
    # trace(A^3) / 6, exact in float64 well below 2^53
    for g in [gen.rmat(10, 16, seed=3), gen.rmat(11, 8, seed=4), gen.erdos_renyi(1500, 30, seed=5)]:
        A = dense(g)
        expect = int(round(np.trace(A @ A @ A) / 6))
        for m in (0, 1, 2):
            assert oracle.tc(g, m) == expect


def test_tc_self_loops_ignored():
    # strict tril/triu: a self-loop must not create or change triangles
    g = gen.random_graph(30, 0.3, seed=11)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    loops = np.arange(0, g.n, 3)
    gl = gen.from_edges(g.n, np.concatenate([rows, loops]), np.concatenate([g.colidx, loops]),
                        symmetric=True, drop_self=False)
    assert gl.nnz == g.nnz + len(loops)
    assert oracle.tc(gl, 1) == oracle.tc(gl, 2) == brute_triangles(g)


def test_tc_relabel_invariance():
    g = gen.rmat(9, 16, seed=21)
    t = oracle.tc(g)
    for s in range(3):
        perm = np.argsort(gen.uniform_open0(g.n, 900 + s)).astype(np.int32)
        assert oracle.tc(permuted(g, perm), 2) == t


def test_tc_sort_heuristic():
    for g in [gen.rmat(12, 16), gen.grid(20, 20), gen.star(30), gen.complete(6)]:
        decision, mean, median = oracle.tc_wants_sort(g)
        d = np.sort(g.degree())
        assert math.isclose(mean, d.mean())
        assert median == d[(g.n - 1) // 2]
        assert decision == (d.mean() > 4 * d[(g.n - 1) // 2])
    assert oracle.tc_wants_sort(gen.rmat(12, 16))[0]      # skewed: Alg. 6 sorts
    assert not oracle.tc_wants_sort(gen.grid(20, 20))[0]  # regular: it does not


# ----------------------------------------------------------------------------------------------
# BFS (Alg. 1)
# ----------------------------------------------------------------------------------------------

def check_parents(g, level, parent, src):
    """parent[v] >= 0 <=> level[v] >= 0; (parent[v], v) is an edge one level up."""
    assert parent[src] == src and level[src] == 0
    assert np.array_equal(parent >= 0, level >= 0)
    for v in np.nonzero(level > 0)[0]:
        u = parent[v]
        row = g.colidx[g.rowptr[u]:g.rowptr[u + 1]]
        assert v in row
        assert level[u] == level[v] - 1


def scipy_levels(g, src):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    M = sp.csr_matrix((np.ones(g.nnz), g.colidx, g.rowptr), shape=(g.n, g.n))
    d = csgraph.shortest_path(M, directed=True, unweighted=True, indices=src)
    return np.where(np.isinf(d), -1, d).astype(np.int64)


def test_bfs_path():
    g = gen.path(50)
    level, parent, depth = oracle.bfs(g, 0)
    assert np.array_equal(level, np.arange(50))
    assert np.array_equal(parent[1:], np.arange(49))
    assert depth == 50
    level, _, _ = oracle.bfs(g, 20)
    assert np.array_equal(level, np.abs(np.arange(50) - 20))


def test_bfs_star():
    g = gen.star(25)
    level, parent, _ = oracle.bfs(g, 0)
    assert level[0] == 0 and (level[1:] == 1).all() and (parent[1:] == 0).all()
    level, parent, _ = oracle.bfs(g, 7)
    expect = np.full(26, 2)
    expect[7], expect[0] = 0, 1
    assert np.array_equal(level, expect)
    check_parents(g, level, parent, 7)


def test_bfs_grid_manhattan():
    R, C = 64, 48
    g = gen.grid(R, C)
    r, c = np.divmod(np.arange(R * C), C)
    level, parent, depth = oracle.bfs(g, 0)
    assert np.array_equal(level, r + c)
    assert depth == R + C - 1
    src = 20 * C + 30
    level, parent, _ = oracle.bfs(g, src)
    assert np.array_equal(level, np.abs(r - 20) + np.abs(c - 30))
    check_parents(g, level, parent, src)


def test_bfs_complete_and_disconnected():
    level, _, _ = oracle.bfs(gen.complete(9), 4)
    assert level[4] == 0 and (np.delete(level, 4) == 1).all()
    two = gen.concat([gen.path(5), gen.cycle(6)])
    level, parent, _ = oracle.bfs(two, 2)
    assert np.array_equal(level[:5], [2, 1, 0, 1, 2])
    assert (level[5:] == -1).all() and (parent[5:] == -1).all()
    level, parent, depth = oracle.bfs(two, 8)
    assert (level[:5] == -1).all() and depth == 4


def test_bfs_isolated_source():
    g = gen.rmat(8, 4, seed=2)
    iso = int(np.nonzero(g.degree() == 0)[0][0])
    level, parent, depth = oracle.bfs(g, iso)
    assert level[iso] == 0 and parent[iso] == iso and depth == 1
    assert (np.delete(level, iso) == -1).all()


def test_bfs_boolean_powers():
    # level[v] = smallest k with (A^k)[src, v] != 0, by repeated boolean products
    g = gen.random_graph(40, 0.06, seed=3, directed=True)
    A = dense(g) != 0
    for src in [0, 5, 17]:
        level, parent, _ = oracle.bfs(g, src)
        reach = np.zeros(g.n, dtype=bool)
        reach[src] = True
        expect = np.full(g.n, -1)
        expect[src] = 0
        frontier = reach.copy()
        for k in range(1, g.n):
            frontier = (frontier[:, None] & A).any(axis=0) & ~reach
            expect[frontier] = k
            reach |= frontier
        assert np.array_equal(level, expect)
        check_parents(g, level, parent, src)


@pytest.mark.parametrize("directed", [False, True])
def test_bfs_scipy_shortest_path(directed):
    g = gen.rmat(10, 8, seed=31, directed=directed)
    for src in gen.sources(g, 4, seed=5):
        level, parent, _ = oracle.bfs(g, src)
        assert np.array_equal(level, scipy_levels(g, src))
        check_parents(g, level, parent, src)


# ----------------------------------------------------------------------------------------------
# PageRank (Alg. 4)
# ----------------------------------------------------------------------------------------------

def dense_pagerank(g, alpha, dangling, W=None, v=None):
    """Fixed point by a dense float64 solve of (I - M) r = b."""
    n = g.n
    A = dense(g) if W is None else W
    if W is None:
        d = A.sum(axis=1)
        P = np.divide(A, d[:, None], out=np.zeros_like(A), where=d[:, None] > 0)
    else:
        P = A
    vv = np.full(n, 1.0 / n) if v is None else v
    M = alpha * P.T
    if dangling:
        dang = (dense(g) != 0).sum(axis=1) == 0
        M = M + alpha * np.outer(vv, dang.astype(np.float64))
    return np.linalg.solve(np.eye(n) - M, (1 - alpha) * vv)


@pytest.mark.parametrize("dangling", [False, True])
def test_pagerank_dense_solve(dangling):
    for g in [gen.rmat(9, 8, seed=1), gen.rmat(8, 16, seed=2, directed=True),
              gen.random_graph(60, 0.05, seed=9, directed=True)]:
        r, k, res = oracle.pagerank(g, 0.85, 1e-14, 2000, dangling)
        assert res < 1e-14
        np.testing.assert_allclose(r, dense_pagerank(g, 0.85, dangling), rtol=0, atol=1e-12)


def test_pagerank_dense_power_iteration():
    # the same iteration written as dense matrix-vector products, step for step
    g = gen.rmat(8, 8, seed=6, directed=True)
    A = dense(g)
    d = A.sum(axis=1)
    alpha = 0.85
    r = np.full(g.n, 1.0 / g.n)
    for _ in range(7):
        w = np.divide(alpha * r, d, out=np.zeros_like(r), where=d > 0)
        r = (1 - alpha) / g.n + A.T @ w
    ro, k, _ = oracle.pagerank(g, alpha, 0.0, 7, False)
    assert k == 7
    np.testing.assert_allclose(ro, r, rtol=0, atol=1e-15)


def test_pagerank_regular_graphs_uniform():
    for g in [gen.cycle(31), gen.complete(12), gen.grid(1, 2)]:
        r, _, _ = oracle.pagerank(g, 0.85, 1e-14, 500)
        np.testing.assert_allclose(r, 1.0 / g.n, rtol=0, atol=1e-15)
    # 2D torus (every vertex degree 4)
    R = C = 8
    v = np.arange(R * C)
    rr, cc = np.divmod(v, C)
    right = rr * C + (cc + 1) % C
    down = ((rr + 1) % R) * C + cc
    torus = gen.from_edges(R * C, np.concatenate([v, v]), np.concatenate([right, down]))
    r, _, _ = oracle.pagerank(torus, 0.85, 1e-14, 500)
    np.testing.assert_allclose(r, 1.0 / (R * C), rtol=0, atol=1e-15)


def test_pagerank_star_closed_form():
    # centre: r_c = a (1 + alpha s) / (1 - alpha^2); leaf: r_l = a + alpha r_c / s, a = (1-alpha)/n
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        cases = json.load(f)["pagerank_star"]["cases"]
    for case in cases:
        s, alpha = case["s"], case["alpha"]
        r, _, _ = oracle.pagerank(gen.star(s), alpha, 1e-15, 5000)
        assert abs(r[0] - case["r_centre"]) < 1e-13
        np.testing.assert_allclose(r[1:], case["r_leaf"], rtol=0, atol=1e-13)
        assert abs(r.sum() - 1.0) < 1e-12


def test_pagerank_mass():
    g = gen.rmat(12, 16)                       # has isolated (dangling) vertices
    r, _, _ = oracle.pagerank(g, 0.85, 1e-12, 1000, dangling=True)
    assert abs(r.sum() - 1.0) < 1e-10
    r_gap, _, _ = oracle.pagerank(g, 0.85, 1e-12, 1000, dangling=False)
    assert r_gap.sum() < 1.0 - 1e-3            # GAP form drops the dangling mass


def test_pagerank_tolerance_bound():
    # res < tol puts the iterate within tol * alpha / (1 - alpha) of the fixed point (L1)
    g = gen.rmat(12, 16)
    r_tol, k, res = oracle.pagerank(g, 0.85, 1e-7, 100)
    r_ex, _, _ = oracle.pagerank(g, 0.85, 1e-15, 5000)
    assert res < 1e-7
    assert np.abs(r_tol - r_ex).sum() <= 1e-7 * 0.85 / 0.15
    assert np.abs(r_tol - r_ex).max() < 1e-6


def test_pagerank_itermax():
    g = gen.rmat(10, 16, seed=8)
    _, k, res = oracle.pagerank(g, 0.85, 0.0, 5)
    assert k == 5 and res > 0


# ----------------------------------------------------------------------------------------------
# Weighted PageRank and its adjoint
# ----------------------------------------------------------------------------------------------

def weighted_case(scale=7, seed=3):
    g = gen.rmat_weighted_directed(scale, 8, seed=seed)
    return g, g.meta["val64"]


@pytest.mark.parametrize("dangling", [False, True])
def test_weighted_matches_unweighted_on_degree_weights(dangling):
    g = gen.rmat(9, 8, seed=12, directed=True)
    d = np.diff(g.rowptr)
    val = 1.0 / np.repeat(d, d)
    r1, k1, _ = oracle.pagerank(g, 0.85, 1e-13, 1000, dangling)
    r2, k2, _ = oracle.pagerank_weighted(g, val, None, 0.85, 1e-13, 1000, dangling)
    np.testing.assert_allclose(r1, r2, rtol=0, atol=1e-14)
    assert k1 == k2


@pytest.mark.parametrize("dangling", [False, True])
def test_weighted_dense_solve(dangling):
    g, w = weighted_case()
    v = gen.uniform_open0(g.n, 77)
    v /= v.sum()
    W = dense(gen.Graph(g.n, g.rowptr, g.colidx, True, w))
    r, _, _ = oracle.pagerank_weighted(g, w, v, 0.85, 1e-15, 5000, dangling)
    np.testing.assert_allclose(r, dense_pagerank(g, 0.85, dangling, W=W, v=v), rtol=0, atol=1e-13)


@pytest.mark.parametrize("dangling", [False, True])
def test_adjoint_finite_differences(dangling):
    g, w = weighted_case(7, 5)
    v = np.full(g.n, 1.0 / g.n)
    c = gen.normal(g.n, 123)
    alpha = 0.85
    r, _, _ = oracle.pagerank_weighted(g, w, v, alpha, 1e-15, 5000, dangling)
    dW, dv, _, _ = oracle.pagerank_adjoint(g, w, r, c, v, alpha, 1e-15, 5000, dangling)
    sample = np.unique((gen.uniform_open0(32, 55) * g.nnz).astype(np.int64))
    for e in sample:
        h = 1e-6 * max(abs(w[e]), 1e-3)
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        Lp = c @ oracle.pagerank_weighted(g, wp, v, alpha, 1e-15, 5000, dangling)[0]
        Lm = c @ oracle.pagerank_weighted(g, wm, v, alpha, 1e-15, 5000, dangling)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dW[e]) <= 1e-6 * max(1.0, abs(dW).max())
    # teleport gradient by central differences on a few coordinates
    for j in [0, 3, g.n - 1]:
        h = 1e-7
        vp, vm = v.copy(), v.copy()
        vp[j] += h
        vm[j] -= h
        Lp = c @ oracle.pagerank_weighted(g, w, vp, alpha, 1e-15, 5000, dangling)[0]
        Lm = c @ oracle.pagerank_weighted(g, w, vm, alpha, 1e-15, 5000, dangling)[0]
        assert abs((Lp - Lm) / (2 * h) - dv[j]) <= 1e-6 * max(1.0, abs(dv).max())


@pytest.mark.parametrize("dangling", [False, True])
def test_adjoint_dense_autograd(dangling):
    torch = pytest.importorskip("torch")
    g, w = weighted_case(8, 9)
    n = g.n
    alpha = 0.85
    c = gen.normal(n, 321)
    v = np.full(n, 1.0 / n)
    r, _, _ = oracle.pagerank_weighted(g, w, v, alpha, 1e-15, 5000, dangling)
    dW, dv, _, _ = oracle.pagerank_adjoint(g, w, r, c, v, alpha, 1e-15, 5000, dangling)

    rows = torch.as_tensor(np.repeat(np.arange(n), np.diff(g.rowptr)))
    cols = torch.as_tensor(g.colidx.astype(np.int64))
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    vt = torch.tensor(v, dtype=torch.float64, requires_grad=True)
    W = torch.zeros(n, n, dtype=torch.float64).index_put((rows, cols), wt)
    M = alpha * W.T
    if dangling:
        dang = torch.as_tensor(np.diff(g.rowptr) == 0, dtype=torch.float64)
        M = M + alpha * torch.outer(vt, dang)
    rt = torch.linalg.solve(torch.eye(n, dtype=torch.float64) - M, (1 - alpha) * vt)
    L = torch.dot(torch.as_tensor(c), rt)
    gw, gv = torch.autograd.grad(L, (wt, vt))
    gw, gv = gw.numpy(), gv.numpy()
    assert np.linalg.norm(dW - gw) <= 1e-9 * np.linalg.norm(gw)
    assert np.linalg.norm(dv - gv) <= 1e-9 * np.linalg.norm(gv)


def test_adjoint_euler_identity():
    # GAP form (no dangling term): r is linear in v, so sum_j dL/dv_j v_j = L
    g, w = weighted_case(8, 10)
    v = gen.uniform_open0(g.n, 5)
    v /= v.sum()
    c = gen.normal(g.n, 6)
    r, _, _ = oracle.pagerank_weighted(g, w, v, 0.85, 1e-15, 5000, False)
    _, dv, _, _ = oracle.pagerank_adjoint(g, w, r, c, v, 0.85, 1e-15, 5000, False)
    assert abs(dv @ v - c @ r) < 1e-12 * max(1.0, abs(c @ r))


# ----------------------------------------------------------------------------------------------
# Stored golden values
# ----------------------------------------------------------------------------------------------

def test_golden_closed_forms_file():
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        cf = json.load(f)
    for case in cf["triangles"]["cases"]:
        g = getattr(gen, case["graph"])(*case["args"])
        assert oracle.tc(g) == case["t"]


def test_golden_rmat12(rmat12):
    with open(os.path.join(GOLDEN, "rmat12_oracle.json")) as f:
        gold = json.load(f)
    g = rmat12
    assert g.nnz == gold["nnz"]
    assert int(np.bitwise_xor.reduce(g.colidx.astype(np.int64) * 2654435761 % 2**32)) == gold["colidx_hash"]
    assert oracle.tc(g) == gold["triangles"]
    level, _, depth = oracle.bfs(g, 0)
    assert depth == gold["bfs0_depth"]
    assert np.bincount(level[level >= 0]).tolist() == gold["bfs0_level_histogram"]
