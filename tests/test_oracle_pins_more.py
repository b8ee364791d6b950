"""Pins of the oracle's newer functions: C<s(L)> kept (Alg. 6), FastSV (Alg. 7), delta-stepping
SSSP (Alg. 5) and batched betweenness centrality (Alg. 3).

As in test_oracle_pins.py, every check here ties the oracle to something that does not come from
the oracle: a closed form, a brute-force count over all vertex triples / pairs, a library routine
(scipy's connected components and Dijkstra) or an invariant of the mathematics (the sum of C is t;
the shortest-path distances are the least fixed point of the float32 Bellman equations, so they do
not depend on delta).
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import gen
import oracle


def dense_bool(g):
    A = np.zeros((g.n, g.n), dtype=bool)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    A[rows, g.colidx] = True
    return A


def csr_scipy(g, values=None):
    v = np.ones(g.nnz) if values is None else values
    return sp.csr_matrix((v, g.colidx, g.rowptr), shape=(g.n, g.n))


def entries(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    return rows, g.colidx.astype(np.int64)


# ----------------------------------------------------------------------------------------------
# C<s(L)> = L plus.pair U' kept (Alg. 6, unfused)
# ----------------------------------------------------------------------------------------------

def degree_order(g):
    """New label of every vertex under the ascending (degree, id) order of Alg. 6."""
    deg = np.diff(g.rowptr)
    order = np.lexsort((np.arange(g.n), deg))   # old vertex of each new label
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    return rank


def brute_c(g, rank):
    """C(i,j) = #{k : j < k < i, k adjacent to both} in the labels `rank`, at every stored entry
    (i,j) with rank i > rank j; 0 at the other entries."""
    A = dense_bool(g)
    inv = np.argsort(rank)
    Ar = A[np.ix_(inv, inv)]                      # Ar[a, b] = A(old a, old b)
    rows, cols = entries(g)
    out = np.zeros(g.nnz, dtype=np.int64)
    for e, (u, v) in enumerate(zip(rows, cols)):
        i, j = rank[u], rank[v]
        if i > j:
            out[e] = int((Ar[i, j + 1:i] & Ar[j, j + 1:i]).sum())
    return out


def test_tc_edges_complete_graph_closed_form():
    # K_n on its own labels: every k strictly between j and i closes a triangle, C(i,j) = i - j - 1
    n = 23
    g = gen.complete(n)
    c, t = oracle.tc_edges(g, oracle.TC_NOSORT)
    rows, cols = entries(g)
    expect = np.where(rows > cols, rows - cols - 1, 0)
    assert np.array_equal(c.astype(np.int64), expect)
    assert t == math.comb(n, 3)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_edges_brute_force(method):
    for seed in range(4):
        g = gen.random_graph(60, 0.2, seed)
        c, t = oracle.tc_edges(g, method)
        sort = method == 1 or (method == 0 and oracle.tc_wants_sort(g)[0])
        rank = degree_order(g) if sort else np.arange(g.n)
        assert np.array_equal(c.astype(np.int64), brute_c(g, rank))
        assert t == int(c.sum()) == oracle.tc(g, method)


def test_tc_edges_skewed_graph_sorts():
    g = gen.rmat(11, 4, seed=5)
    assert oracle.tc_wants_sort(g)[0]
    c, t = oracle.tc_edges(g, oracle.TC_AUTO)
    assert np.array_equal(c.astype(np.int64), brute_c(g, degree_order(g)))
    # every triangle {a<b<c} (new labels) is counted at exactly one entry, (c, a)
    assert t == int(c.sum())
    rows, cols = entries(g)
    rk = degree_order(g)
    assert (c[rk[rows] < rk[cols]] == 0).all()


# ----------------------------------------------------------------------------------------------
# FastSV connected components (Alg. 7)
# ----------------------------------------------------------------------------------------------

def min_label_components(g):
    """The smallest vertex id of each vertex's component, from scipy."""
    ncomp, lab = csg.connected_components(csr_scipy(g), directed=False)
    first = np.full(ncomp, g.n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(g.n))
    return first[lab]


@pytest.mark.parametrize("case", ["rmat", "er", "grid", "forest", "path_reversed"])
def test_fastsv_scipy(case):
    if case == "rmat":
        g = gen.rmat(11, 4, seed=3)            # many small components and isolated vertices
    elif case == "er":
        g = gen.erdos_renyi(3000, 1.2, seed=4)  # near the percolation threshold
    elif case == "grid":
        g = gen.grid(17, 29)
    elif case == "forest":
        g = gen.binary_tree(500)
        rows, cols = entries(g)
        keep = (rows % 7 != 3) & (cols % 7 != 3)  # cut the tree into pieces
        g = gen.from_edges(g.n, rows[keep], cols[keep])
    else:  # a path whose labels decrease along it: the minimum sits at the far end
        n = 300
        v = np.arange(n)[::-1].copy()
        g = gen.from_edges(n, v[:-1], v[1:])
    f, rounds = oracle.fastsv(g)
    assert np.array_equal(f.astype(np.int64), min_label_components(g))
    assert rounds >= 1


def test_fastsv_isolated_and_complete():
    g = gen.from_edges(10, np.array([], dtype=np.int32), np.array([], dtype=np.int32))
    f, _ = oracle.fastsv(g)
    assert np.array_equal(f, np.arange(10))
    f, _ = oracle.fastsv(gen.complete(12))
    assert (f == 0).all()


def test_fastsv_rounds_logarithmic_on_a_path():
    # shortcutting halves the distance to the root: a path of 4096 vertices needs O(log n) rounds
    n = 4096
    g = gen.path(n)
    f, rounds = oracle.fastsv(g)
    assert (f == 0).all()
    assert rounds <= 4 * int(math.log2(n))


# ----------------------------------------------------------------------------------------------
# Delta-stepping SSSP (Alg. 5), float32
# ----------------------------------------------------------------------------------------------

def bellman_ford_f32(g, w, src):
    """Least fixed point of t(v) = min(t(v), fl32(t(u) + w(u,v))), by repeated full relaxation."""
    t = np.full(g.n, np.inf, dtype=np.float32)
    t[src] = 0
    rows, cols = entries(g)
    while True:
        cand = (t[rows] + w).astype(np.float32)
        new = t.copy()
        np.minimum.at(new, cols, cand)
        if np.array_equal(new, t):
            return t
        t = new


def test_sssp_path_prefix_sums():
    # a path has one route: t(k) is the float32 running sum of the weights from the source
    n = 200
    g = gen.with_pair_weights(gen.path(n), seed=9)
    t, _ = oracle.sssp_delta(g, 0, 0.25)
    rows, cols = entries(g)
    step = g.val[(cols == rows + 1)]  # weight of (k, k+1), k ascending
    acc = np.float32(0)
    expect = [acc]
    for x in step:
        acc = np.float32(acc + x)
        expect.append(acc)
    assert np.array_equal(t, np.array(expect, dtype=np.float32))


def test_sssp_unit_weights_are_hop_counts():
    g = gen.rmat(10, 8, seed=2)
    w = np.ones(g.nnz, dtype=np.float32)
    t, _ = oracle.sssp_delta(g, 0, 1.5, weights=w)
    d = csg.shortest_path(csr_scipy(g), unweighted=True, indices=0)
    assert np.array_equal(t, d.astype(np.float32))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sssp_dijkstra_and_fixed_point(seed):
    g = gen.with_pair_weights(gen.erdos_renyi(600, 5.0, seed=seed), seed=seed)
    src = int(gen.sources(g, 1, seed=seed)[0])
    t, buckets = oracle.sssp_delta(g, src, 0.1)
    d = csg.dijkstra(csr_scipy(g, g.val.astype(np.float64)), indices=src)
    fin = np.isfinite(d)
    assert np.array_equal(np.isfinite(t), fin)
    assert np.abs(t[fin] - d[fin]).max() <= 1e-5 * max(1.0, d[fin].max())
    assert np.array_equal(t, bellman_ford_f32(g, g.val, src))
    assert buckets >= 1


def test_sssp_delta_invariance_and_directed():
    g = gen.with_pair_weights(gen.rmat(10, 16, seed=7), seed=7)
    ref, _ = oracle.sssp_delta(g, 0, 0.05)
    for delta in (0.01, 0.3, 1.0, 1e9):  # 1e9: every edge light, one bucket (Bellman-Ford)
        t, _ = oracle.sssp_delta(g, 0, delta)
        assert np.array_equal(t, ref)
    gd = gen.rmat(9, 8, seed=11, directed=True)
    w = gen.uniform_open0(gd.nnz, 5).astype(np.float32)
    t, _ = oracle.sssp_delta(gd, 0, 0.2, weights=w)
    assert np.array_equal(t, bellman_ford_f32(gd, w, 0))
    d = csg.dijkstra(csr_scipy(gd, w.astype(np.float64)), directed=True, indices=0)
    assert np.array_equal(np.isfinite(t), np.isfinite(d))


# ----------------------------------------------------------------------------------------------
# Batched betweenness centrality (Alg. 3)
# ----------------------------------------------------------------------------------------------

def brute_bc(g, sources):
    """sum over s in sources, t != s, v not in {s, t} of sigma(s,t | v) / sigma(s,t), from
    breadth-first distances and shortest-path counts between all pairs (directed edges u -> v)."""
    A = dense_bool(g)
    n = g.n
    dist = np.full((n, n), -1, dtype=np.int64)
    sig = np.zeros((n, n), dtype=np.float64)
    for s in range(n):
        dist[s, s] = 0
        sig[s, s] = 1.0
        frontier = [s]
        d = 0
        while frontier:
            d += 1
            nxt = []
            for u in frontier:
                for v in np.nonzero(A[u])[0]:
                    if dist[s, v] == -1:
                        dist[s, v] = d
                        nxt.append(v)
                    if dist[s, v] == d:
                        sig[s, v] += sig[s, u]
            frontier = nxt
    c = np.zeros(n)
    for s in sources:
        for t in range(n):
            if t == s or dist[s, t] < 0:
                continue
            for v in range(n):
                if v in (s, t) or dist[s, v] < 0 or dist[v, t] < 0:
                    continue
                if dist[s, v] + dist[v, t] == dist[s, t]:
                    c[v] += sig[s, v] * sig[v, t] / sig[s, t]
    return c


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bc_brute_force_undirected(seed):
    g = gen.random_graph(40, 0.08, seed)
    srcs = [int(s) for s in gen.sources(g, 5, seed=seed)]
    c, _ = oracle.bc(g, srcs)
    np.testing.assert_allclose(c, brute_bc(g, srcs), rtol=1e-12, atol=1e-12)


def test_bc_brute_force_directed_and_duplicates():
    g = gen.random_graph(35, 0.1, 7, directed=True)
    srcs = [0, 3, 3, 17]  # a repeated source counts twice
    c, _ = oracle.bc(g, srcs)
    np.testing.assert_allclose(c, brute_bc(g, srcs), rtol=1e-12, atol=1e-12)


def test_bc_closed_forms():
    n = 30
    # a path from one end: every interior vertex v lies on the paths to the n-1-v vertices beyond it
    c, levels = oracle.bc(gen.path(n), [0])
    expect = np.array([0.0] + [float(n - 1 - v) for v in range(1, n)])
    assert np.array_equal(c, expect) and levels == n - 1
    # a star: from the centre nothing, from a leaf the centre carries the other s - 1 leaves
    s = 12
    c, _ = oracle.bc(gen.star(s), [0])
    assert np.array_equal(c, np.zeros(s + 1))
    c, _ = oracle.bc(gen.star(s), [1])
    assert c[0] == s - 1 and (c[1:] == 0).all()
    # complete graph: every pair adjacent, no vertex in between
    c, _ = oracle.bc(gen.complete(9), [0, 4, 8])
    assert (c == 0).all()
    # a 2 x k grid ladder from a corner: path counts split evenly, dependencies are binomial sums
    g = gen.grid(2, 6)
    c, _ = oracle.bc(g, [0])
    np.testing.assert_allclose(c, brute_bc(g, [0]), rtol=1e-12)


def test_bc_isolated_source():
    g = gen.from_edges(6, np.array([1, 2], dtype=np.int32), np.array([2, 3], dtype=np.int32))
    c, levels = oracle.bc(g, [0])
    assert (c == 0).all() and levels == 0
