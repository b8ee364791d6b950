"""Parity at the full benchmark sizes, in the configuration bench.py times.

Where the single-threaded oracle finishes in seconds (BFS, a fixed number of PageRank iterations,
the adjoint) the GPU result is compared element by element; the triangle count of the scale-22
R-MAT (minutes of oracle time) is compared with the oracle's count stored in
tests/golden/rmat22_oracle.json by tests/golden/make_golden.py, and is also checked for invariance
under relabelling and under the choice of orientation.
"""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import check_parents, pr_close

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEED = 20210404
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rmat22_oracle.json")


def golden22():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def L():
    import torch
    import paper_2104_01661_gb300 as lagr
    assert torch.cuda.is_available()
    lagr.load_library()
    return lagr


@pytest.fixture(scope="module")
def rmat22():
    return gen.rmat(22, 16, seed=SEED)


def test_rmat22_bfs_16_sources(L, rmat22):
    """All 16 bench sources through lagr_bfs_multi (the call bench.py times), every level array
    against the oracle element by element, every parent array checked; the oracle's depths and
    level histograms also match the stored golden values."""
    g = rmat22
    G = L.Graph.from_host(g)
    srcs = [int(s) for s in gen.sources(g, 16, seed=SEED)]
    assert len(set(srcs)) == 16
    gold = golden22()
    assert gold["nnz"] == g.nnz and gold["sources"] == srcs
    lv, par, depths = L.lagr_bfs_multi(G, srcs)
    lv = lv.cpu().numpy()
    par = par.cpu().numpy()
    for i, s in enumerate(srcs):
        olevel, _, odepth = oracle.bfs(g, s)
        assert odepth == gold["bfs"][i]["depth"]
        assert np.bincount(olevel[olevel >= 0]).tolist() == gold["bfs"][i]["level_histogram"]
        assert np.array_equal(lv[i], olevel), i
        assert depths[i] == odepth
        check_parents(g, lv[i], par[i], s)
    # lagr_bfs (one source per call) on a sample, against the same oracle levels
    for i in (0, 7, 15):
        level, parent, depth = L.lagr_bfs(G, srcs[i])
        assert np.array_equal(level.cpu().numpy(), lv[i]) and depth == depths[i]


def test_rmat22_tc_golden_and_invariants(L, rmat22):
    g = rmat22
    G = L.Graph.from_host(g)
    t_auto = L.lagr_tc(G, L.LAGR_TC_AUTO)
    gold = golden22()
    assert gold["nnz"] == g.nnz
    assert t_auto == gold["triangles"]  # the oracle's count (Alg. 6 as written, method AUTO)
    assert L.lagr_tc(G, L.LAGR_TC_SORT) == t_auto
    assert oracle.tc_wants_sort(g)[0]          # Alg. 6 sorts this graph
    G.free()
    perm = np.argsort(gen.uniform_open0(g.n, 12345)).astype(np.int32)
    rows = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.rowptr))
    gp = gen.from_edges(g.n, perm[rows], perm[g.colidx])
    Gp = L.Graph.from_host(gp)
    assert L.lagr_tc(Gp, L.LAGR_TC_AUTO) == t_auto
    assert t_auto > 0


def test_rmat22_pagerank_fixed_iterations(L, rmat22):
    g = rmat22
    G = L.Graph.from_host(g)
    r, it = L.lagr_pagerank(G, 0.85, 0.0, 12)
    ro, ito, _ = oracle.pagerank(g, 0.85, 0.0, 12)
    assert it == ito == 12
    pr_close(r.cpu().numpy(), ro)


def test_er_and_grid_bfs_pagerank(L):
    er = gen.erdos_renyi(1 << 23, 8, seed=SEED)
    G = L.Graph.from_host(er)
    for s in gen.sources(er, 2, seed=SEED):
        level, parent, _ = L.lagr_bfs(G, int(s))
        level = level.cpu().numpy()
        assert np.array_equal(level, oracle.bfs(er, int(s))[0])
        check_parents(er, level, parent.cpu().numpy(), int(s))
    r, _ = L.lagr_pagerank(G, 0.85, 0.0, 10)
    pr_close(r.cpu().numpy(), oracle.pagerank(er, 0.85, 0.0, 10)[0])
    G.free()
    del er
    grid = gen.grid(4096, 4096)
    Gg = L.Graph.from_host(grid)
    level, parent, depth = L.lagr_bfs(Gg, 0)
    r_, c_ = np.divmod(np.arange(grid.n), 4096)
    level = level.cpu().numpy()
    assert np.array_equal(level, r_ + c_) and depth == 8191
    check_parents(grid, level, parent.cpu().numpy(), 0)
    r, _ = L.lagr_pagerank(Gg, 0.85, 0.0, 10)
    pr_close(r.cpu().numpy(), oracle.pagerank(grid, 0.85, 0.0, 10)[0])


def test_rmat20_batch64(L):
    g = gen.rmat(20, 16, seed=SEED)
    G = L.Graph.from_host(g)
    srcs = gen.sources(g, 64, seed=SEED)
    lv = L.lagr_bfs_batch64(G, srcs).cpu().numpy()
    for i in (0, 21, 63):
        assert np.array_equal(lv[i], oracle.bfs(g, int(srcs[i]))[0])
    for i in range(0, 64, 9):
        lp, _, _ = L.lagr_bfs(G, int(srcs[i]))
        assert np.array_equal(lv[i], lp.cpu().numpy())


def test_rmat20_weighted_adjoint(L):
    import torch
    g = gen.rmat_weighted_directed(20, 16, seed=SEED)
    G = L.Graph.from_host(g)
    c = gen.normal(g.n, SEED)
    flags = L.LAGR_PR_WEIGHTED
    r, _ = L.lagr_pagerank(G, 0.85, 1e-7, 100, flags=flags)
    ro, _, _ = oracle.pagerank_weighted(g, g.meta["val64"], None, 0.85, 1e-12, 1000)
    pr_close(r.cpu().numpy(), ro)
    dw, dv, _ = L.lagr_pagerank_backward(G, torch.tensor(c, dtype=torch.float32, device="cuda"), r, 0.85, 1e-6, 300)
    dwo, dvo, _, _ = oracle.pagerank_adjoint(g, g.meta["val64"], ro, c, None, 0.85, 1e-12, 1000)
    dw = dw.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(dw - dwo) <= 1e-3 * np.linalg.norm(dwo)
    assert np.abs(dw - dwo).max() <= 1e-3 * np.abs(dwo).max()
    dv = dv.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(dv - dvo) <= 1e-3 * np.linalg.norm(dvo)


def test_batch512_matches_plain_calls(L):
    import torch
    b = gen.rmat_batch(512, seed=SEED)
    parts = b.meta["parts"]
    B = L.Batch(b.voff, torch.from_numpy(b.rowptr).cuda(), torch.from_numpy(b.colidx).cuda(), 0.85, 20)
    ntri, rank = B.run()
    ntri = ntri.cpu().numpy()
    rank = rank.cpu().numpy()
    for i, p in enumerate(parts):
        Gi = L.Graph.from_host(p)
        assert int(ntri[i]) == L.lagr_tc(Gi), i
        ri, _ = L.lagr_pagerank(Gi, 0.85, 0.0, 20)
        pr_close(rank[b.voff[i]:b.voff[i + 1]], ri.cpu().numpy().astype(np.float64), atol=1e-6, rel=1e-4, l1=1e-5)
        Gi.free()
    for i in range(0, 512, 97):   # oracle on a sample of the members
        assert int(ntri[i]) == oracle.tc(parts[i])
        ro, ito, _ = oracle.pagerank(parts[i], 0.85, 0.0, 20)
        assert ito == 20
        pr_close(rank[b.voff[i]:b.voff[i + 1]], ro)


# ----------------------------------------------------------------------------------------------
# the next rows at the sizes bench.py measures them (R-MAT 22 with pair weights; kept C at R-MAT 20,
# whose oracle takes seconds, and at R-MAT 22 against the stored oracle count)
# ----------------------------------------------------------------------------------------------

def test_rmat22_fastsv_sssp_bc(L, rmat22):
    g = gen.with_pair_weights(rmat22, seed=SEED)
    G = L.Graph.from_host(g)
    f, _ = L.lagr_connected_components(G)
    fo, _ = oracle.fastsv(rmat22)
    assert np.array_equal(f.cpu().numpy(), fo)
    src = int(gen.sources(g, 1, seed=SEED)[0])
    for delta in (0.1, 0.2):  # the deltas the bench tries
        d, _ = L.lagr_sssp(G, src, delta)
        assert np.array_equal(d.cpu().numpy(), oracle.sssp_delta(g, src, delta)[0])
    srcs = [int(s) for s in gen.sources(g, 4, seed=SEED)]
    c, levels = L.lagr_betweenness(G, srcs)
    co, lo = oracle.bc(rmat22, srcs)
    assert levels == lo
    c = c.cpu().numpy()
    assert np.abs(c - co).max() <= 1e-9 * max(np.abs(co).max(), 1.0)


def test_kept_c_rmat19_and_rmat22(L, rmat22):
    g = gen.rmat(19, 16, seed=SEED)
    G = L.Graph.from_host(g)
    c, t = L.lagr_tc_edges(G)
    co, to = oracle.tc_edges(g)
    assert t == to and np.array_equal(c.cpu().numpy().view(np.uint32), co)
    G.free()
    G22 = L.Graph.from_host(rmat22)
    c22, t22 = L.lagr_tc_edges(G22)
    assert t22 == golden22()["triangles"]
    c22 = c22.cpu().numpy().view(np.uint32)
    assert int(c22.sum(dtype=np.uint64)) == t22
    # the U side of every edge holds 0; the L side of each triangle's first-last edge its count
    deg = np.diff(rmat22.rowptr).astype(np.int64)
    rank = np.empty(rmat22.n, dtype=np.int64)
    rank[np.lexsort((np.arange(rmat22.n), deg))] = np.arange(rmat22.n)
    rows = np.repeat(np.arange(rmat22.n, dtype=np.int64), deg)
    assert (c22[rank[rows] < rank[rmat22.colidx]] == 0).all()
