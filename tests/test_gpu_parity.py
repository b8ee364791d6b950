"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Triangle counts and BFS levels are compared bit-exactly; BFS parents are checked for validity
(the any monoid leaves the choice free); PageRank scores (float32) against the float64 oracle
within max-abs 1e-6 plus the relative and L1 bounds of gpu_helpers.pr_close; gradients within
relative error 1e-3.  Sizes span several CTA tiles, heavy rows and ragged tails while the oracle
still finishes in seconds.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import check_parents, pr_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    import paper_2104_01661_gb300 as lagr
    assert torch.cuda.is_available()
    lagr.load_library()
    return lagr


def dev(L, g, values=True):
    return L.Graph.from_host(g, with_values=values)


# ---------------------------------------------------------------------------------------------
# triangle counting
# ---------------------------------------------------------------------------------------------

SMALL = [gen.complete(3), gen.complete(17), gen.complete(40), gen.wheel(4), gen.wheel(33), gen.grid(9, 13),
         gen.star(70), gen.path(9), gen.complete_bipartite(5, 8), gen.binary_tree(100), gen.cycle(3)]


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_small_families(L, method):
    for g in SMALL:
        G = dev(L, g)
        assert L.lagr_tc(G, method) == oracle.tc(g), g.name


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_random_tiny(L, method):
    for seed in range(12):
        g = gen.random_graph(30 + 7 * seed, 0.25, seed=500 + seed)
        assert L.lagr_tc(dev(L, g), method) == oracle.tc(g)


@pytest.mark.parametrize("scale,ef", [(12, 16), (14, 16), (16, 16), (13, 32)])
def test_tc_rmat(L, scale, ef):
    g = gen.rmat(scale, ef, seed=scale * 7 + ef)
    G = dev(L, g)
    t = oracle.tc(g)
    for m in (0, 1, 2):
        assert L.lagr_tc(G, m) == t
    assert L.lagr_tc(G, 0) == t  # cached orientation


def test_tc_config1_golden(L, rmat12):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rmat12_oracle.json")))
    assert L.lagr_tc(dev(L, rmat12)) == gold["triangles"]


def test_tc_erdos_renyi(L):
    g = gen.erdos_renyi(30000, 24, seed=3)
    assert L.lagr_tc(dev(L, g)) == oracle.tc(g)


def test_tc_long_anchor_list(L):
    # without sorting the hub of a wheel keeps its whole rim in U (d+ > 4096): the CTA kernel's
    # binary-search path; sorted, the hub has the largest key and anchors nothing
    for k in (5000, 9000):
        g = gen.wheel(k)
        G = dev(L, g)
        assert L.lagr_tc(G, 2) == k
        assert L.lagr_tc(G, 1) == k


def test_tc_high_degree_chunks(L):
    # a hub of degree 20000 with a dense neighbourhood: CTA items split its neighbours into chunks
    rng_src = []
    rng_dst = []
    hub = 0
    for v in range(1, 20001):
        rng_src.append(hub)
        rng_dst.append(v)
    for v in range(1, 20000, 2):
        rng_src.append(v)
        rng_dst.append(v + 1)
    g = gen.from_edges(20001, np.array(rng_src), np.array(rng_dst))
    assert L.lagr_tc(dev(L, g)) == oracle.tc(g) == 10000


def test_tc_empty_and_trivial(L):
    import torch
    for n in (1, 5, 64):
        g = gen.Graph(n=n, rowptr=np.zeros(n + 1, np.int32), colidx=np.zeros(0, np.int32))
        G = L.Graph(torch.zeros(n + 1, dtype=torch.int32, device="cuda"),
                    torch.zeros(1, dtype=torch.int32, device="cuda")[:0])
        assert L.lagr_tc(G) == 0


def test_tc_relabel_invariance(L):
    g = gen.rmat(14, 16, seed=9)
    t = L.lagr_tc(dev(L, g))
    perm = np.argsort(gen.uniform_open0(g.n, 4)).astype(np.int32)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    gp = gen.from_edges(g.n, perm[rows], perm[g.colidx])
    assert L.lagr_tc(dev(L, gp)) == t == oracle.tc(g)


# ---------------------------------------------------------------------------------------------
# BFS
# ---------------------------------------------------------------------------------------------

def run_bfs(L, g, G, src, flags=0):
    level, parent, depth = L.lagr_bfs(G, int(src), flags)
    level, parent = level.cpu().numpy(), parent.cpu().numpy()
    olevel, _, odepth = oracle.bfs(g, int(src))
    assert np.array_equal(level, olevel)
    assert depth == odepth
    check_parents(g, level, parent, int(src))
    return level


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_bfs_config1(L, rmat12, flags):
    G = dev(L, rmat12)
    run_bfs(L, rmat12, G, 0, flags)
    for s in gen.sources(rmat12, 5, seed=1):
        run_bfs(L, rmat12, G, s, flags)


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_bfs_rmat_larger(L, flags):
    g = gen.rmat(16, 16, seed=5)
    G = dev(L, g)
    for s in gen.sources(g, 4, seed=2):
        run_bfs(L, g, G, s, flags)
    st = G.struct
    assert st.last_levels >= 1


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_bfs_directed(L, flags):
    g = gen.rmat(13, 8, seed=11, directed=True)
    G = dev(L, g)
    for s in gen.sources(g, 4, seed=3):
        run_bfs(L, g, G, s, flags)


def test_bfs_grid_many_levels(L):
    g = gen.grid(300, 211)
    G = dev(L, g)
    r, c = np.divmod(np.arange(g.n), 211)
    level = run_bfs(L, g, G, 0)
    assert np.array_equal(level, r + c)
    run_bfs(L, g, G, 150 * 211 + 100, 0)
    run_bfs(L, g, G, 7, 2)


def test_bfs_path_and_special(L):
    g = gen.path(5000)
    G = dev(L, g)
    assert np.array_equal(run_bfs(L, g, G, 0), np.arange(5000))
    two = gen.concat([gen.path(50), gen.cycle(70), gen.star(40)])
    G2 = dev(L, two)
    for s in (0, 60, 125):
        run_bfs(L, two, G2, s)
    gi = gen.rmat(10, 4, seed=2)
    iso = int(np.nonzero(gi.degree() == 0)[0][0])
    lvl = run_bfs(L, gi, dev(L, gi), iso)
    assert (lvl >= 0).sum() == 1


def test_bfs_erdos_renyi_pull_heavy(L):
    g = gen.erdos_renyi(200003, 8, seed=4)
    G = dev(L, g)
    run_bfs(L, g, G, 17)
    assert G.struct.last_pull_levels >= 1


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_bfs_multi_matches_single(L, rmat12, flags):
    # independent traversals interleaved on side streams: duplicates, an isolated source, more
    # sources than side streams
    G = dev(L, rmat12)
    iso = int(np.nonzero(rmat12.degree() == 0)[0][0]) if (rmat12.degree() == 0).any() else 0
    srcs = [int(x) for x in gen.sources(rmat12, 17, seed=31)] + [iso, 5, 5]
    lv, par, depths = L.lagr_bfs_multi(G, srcs, flags)
    lv, par = lv.cpu().numpy(), par.cpu().numpy()
    for t, s in enumerate(srcs):
        olevel, _, odepth = oracle.bfs(rmat12, s)
        assert np.array_equal(lv[t], olevel), t
        assert depths[t] == odepth
        check_parents(rmat12, lv[t], par[t], s)


def test_bfs_multi_directed_and_limits(L):
    import torch
    g = gen.rmat(13, 8, seed=11, directed=True)
    G = dev(L, g)
    srcs = [int(x) for x in gen.sources(g, 3, seed=4)]
    lv, par, depths = L.lagr_bfs_multi(G, srcs)
    for t, s in enumerate(srcs):
        olevel, _, odepth = oracle.bfs(g, s)
        assert np.array_equal(lv[t].cpu().numpy(), olevel) and depths[t] == odepth
        check_parents(g, lv[t].cpu().numpy(), par[t].cpu().numpy(), s)
    ge = gen.erdos_renyi(5000, 6, seed=9)
    Ge = dev(L, ge)
    srcs = list(range(0, 5000, 79))[:64]  # the maximum k
    lv, par, _ = L.lagr_bfs_multi(Ge, srcs, want_parent=False)
    assert par is None and lv.shape == (64, 5000)
    for t in (0, 31, 63):
        assert np.array_equal(lv[t].cpu().numpy(), oracle.bfs(ge, srcs[t])[0])
    _, par1, d1 = L.lagr_bfs_multi(Ge, [17], want_level=False)
    check_parents(ge, oracle.bfs(ge, 17)[0], par1[0].cpu().numpy(), 17)
    assert d1[0] == oracle.bfs(ge, 17)[2]
    # the caller's stream: the results are there once the call returns on a side stream of torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lv2, _, _ = L.lagr_bfs_multi(Ge, [3, 4], stream=s)
    s.synchronize()
    assert np.array_equal(lv2[1].cpu().numpy(), oracle.bfs(ge, 4)[0])


def test_bfs_outputs_optional(L, rmat12):
    G = dev(L, rmat12)
    lvl, par, depth = L.lagr_bfs(G, 0, want_parent=False)
    assert par is None and depth == oracle.bfs(rmat12, 0)[2]
    lvl, par, depth = L.lagr_bfs(G, 0, want_level=False, want_parent=False)
    assert depth == oracle.bfs(rmat12, 0)[2]


def test_bfs_batch64(L, rmat12):
    G = dev(L, rmat12)
    srcs = gen.sources(rmat12, 64, seed=8)
    lv = L.lagr_bfs_batch64(G, srcs).cpu().numpy()
    for i, s in enumerate(srcs):
        assert np.array_equal(lv[i], oracle.bfs(rmat12, int(s))[0])


def test_bfs_batch64_ragged_and_duplicates(L):
    g = gen.erdos_renyi(5000, 6, seed=9)
    G = dev(L, g)
    srcs = [0, 17, 17, 4999, 1234, 5, 6]
    lv = L.lagr_bfs_batch64(G, srcs).cpu().numpy()
    for i, s in enumerate(srcs):
        assert np.array_equal(lv[i], oracle.bfs(g, s)[0])
    lv1 = L.lagr_bfs_batch64(G, [33]).cpu().numpy()
    assert np.array_equal(lv1[0], oracle.bfs(g, 33)[0])


# ---------------------------------------------------------------------------------------------
# PageRank
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dangling", [False, True])
def test_pagerank_config1(L, rmat12, dangling):
    G = dev(L, rmat12)
    flags = L.LAGR_PR_DANGLING if dangling else 0
    r, it = L.lagr_pagerank(G, 0.85, 1e-7, 100, flags=flags)
    ro, ito, _ = oracle.pagerank(rmat12, 0.85, 1e-7, 100, dangling)
    pr_close(r.cpu().numpy(), ro)
    assert abs(it - ito) <= 2
    if dangling:
        assert abs(float(r.double().sum()) - 1.0) < 1e-5


@pytest.mark.parametrize("dangling", [False, True])
def test_pagerank_directed(L, dangling):
    g = gen.rmat(14, 8, seed=21, directed=True)
    G = dev(L, g)
    r, _ = L.lagr_pagerank(G, 0.85, 1e-7, 100, flags=L.LAGR_PR_DANGLING if dangling else 0)
    ro, _, _ = oracle.pagerank(g, 0.85, 1e-7, 100, dangling)
    pr_close(r.cpu().numpy(), ro)


@pytest.mark.parametrize("directed,dangling", [(False, False), (True, True)])
def test_pagerank_rmat16_and_er(L, directed, dangling):
    # many warp items and heavy-row chunks per gather; twice on one graph (cached row plans), then
    # a graph of short rows only
    g = gen.rmat(16, 16, seed=61, directed=directed)
    G = dev(L, g)
    flags = L.LAGR_PR_DANGLING if dangling else 0
    ro, ito, _ = oracle.pagerank(g, 0.85, 1e-7, 100, dangling)
    for _ in range(2):
        r, it = L.lagr_pagerank(G, 0.85, 1e-7, 100, flags=flags)
        pr_close(r.cpu().numpy(), ro)
        assert abs(it - ito) <= 2
    ge = gen.erdos_renyi(40000, 6, seed=62)
    r, _ = L.lagr_pagerank(dev(L, ge), 0.85, 1e-7, 100)
    pr_close(r.cpu().numpy(), oracle.pagerank(ge, 0.85, 1e-7, 100)[0])


def test_pagerank_fixed_iterations_and_heavy_rows(L):
    g = gen.concat([gen.star(9000), gen.rmat(12, 16, seed=3)])   # a row longer than the CTA threshold
    G = dev(L, g)
    r, it = L.lagr_pagerank(G, 0.85, 0.0, 20)
    ro, ito, _ = oracle.pagerank(g, 0.85, 0.0, 20)
    assert it == ito == 20
    pr_close(r.cpu().numpy(), ro)


def test_pagerank_warm_start_and_teleport(L, rmat12):
    import torch
    G = dev(L, rmat12)
    ro, _, _ = oracle.pagerank(rmat12, 0.85, 1e-12, 1000)
    warm = torch.tensor(ro, dtype=torch.float32, device="cuda")
    r, it = L.lagr_pagerank(G, 0.85, 1e-6, 100, flags=L.LAGR_PR_WARM_START, rank=warm)
    assert it <= 3
    pr_close(r.cpu().numpy(), ro)
    v = gen.uniform_open0(rmat12.n, 3)
    v /= v.sum()
    d = np.diff(rmat12.rowptr)
    w = 1.0 / np.repeat(d, d)
    rw, _, _ = oracle.pagerank_weighted(rmat12, w, v, 0.85, 1e-9, 1000, False)
    r2, _ = L.lagr_pagerank(G, 0.85, 1e-7, 200, teleport=torch.tensor(v, dtype=torch.float32, device="cuda"))
    pr_close(r2.cpu().numpy(), rw)


@pytest.mark.parametrize("dangling", [False, True])
def test_pagerank_weighted(L, dangling):
    g = gen.rmat_weighted_directed(13, 16, seed=5)
    G = dev(L, g)
    flags = L.LAGR_PR_WEIGHTED | (L.LAGR_PR_DANGLING if dangling else 0)
    r, _ = L.lagr_pagerank(G, 0.85, 1e-7, 100, flags=flags)
    ro, _, _ = oracle.pagerank_weighted(g, g.meta["val64"], None, 0.85, 1e-7, 100, dangling)
    pr_close(r.cpu().numpy(), ro)


def test_pagerank_regular_is_uniform(L):
    g = gen.cycle(1001)
    r, _ = L.lagr_pagerank(dev(L, g), 0.85, 1e-7, 100)
    assert np.abs(r.cpu().numpy() - 1.0 / 1001).max() < 1e-9


# ---------------------------------------------------------------------------------------------
# PageRank adjoint
# ---------------------------------------------------------------------------------------------

def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dangling", [False, True])
def test_adjoint_vs_oracle(L, dangling):
    import torch
    g = gen.rmat_weighted_directed(12, 16, seed=13)
    w64 = g.meta["val64"]
    G = dev(L, g)
    c = gen.normal(g.n, 99)
    flags = L.LAGR_PR_WEIGHTED | (L.LAGR_PR_DANGLING if dangling else 0)
    r, _ = L.lagr_pagerank(G, 0.85, 1e-7, 200, flags=flags)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    dw, dv, it = L.lagr_pagerank_backward(G, ct, r, 0.85, 1e-6, 300, flags=flags)
    ro, _, _ = oracle.pagerank_weighted(g, w64, None, 0.85, 1e-14, 5000, dangling)
    dwo, dvo, _, _ = oracle.pagerank_adjoint(g, w64, ro, c, None, 0.85, 1e-14, 5000, dangling)
    assert rel_err(dw.cpu().numpy(), dwo) <= 1e-3
    assert np.abs(dw.cpu().numpy() - dwo).max() <= 1e-3 * np.abs(dwo).max()
    assert rel_err(dv.cpu().numpy(), dvo) <= 1e-3
    # recompute path (rank not given)
    dw2, _, _ = L.lagr_pagerank_backward(G, ct, None, 0.85, 1e-6, 300, flags=flags)
    assert rel_err(dw2.cpu().numpy(), dwo) <= 1e-3


def test_adjoint_finite_differences(L):
    import torch
    g = gen.rmat_weighted_directed(10, 16, seed=17)
    w64 = g.meta["val64"]
    c = gen.normal(g.n, 5)
    G = dev(L, g)
    r, _ = L.lagr_pagerank(G, 0.85, 1e-7, 200, flags=L.LAGR_PR_WEIGHTED)
    dw, _, _ = L.lagr_pagerank_backward(G, torch.tensor(c, dtype=torch.float32, device="cuda"), r, 0.85, 1e-7, 300)
    dw = dw.cpu().numpy()
    edges = np.unique((gen.uniform_open0(32, 77) * g.nnz).astype(np.int64))
    fd = []
    for e in edges:
        h = 1e-6 * max(abs(w64[e]), 1e-3)
        wp, wm = w64.copy(), w64.copy()
        wp[e] += h
        wm[e] -= h
        Lp = c @ oracle.pagerank_weighted(g, wp, None, 0.85, 1e-15, 5000)[0]
        Lm = c @ oracle.pagerank_weighted(g, wm, None, 0.85, 1e-15, 5000)[0]
        fd.append((Lp - Lm) / (2 * h))
    fd = np.array(fd)
    assert rel_err(dw[edges], fd) <= 1e-3
    assert np.abs(dw[edges] - fd).max() <= 1e-3 * np.abs(fd).max()


def test_autograd_function_dense_reference(L):
    import torch
    g = gen.rmat_weighted_directed(10, 16, seed=23)
    n = g.n
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    w = torch.tensor(g.val, device="cuda", requires_grad=True)
    v = torch.full((n,), 1.0 / n, device="cuda", requires_grad=True)
    c = torch.tensor(gen.normal(n, 31), dtype=torch.float32, device="cuda")
    r = L.pagerank_autograd(rp, ci, w, v, 0.85, 1e-7, 300)
    (r * c).sum().backward()
    # dense float64 reference: r = (1-a)(I - a W')^-1 v, autograd through a dense solve
    rows = torch.as_tensor(np.repeat(np.arange(n), np.diff(g.rowptr)))
    cols = torch.as_tensor(g.colidx.astype(np.int64))
    wd = torch.tensor(g.meta["val64"], dtype=torch.float64, requires_grad=True)
    vd = torch.full((n,), 1.0 / n, dtype=torch.float64, requires_grad=True)
    W = torch.zeros(n, n, dtype=torch.float64).index_put((rows, cols), wd)
    rd = torch.linalg.solve(torch.eye(n, dtype=torch.float64) - 0.85 * W.T, 0.15 * vd)
    Ld = torch.dot(c.double().cpu(), rd)
    gw, gv = torch.autograd.grad(Ld, (wd, vd))
    assert rel_err(w.grad.cpu().numpy(), gw.numpy()) <= 1e-3
    assert rel_err(v.grad.cpu().numpy(), gv.numpy()) <= 1e-3
    np.testing.assert_allclose(r.detach().cpu().numpy(), rd.detach().numpy(), rtol=0, atol=1e-6)


# ---------------------------------------------------------------------------------------------
# many graphs in one launch
# ---------------------------------------------------------------------------------------------

def test_batch_tc_pagerank(L, tmp_path):
    import torch
    b = gen.rmat_batch(24, seed=3, scale_lo=5, scale_hi=11, ef_lo=4, ef_hi=24)
    parts = b.meta["parts"]
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    cache = str(tmp_path / "tune.json")
    B = L.Batch(b.voff, rp, ci, damping=0.85, iters=20, tile=0, tune_cache=cache)
    assert B.tile >= 32
    for rep in range(2):
        ntri, rank = B.run()
        ntri = ntri.cpu().numpy()
        rank = rank.cpu().numpy()
        for i, p in enumerate(parts):
            assert int(ntri[i]) == oracle.tc(p), i
            ro, _, _ = oracle.pagerank(p, 0.85, 0.0, 20)
            pr_close(rank[b.voff[i]:b.voff[i + 1]], ro)
    # the cached choice is reused
    B2 = L.Batch(b.voff, rp, ci, damping=0.85, iters=20, tile=0, tune_cache=cache)
    assert B2.tile == B.tile
    B3 = L.Batch(b.voff, rp, ci, damping=0.85, iters=3, tile=128)
    ntri3, _ = B3.run()
    assert [int(x) for x in ntri3.cpu()] == [oracle.tc(p) for p in parts]


# ---------------------------------------------------------------------------------------------
# CheckGraph
# ---------------------------------------------------------------------------------------------

def test_graph_check(L, rmat12):
    import torch
    G = dev(L, rmat12)
    L.lagr_graph_check(G)
    assert G.struct.ndiag == 0 and G.struct.a_pattern_is_symmetric == 1
    bad = rmat12.colidx.copy()
    r0, r1 = rmat12.rowptr[0], rmat12.rowptr[1]
    bad[r0], bad[r0 + 1] = bad[r0 + 1], bad[r0]     # unsorted row
    Gb = L.Graph(torch.from_numpy(rmat12.rowptr).cuda(), torch.from_numpy(bad).cuda())
    with pytest.raises(L.LagrError) as e:
        L.lagr_graph_check(Gb)
    assert e.value.code == L.LAGR_ERR_INVALID_GRAPH
    bad2 = rmat12.colidx.copy()
    bad2[-1] = rmat12.n + 5                           # out of range
    Gb2 = L.Graph(torch.from_numpy(rmat12.rowptr).cuda(), torch.from_numpy(bad2).cuda())
    with pytest.raises(L.LagrError):
        L.lagr_graph_check(Gb2)
    d = gen.rmat(10, 8, seed=4, directed=True)       # asymmetric, marked undirected
    Gd = L.Graph(torch.from_numpy(d.rowptr).cuda(), torch.from_numpy(d.colidx).cuda(), directed=False)
    with pytest.raises(L.LagrError):
        L.lagr_graph_check(Gd)
    Gok = L.Graph(torch.from_numpy(d.rowptr).cuda(), torch.from_numpy(d.colidx).cuda(), directed=True)
    L.lagr_graph_check(Gok)
    assert Gok.struct.a_pattern_is_symmetric == 0


def test_bfs_batch64_push_pull_and_heavy_rows(L):
    # a hub of degree 6000 (a row past the row-block limit) joined to an R-MAT graph: the first
    # levels push, the wide ones pull, and the hub's row is scanned by the heavy-row CTAs
    base = gen.rmat(13, 8, seed=41)
    hub = base.n
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    leaves = np.arange(0, 6000 * 2, 2) % base.n
    src = np.concatenate([rows, np.full(leaves.size, hub)])
    dst = np.concatenate([base.colidx, leaves])
    g = gen.from_edges(base.n + 1, src, dst)
    G = dev(L, g)
    for srcs in ([hub], [0, hub, 5], list(gen.sources(g, 64, seed=3)), list(gen.sources(g, 37, seed=4))):
        lv = L.lagr_bfs_batch64(G, [int(x) for x in srcs]).cpu().numpy()
        for i, s in enumerate(srcs):
            assert np.array_equal(lv[i], oracle.bfs(g, int(s))[0]), (i, s)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_tc_beyond_the_rank_window(L, method):
    # more vertices than the CTA kernel's window of ranks (2^17): entries below the window go to
    # the hash table (or, for anchors with none there, need no lookup at all).  Without the degree
    # order (method 2) a power-law hub keeps thousands of low labels and takes the slow scan path,
    # so that case runs on the uniform graph only.
    graphs = [gen.erdos_renyi(300000, 12, seed=6)]
    if method != 2:
        graphs.append(gen.rmat(18, 8, seed=5))
    for g in graphs:
        assert L.lagr_tc(dev(L, g), method) == oracle.tc(g), g.name


def _offset_copy(torch, a, dtype):
    """`a` on the device as a view that starts 4 bytes past a 16-byte boundary."""
    buf = torch.empty(a.size + 1, dtype=dtype, device="cuda")
    buf[1:] = torch.from_numpy(a).to("cuda")
    v = buf[1:]
    assert v.data_ptr() % 16 == 4
    return v


def test_pagerank_misaligned_csr(L):
    # colidx / val not 16-byte aligned: the gather takes its scalar loads; same sums, same order
    import torch
    g = gen.rmat(13, 16, seed=41)
    G = dev(L, g)
    r_al, it_al = L.lagr_pagerank(G, 0.85, 0.0, 15)
    Gm = L.Graph(torch.from_numpy(g.rowptr).to("cuda"), _offset_copy(torch, g.colidx, torch.int32))
    r_mis, it_mis = L.lagr_pagerank(Gm, 0.85, 0.0, 15)
    assert it_al == it_mis == 15
    assert torch.equal(r_al, r_mis)
    ro, _, _ = oracle.pagerank(g, 0.85, 0.0, 15)
    pr_close(r_mis.cpu().numpy(), ro)
    # the adjoint gathers over the rows of W with its values: misaligned colidx and val
    gw = gen.rmat_weighted_directed(11, 16, seed=43)
    w64 = gw.meta["val64"]
    c = gen.normal(gw.n, 7)
    ct = torch.tensor(c, dtype=torch.float32, device="cuda")
    Gw = dev(L, gw)
    Gwm = L.Graph(torch.from_numpy(gw.rowptr).to("cuda"), _offset_copy(torch, gw.colidx, torch.int32),
                  _offset_copy(torch, gw.val, torch.float32), directed=True)
    flags = L.LAGR_PR_WEIGHTED
    r1, _ = L.lagr_pagerank(Gw, 0.85, 0.0, 60, flags=flags)
    r2, _ = L.lagr_pagerank(Gwm, 0.85, 0.0, 60, flags=flags)
    assert torch.equal(r1, r2)
    dw1, dv1, _ = L.lagr_pagerank_backward(Gw, ct, r1, 0.85, 0.0, 80, flags=flags)
    dw2, dv2, _ = L.lagr_pagerank_backward(Gwm, ct, r2, 0.85, 0.0, 80, flags=flags)
    assert torch.equal(dw1, dw2) and torch.equal(dv1, dv2)
    ro, _, _ = oracle.pagerank_weighted(gw, w64, None, 0.85, 1e-14, 5000)
    dwo, _, _, _ = oracle.pagerank_adjoint(gw, w64, ro, c, None, 0.85, 1e-14, 5000)
    assert rel_err(dw2.cpu().numpy(), dwo) <= 1e-3


def test_kernel_timing_counts_launches(L, rmat12):
    import torch
    G = dev(L, rmat12)
    L.timing_reset()
    L.timing_enable(True)
    try:
        _, it = L.lagr_pagerank(G, 0.85, 0.0, 7)
        t = L.lagr_tc(G, L.LAGR_TC_AUTO)
        L.lagr_bfs(G, 0, 0, level=torch.empty(rmat12.n, dtype=torch.int32, device="cuda"))
    finally:
        L.timing_enable(False)
    ms, cnt = L.timing_read("pr_gather")
    assert it == 7 and cnt == 7 and ms > 0.0
    for k in ("tc_count_cta", "tc_count_warp"):
        ms, cnt = L.timing_read(k)
        assert cnt == 1 and ms > 0.0
    assert sum(L.timing_read(k)[1] for k in ("bfs_push_small", "bfs_push_lb", "bfs_pull")) >= 1
    assert t == oracle.tc(rmat12)
    # nothing is recorded once timing is off
    L.timing_reset()
    L.lagr_pagerank(G, 0.85, 0.0, 3)
    assert L.timing_read("pr_gather") == (0.0, 0)


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("n", [3000, 10000, 20000])
def test_tc_sorted_and_unsorted_probe_lists(L, method, n):
    # two hubs joined to each other and to every other vertex: n - 2 triangles.  Without the degree
    # order (NOSORT) the second hub's list U(1) = {2..n-1} is a long probe list: sorted by a whole
    # CTA at n = 3000 and 10000, longer than the rows that are kept sorted at n = 20000 (its probe
    # walk must then run to the end); with the degree order the lists are short.
    v = np.arange(2, n, dtype=np.int64)
    src = np.concatenate([[0], np.zeros_like(v), np.ones_like(v)])
    dst = np.concatenate([[1], v, v])
    g = gen.from_edges(n, src, dst)
    G = dev(L, g)
    assert L.lagr_tc(G, method) == n - 2
    # plus a cycle through the leaves: each cycle edge (v, v+1) closes two more triangles
    src2 = np.concatenate([src, v[:-1]])
    dst2 = np.concatenate([dst, v[1:]])
    g2 = gen.from_edges(n, src2, dst2)
    assert L.lagr_tc(dev(L, g2), method) == (n - 2) + 2 * (n - 3) == oracle.tc(g2)


def test_release_memory_between_graphs(L, rmat12):
    # graphs freed, their pooled memory trimmed, then a new graph allocates again from the pool
    t = oracle.tc(rmat12)
    for keep in (0, 1 << 30):
        G = dev(L, rmat12)
        assert L.lagr_tc(G) == t
        G.free()
        L.lagr_release_memory(keep)
    assert L.lagr_tc(dev(L, rmat12)) == t


@pytest.mark.parametrize("which", ["cta", "warp"])
def test_tc_anchor_list_overflow_is_an_error(L, rmat12, which):
    """The anchor lists of the triangle count have capacities derived from nnz (a bound that holds
    on every symmetric graph).  With a capacity forced below what the graph needs (R-MAT 12 on the
    given labels has 39 CTA items and 17 chunked warp items), the classification skips the writes
    past the end and the count kernels read no further than the capacity: lagr_tc reports
    LAGR_ERR_INVALID_GRAPH, and a later call with the computed capacities is exact again."""
    lib = L.load_library()
    t = oracle.tc(rmat12, oracle.TC_NOSORT)
    try:
        assert lib.lagr_debug_tc_capacity(1 if which == "cta" else 0, 1 if which == "warp" else 0) == 0
        G = dev(L, rmat12)
        with pytest.raises(L.LagrError) as e:
            L.lagr_tc(G, L.LAGR_TC_NOSORT)
        assert e.value.code == L.LAGR_ERR_INVALID_GRAPH
    finally:
        assert lib.lagr_debug_tc_capacity(0, 0) == 0
    assert L.lagr_tc(G, L.LAGR_TC_NOSORT) == t   # the orientation is rebuilt with full capacities
    assert L.lagr_tc(dev(L, rmat12), L.LAGR_TC_NOSORT) == t
    assert lib.lagr_debug_tc_capacity(-1, 0) == L.LAGR_ERR_INVALID_VALUE
