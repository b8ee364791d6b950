"""CUDA path vs the CPU oracle for the kept C<s(L)> of Alg. 6, FastSV (Alg. 7), delta-stepping
SSSP (Alg. 5) and batched betweenness centrality (Alg. 3), through the C ABI.

C values, component labels and shortest-path distances are compared bit-exactly (distances are
the least fixed point of the float32 Bellman equations, reached by any order of relaxations);
betweenness centrality (float64 sums in a different order) within a relative error of 1e-9 of
the largest score.  Cases span several chunks and row blocks, heavy rows, ragged tails, isolated
vertices and unreachable parts.
"""
import numpy as np
import pytest

import gen
import oracle

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


def wheel_star(k):
    """A hub joined to k leaves that form a cycle: k triangles, the hub's row k entries long."""
    leaves = np.arange(1, k + 1, dtype=np.int32)
    src = np.concatenate([np.zeros(k, dtype=np.int32), leaves])
    dst = np.concatenate([leaves, np.roll(leaves, -1)])
    return gen.from_edges(k + 1, src, dst)


# ----------------------------------------------------------------------------------------------
# C<s(L)> kept
# ----------------------------------------------------------------------------------------------

TC_CASES = ["k40", "grid", "rmat12", "rmat14", "er", "wheel_star"]


def tc_case(name):
    return {"k40": lambda: gen.complete(40), "grid": lambda: gen.grid(33, 17),
            "rmat12": lambda: gen.rmat(12, 16), "rmat14": lambda: gen.rmat(14, 16, seed=3),
            "er": lambda: gen.erdos_renyi(20000, 12.0, seed=2), "wheel_star": lambda: wheel_star(9000)}[name]()


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("case", TC_CASES)
def test_tc_edges_matches_oracle(L, case, method):
    # NOSORT on the hub graphs puts anchors in every class: warp (d+ <= 256), CTA (<= 8192) and the
    # global-table class (the wheel's hub has d+ = 9000 on its own labels)
    g = tc_case(case)
    G = dev(L, g)
    c, t = L.lagr_tc_edges(G, method)
    co, to = oracle.tc_edges(g, method)
    assert t == to
    assert np.array_equal(c.cpu().numpy().view(np.uint32), co)
    assert L.lagr_tc(G, method) == to  # the fused count on the same cached orientation


def test_tc_edges_empty_and_after_fused(L):
    g = gen.from_edges(5, np.array([], dtype=np.int32), np.array([], dtype=np.int32))
    c, t = L.lagr_tc_edges(dev(L, g))
    assert t == 0
    g = gen.rmat(12, 16)
    G = dev(L, g)
    t0 = L.lagr_tc(G)                      # orientation built by the fused count first
    c, t = L.lagr_tc_edges(G)
    assert t == t0 and np.array_equal(c.cpu().numpy().view(np.uint32), oracle.tc_edges(g)[0])


# ----------------------------------------------------------------------------------------------
# FastSV
# ----------------------------------------------------------------------------------------------

def cc_case(name):
    if name == "rmat":
        return gen.rmat(14, 4, seed=3)
    if name == "er_sparse":
        return gen.erdos_renyi(50000, 1.1, seed=4)
    if name == "grid":
        return gen.grid(64, 129)
    if name == "path_reversed":
        n = 5000
        v = np.arange(n, dtype=np.int32)[::-1].copy()
        return gen.from_edges(n, v[:-1], v[1:])
    if name == "hubs":   # rows past the row blocks' limit, cut into chunks
        k = 20000
        leaves = np.arange(1, k + 1, dtype=np.int32)
        return gen.from_edges(k + 1 + 50, np.zeros(k, dtype=np.int32) + k, leaves - 1)
    if name == "isolated":
        return gen.from_edges(300, np.array([5, 7], dtype=np.int32), np.array([6, 8], dtype=np.int32))
    raise KeyError(name)


@pytest.mark.parametrize("case", ["rmat", "er_sparse", "grid", "path_reversed", "hubs", "isolated"])
def test_fastsv_matches_oracle(L, case):
    g = cc_case(case)
    G = dev(L, g)
    f, rounds = L.lagr_connected_components(G)
    fo, _ = oracle.fastsv(g)
    assert np.array_equal(f.cpu().numpy(), fo)
    assert rounds >= 1


def test_fastsv_rejects_directed(L):
    g = gen.rmat(8, 8, directed=True)
    with pytest.raises(L.LagrError) as e:
        L.lagr_connected_components(dev(L, g))
    assert e.value.code == L.LAGR_ERR_INVALID_GRAPH


# ----------------------------------------------------------------------------------------------
# delta-stepping SSSP
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case,delta", [("rmat12", 0.05), ("rmat12", 0.3), ("rmat12", 1e9), ("er", 0.1),
                                        ("grid", 0.5), ("rmat16", 0.02), ("hubs", 0.2)])
def test_sssp_matches_oracle(L, case, delta):
    base = {"rmat12": lambda: gen.rmat(12, 16), "er": lambda: gen.erdos_renyi(30000, 6.0, seed=5),
            "grid": lambda: gen.grid(40, 70), "rmat16": lambda: gen.rmat(16, 16, seed=9),
            "hubs": lambda: wheel_star(5000)}[case]()
    g = gen.with_pair_weights(base, seed=11)
    G = dev(L, g)
    src = int(gen.sources(g, 1, seed=3)[0])
    d, buckets = L.lagr_sssp(G, src, delta)
    do, _ = oracle.sssp_delta(g, src, delta)
    assert np.array_equal(d.cpu().numpy(), do)  # bit-exact, +inf where unreachable
    assert buckets >= 1


def test_sssp_directed_unreachable_and_errors(L):
    g = gen.rmat(12, 8, seed=4, directed=True)
    g.val = gen.uniform_open0(g.nnz, 8).astype(np.float32)
    G = dev(L, g)
    for src, delta in ((0, 0.1), (17, 0.5)):
        d, _ = L.lagr_sssp(G, src, delta)
        do, _ = oracle.sssp_delta(g, src, delta)
        dd = d.cpu().numpy()
        assert np.array_equal(dd, do) and np.isinf(dd).any()
    with pytest.raises(L.LagrError):
        L.lagr_sssp(G, g.n, 0.1)
    with pytest.raises(L.LagrError):
        L.lagr_sssp(G, 0, 0.0)
    with pytest.raises(L.LagrError):
        L.lagr_sssp(dev(L, g, values=False), 0, 0.1)


# ----------------------------------------------------------------------------------------------
# batched betweenness centrality
# ----------------------------------------------------------------------------------------------

def bc_close(c_gpu, c_ref, rel=1e-9):
    c_gpu = np.asarray(c_gpu)
    scale = max(np.abs(c_ref).max(), 1.0)
    assert np.abs(c_gpu - c_ref).max() <= rel * scale, np.abs(c_gpu - c_ref).max() / scale


@pytest.mark.parametrize("k", [1, 4, 13, 64])
def test_bc_rmat_matches_oracle(L, k):
    # with at most 8 sources the wide levels of an R-MAT traversal late in the BFS phase take the pull
    # direction (the per-lane kernels for 4 and 8 sources); with more, every level pushes
    g = gen.rmat(12, 16)
    srcs = [int(s) for s in gen.sources(g, k, seed=5)]
    G = dev(L, g)
    c, levels = L.lagr_betweenness(G, srcs)
    co, lo = oracle.bc(g, srcs)
    assert levels == lo
    assert G.struct.last_push_levels >= 1
    assert (G.struct.last_pull_levels >= 1) == (k <= 8)
    bc_close(c.cpu().numpy(), co)


def test_bc_directed_duplicates_isolated(L):
    g = gen.rmat(11, 8, seed=2, directed=True)
    srcs = [0, 5, 5, 100, 2047]
    c, levels = L.lagr_betweenness(dev(L, g), srcs)
    co, lo = oracle.bc(g, srcs)
    assert levels == lo
    bc_close(c.cpu().numpy(), co)
    gi = gen.from_edges(6, np.array([1, 2], dtype=np.int32), np.array([2, 3], dtype=np.int32))
    c, levels = L.lagr_betweenness(dev(L, gi), [0])
    assert levels == 0 and (c.cpu().numpy() == 0).all()


def test_bc_path_grid_and_hubs(L):
    n = 300
    c, levels = L.lagr_betweenness(dev(L, gen.path(n)), [0])
    assert levels == n - 1
    assert np.array_equal(c.cpu().numpy(), np.array([0.0] + [float(n - 1 - v) for v in range(1, n)]))
    for g, srcs in ((gen.grid(30, 45), [0, 77, 1349]), (wheel_star(7000), [0, 1, 3500])):
        c, _ = L.lagr_betweenness(dev(L, g), srcs)
        bc_close(c.cpu().numpy(), oracle.bc(g, srcs)[0])


def test_bc_rejects_bad_sources(L):
    g = gen.rmat(8, 8)
    G = dev(L, g)
    with pytest.raises(L.LagrError):
        L.lagr_betweenness(G, [])
    with pytest.raises(L.LagrError):
        L.lagr_betweenness(G, [0] * 65)
    with pytest.raises(L.LagrError):
        L.lagr_betweenness(G, [g.n])
