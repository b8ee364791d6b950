"""lagr_bfs_noalloc: the BFS for callers that cannot allocate device memory.

It must give the same levels as lagr_bfs and as the oracle (exact: levels are integers) and valid
parents, on two calls in a row (the built-in work array keeps the previous call's contents, so the
second call checks that everything that must start cleared is cleared), even while every library
allocation is made to fail.  A second graph is chosen so that its traversal takes the wide push
(the warp-per-vertex kernel that only this entry point uses) and both direction changes.  Runs
last (file name) so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import check_parents

pytestmark = pytest.mark.gpu

# the direction rule and the narrow-frontier limits of the BFS (Beamer's rule, alpha 14, beta 24;
# frontiers of at most 8192 vertices and 16384 edges stay in the single-CTA kernel)
ALPHA, BETA, SMALL_MAX, SMALL_EDGES = 14, 24, 8192, 16384


def phases(g, level):
    """The phases the host loop of the allocation-free BFS takes, replayed on the CPU from the
    oracle's levels: 'small' (single-CTA push, possibly several levels), 'push' (wide push) or
    'pull', in order."""
    deg = np.diff(g.rowptr).astype(np.int64)
    depth = int(level.max()) + 1
    nq = np.bincount(level[level >= 0], minlength=depth).astype(np.int64)
    mfl = np.bincount(level[level >= 0], weights=deg[level >= 0], minlength=depth).astype(np.int64)
    seen = np.cumsum(mfl)
    out, pull, prev, lev = [], False, 0, 0
    while lev < depth and nq[lev] > 0:
        q, mf, mu = nq[lev], mfl[lev], g.nnz - seen[lev]
        pull = (q > prev and mf > mu // ALPHA) if not pull else not (q < g.n // BETA)
        prev = q
        if pull:
            out.append("pull")
            lev += 1
        elif q <= SMALL_MAX and mf <= SMALL_EDGES:
            out.append("small")
            first, grow = True, False
            while True:  # the single-CTA kernel's own exit rule
                if lev >= depth or nq[lev] == 0:
                    break
                if not first and (nq[lev] > SMALL_MAX or mfl[lev] > SMALL_EDGES):
                    break
                if not first and grow and mfl[lev] > (g.nnz - seen[lev]) // ALPHA:
                    break
                grow = lev + 1 < depth and nq[lev + 1] > nq[lev]
                lev += 1
                first = False
        else:
            out.append("push")
            lev += 1
    return out


def test_noalloc_bfs_matches_lagr_bfs_twice():
    import torch
    import paper_2104_01661_gb300 as L

    g = gen.rmat(16, 16, seed=77)
    G = L.Graph.from_host(g)
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    srcs = [int(s) for s in gen.sources(g, 2, seed=78)]
    expect = [L.lagr_bfs(G, s) for s in srcs]
    for (lvl, _, _), s in zip(expect, srcs):
        assert np.array_equal(lvl.cpu().numpy(), oracle.bfs(g, s)[0])

    lib = L.load_library()
    alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    calls = []
    failing_alloc = alloc_t(lambda nbytes, stream, ctx: calls.append(nbytes) or None)
    noop_free = free_t(lambda p, stream, ctx: None)
    assert lib.lagr_set_allocator(ctypes.cast(failing_alloc, ctypes.c_void_p),
                                  ctypes.cast(noop_free, ctypes.c_void_p), None) == 0
    try:
        # the allocating path now fails ...
        G2 = L.Graph(rp, ci)
        with pytest.raises(L.LagrError) as e:
            L.lagr_tc(G2)
        assert e.value.code == L.LAGR_ERR_OUT_OF_MEMORY
        n_failed = len(calls)
        assert n_failed >= 1
        # ... while the allocation-free BFS runs, twice in a row, with stale contents in between
        for (lvl_ref, par_ref, depth_ref), s in zip(expect, srcs):
            level = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            parent = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            depth = L.lagr_bfs_noalloc(rp, ci, s, level, parent)
            torch.cuda.synchronize()
            assert depth == depth_ref
            assert torch.equal(level, lvl_ref)
            check_parents(g, level.cpu().numpy(), parent.cpu().numpy(), s)
        assert len(calls) == n_failed          # no allocation was attempted
    finally:
        lib.lagr_set_allocator(None, None, None)


def test_noalloc_bfs_wide_push_matches_oracle():
    """Erdos-Renyi n = 2^20, average degree 8: from a seeded source the frontier grows past the
    single-CTA limits before the pull pays off, so two levels run the wide push (memset of the next
    bitmap, warp-per-vertex push, bitmap as the next frontier), then the pull, then push again."""
    import torch
    import paper_2104_01661_gb300 as L

    g = gen.erdos_renyi(1 << 20, 8, seed=5)
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    for s in [int(x) for x in gen.sources(g, 2, seed=6)]:
        olevel, _, odepth = oracle.bfs(g, s)
        ph = phases(g, olevel)
        assert ph.count("push") >= 2 and "pull" in ph, ph
        assert ph.index("pull") < len(ph) - 1, ph  # a pull -> push switch after the pull phase
        for _ in range(2):  # twice in a row over the stale work array
            level = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            parent = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            depth = L.lagr_bfs_noalloc(rp, ci, s, level, parent)
            lv = level.cpu().numpy()
            assert depth == odepth
            assert np.array_equal(lv, olevel)
            check_parents(g, lv, parent.cpu().numpy(), s)


def test_noalloc_bfs_rejects_oversize_graphs():
    import paper_2104_01661_gb300 as L
    lib = L.load_library()
    msg = ctypes.create_string_buffer(L.LAGR_MSG_LEN)
    fake = ctypes.c_void_p(0x1000)
    n = L.LAGR_BFS_NOALLOC_MAX_N + 1
    rc = lib.lagr_bfs_noalloc(None, None, None, n, 10, fake, fake, 0, None, msg)
    assert rc == L.LAGR_ERR_TOO_LARGE and b"at most" in msg.value
    rc = lib.lagr_bfs_noalloc(None, None, None, 10, 10, fake, fake, 10, None, msg)
    assert rc == L.LAGR_ERR_INVALID_VALUE
