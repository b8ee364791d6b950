"""lagr_bfs_noalloc: the BFS for callers that cannot allocate device memory.

It must give the same levels as lagr_bfs (exact: levels are integers) and valid parents, on two
calls in a row (the built-in work array keeps the previous call's contents, so the second call
checks that everything that must start cleared is cleared), even while every library allocation
is made to fail.  Runs last (file name) so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

import gen
from gpu_helpers import check_parents

pytestmark = pytest.mark.gpu


def test_noalloc_bfs_matches_lagr_bfs_twice():
    import torch
    import paper_2104_01661_gb300 as L

    g = gen.rmat(16, 16, seed=77)
    G = L.Graph.from_host(g)
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    srcs = [int(s) for s in gen.sources(g, 2, seed=78)]
    expect = [L.lagr_bfs(G, s) for s in srcs]

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
