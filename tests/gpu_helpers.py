"""Shared helpers of the GPU parity tests (no oracle arithmetic here)."""
import numpy as np


def check_parents(g, level, parent, src):
    """BFS parents are valid: parent[v] >= 0 <=> level[v] >= 0, parent[src] = src, and for every
    other reached v the edge (parent[v], v) is stored and level[parent[v]] = level[v] - 1."""
    level = np.asarray(level)
    parent = np.asarray(parent)
    assert parent[src] == src and level[src] == 0
    assert np.array_equal(parent >= 0, level >= 0)
    reached = np.nonzero((level > 0))[0]
    if reached.size == 0:
        return
    u = parent[reached]
    assert (u >= 0).all() and (u < g.n).all()
    assert np.array_equal(level[u], level[reached] - 1)
    # (u, v) stored: binary search of v in row u
    rp, ci = g.rowptr.astype(np.int64), g.colidx
    lo, hi = rp[u], rp[u + 1]
    for _ in range(40):
        mid = (lo + hi) // 2
        go = (mid < hi) & (ci[np.minimum(mid, len(ci) - 1)] < reached)
        lo = np.where(go, mid + 1, lo)
        hi = np.where(go, hi, mid)
    assert ((lo < rp[u + 1]) & (ci[np.minimum(lo, len(ci) - 1)] == reached)).all()


def pr_close(r_gpu, r_ref, atol=1e-6, rel=1e-4, l1=1e-5):
    """PageRank tolerance: max-abs <= 1e-6 per score, and, because that bound is vacuous for
    scores far below 1e-6, max|diff| / max(r_ref) <= rel and sum|diff| <= l1 (absolute, the scores
    summing to at most 1)."""
    r_gpu = np.asarray(r_gpu, dtype=np.float64)
    d = np.abs(r_gpu - r_ref)
    assert d.max() <= atol, d.max()
    assert d.max() / max(np.abs(r_ref).max(), 1e-300) <= rel, d.max() / np.abs(r_ref).max()
    assert d.sum() <= l1, d.sum()
