"""ORACLE -- test infrastructure, not part of the product.

ctypes wrapper around ``oracle.c``: a plain single-threaded C99 restatement of
triangle counting (Alg. 6, fused and with C<s(L)> kept), parents BFS (Alg. 1),
PageRank (Alg. 4, float64, GAP form plus the dangling-redistribution variant),
weighted PageRank and its adjoint, batched betweenness centrality (Alg. 3,
float64), delta-stepping shortest paths (Alg. 5, float32) and FastSV connected
components (Alg. 7).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the CUDA library never does, and the
two share no code.

Every function takes a host CSR graph (``gen.Graph`` or the three arrays) and
returns numpy arrays / Python ints.

Pins: every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, brute force and library routines (see that file's docstrings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TC_AUTO, TC_SORT, TC_NOSORT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c (single-threaded, no vector or arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32 = ctypes.c_int32
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_tc.argtypes = [i32, i32p, i32p, ctypes.c_int]
        lib.oracle_tc.restype = ctypes.c_uint64
        lib.oracle_tc_sample.argtypes = [i32, i32p, i32p, ctypes.c_int, i32, ctypes.POINTER(ctypes.c_int64),
                                         f64p]
        lib.oracle_tc_sample.restype = ctypes.c_uint64
        lib.oracle_tc_wants_sort.argtypes = [i32, i32p, f64p, ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_tc_wants_sort.restype = ctypes.c_int
        lib.oracle_bfs.argtypes = [i32, i32p, i32p, i32, i32p, i32p]
        lib.oracle_bfs.restype = i32
        lib.oracle_pagerank.argtypes = [i32, i32p, i32p, ctypes.c_double, ctypes.c_double, i32,
                                        ctypes.c_int, f64p, f64p]
        lib.oracle_pagerank.restype = i32
        lib.oracle_pagerank_weighted.argtypes = [i32, i32p, i32p, f64p, f64p, ctypes.c_double,
                                                 ctypes.c_double, i32, ctypes.c_int, f64p, f64p]
        lib.oracle_pagerank_weighted.restype = i32
        lib.oracle_pagerank_adjoint.argtypes = [i32, i32p, i32p, f64p, f64p, f64p, f64p,
                                                ctypes.c_double, ctypes.c_double, i32, ctypes.c_int,
                                                f64p, f64p, f64p]
        lib.oracle_pagerank_adjoint.restype = i32
        lib.oracle_tc_edges.argtypes = [i32, i32p, i32p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
        lib.oracle_tc_edges.restype = ctypes.c_uint64
        lib.oracle_fastsv.argtypes = [i32, i32p, i32p, i32p]
        lib.oracle_fastsv.restype = i32
        lib.oracle_sssp_delta.argtypes = [i32, i32p, i32p, ctypes.POINTER(ctypes.c_float), i32, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_float)]
        lib.oracle_sssp_delta.restype = i32
        lib.oracle_bc.argtypes = [i32, i32p, i32p, i32, i32p, f64p]
        lib.oracle_bc.restype = i32
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _csr(g):
    rp, prp = _i32(g.rowptr)
    ci, pci = _i32(g.colidx if len(g.colidx) else np.zeros(1, np.int32))
    return g.n, rp, prp, ci, pci


def tc(g, method: int = TC_AUTO) -> int:
    """Triangle count by Alg. 6 (method: 0 as the paper, 1 always sort, 2 never sort)."""
    n, rp, prp, ci, pci = _csr(g)
    t = _load().oracle_tc(n, prp, pci, method)
    if t == 2**64 - 1:
        raise MemoryError("oracle_tc")
    return int(t)


def tc_sample(g, method: int = TC_AUTO, stride: int = 1):
    """Alg. 6 restricted to mask rows 0, stride, 2*stride, ... of L: (partial count, mask entries
    visited, seconds spent in the masked product)."""
    n, rp, prp, ci, pci = _csr(g)
    ent = ctypes.c_int64()
    sec = ctypes.c_double()
    t = _load().oracle_tc_sample(n, prp, pci, method, stride, ctypes.byref(ent), ctypes.byref(sec))
    if t == 2**64 - 1:
        raise MemoryError("oracle_tc_sample")
    return int(t), int(ent.value), float(sec.value)


def tc_edges(g, method: int = TC_AUTO):
    """(c, t): the unfused form of Alg. 6 -- c[e] (uint32, CSR order of g) is the value of
    C<s(L)> = L plus.pair U' at the stored entry e when e lies in L after the degree ordering
    (0 otherwise), t = sum(c)."""
    n, rp, prp, ci, pci = _csr(g)
    c = np.zeros(max(g.nnz, 1), dtype=np.uint32)
    t = _load().oracle_tc_edges(n, prp, pci, method, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if t == 2**64 - 1:
        raise MemoryError("oracle_tc_edges")
    return c[:g.nnz], int(t)


def fastsv(g):
    """(f, rounds): connected components by Alg. 7 (FastSV); f[u] = the smallest vertex id of u's
    component."""
    n, rp, prp, ci, pci = _csr(g)
    f = np.empty(max(n, 1), dtype=np.int32)
    k = _load().oracle_fastsv(n, prp, pci, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if k < 0:
        raise MemoryError("oracle_fastsv")
    return f[:n], int(k)


def sssp_delta(g, src: int, delta: float, weights=None):
    """(t, buckets): single-source shortest paths by Alg. 5 (delta-stepping) in float32 arithmetic;
    t[v] = +inf where v is unreachable.  weights: float32 [nnz] (default g.val)."""
    n, rp, prp, ci, pci = _csr(g)
    w = np.ascontiguousarray(g.val if weights is None else weights, dtype=np.float32)
    if w.size == 0:
        w = np.zeros(1, dtype=np.float32)
    t = np.empty(max(n, 1), dtype=np.float32)
    k = _load().oracle_sssp_delta(n, prp, pci, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(src),
                                  float(delta), t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if k < 0:
        raise ValueError("oracle_sssp_delta: bad source or delta, or out of memory")
    return t[:n], int(k)


def bc(g, sources):
    """(centrality, levels): batched betweenness centrality by Alg. 3 in float64 from the given
    sources; centrality[j] = sum over the sources s of the dependency of s on j."""
    n, rp, prp, ci, pci = _csr(g)
    src, psrc = _i32(np.asarray(sources, dtype=np.int32))
    c = np.empty(max(n, 1), dtype=np.float64)
    k = _load().oracle_bc(n, prp, pci, len(src), psrc, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if k < 0:
        raise ValueError("oracle_bc: bad source or out of memory")
    return c[:n], int(k)


def tc_wants_sort(g):
    """(decision, mean, median) of the degree heuristic of Alg. 6."""
    n, rp, prp, _, _ = _csr(g)
    mean = ctypes.c_double()
    med = ctypes.c_int64()
    d = _load().oracle_tc_wants_sort(n, prp, ctypes.byref(mean), ctypes.byref(med))
    return bool(d), mean.value, med.value


def bfs(g, src: int):
    """(level, parent, depth) by the parents BFS of Alg. 1 (push over A's rows)."""
    n, rp, prp, ci, pci = _csr(g)
    level = np.empty(max(n, 1), dtype=np.int32)
    parent = np.empty(max(n, 1), dtype=np.int32)
    depth = _load().oracle_bfs(n, prp, pci, int(src), level.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if depth < 0:
        raise ValueError("oracle_bfs: bad source")
    return level[:n], parent[:n], int(depth)


def pagerank(g, damping: float = 0.85, tol: float = 1e-7, itermax: int = 100, dangling: bool = False):
    """(r, iterations, last residual) by Alg. 4 in float64 (plus.second, edge values ignored)."""
    n, rp, prp, ci, pci = _csr(g)
    r = np.empty(max(n, 1), dtype=np.float64)
    res = ctypes.c_double()
    k = _load().oracle_pagerank(n, prp, pci, damping, tol, itermax, int(dangling),
                                r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(res))
    if k < 0:
        raise MemoryError("oracle_pagerank")
    return r[:n], int(k), res.value


def pagerank_weighted(g, val, v=None, damping: float = 0.85, tol: float = 1e-7, itermax: int = 100,
                      dangling: bool = False):
    """(r, iterations, last residual) of r = (1-a) v + a W' r [+ a (dangling mass) v]."""
    n, rp, prp, ci, pci = _csr(g)
    val, pval = _f64(val)
    v, pv = _f64(v)
    r = np.empty(max(n, 1), dtype=np.float64)
    res = ctypes.c_double()
    k = _load().oracle_pagerank_weighted(n, prp, pci, pval, pv, damping, tol, itermax, int(dangling),
                                         r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(res))
    if k < 0:
        raise MemoryError("oracle_pagerank_weighted")
    return r[:n], int(k), res.value


def pagerank_adjoint(g, val, r, c, v=None, damping: float = 0.85, tol: float = 1e-14,
                     itermax: int = 1000, dangling: bool = False):
    """(dL/dW in CSR order, dL/dv, lambda, iterations) for L = c . r at the fixed point r."""
    n, rp, prp, ci, pci = _csr(g)
    val, pval = _f64(val)
    v, pv = _f64(v)
    r, pr = _f64(r)
    c, pc = _f64(c)
    dW = np.empty(max(g.nnz, 1), dtype=np.float64)
    dv = np.empty(max(n, 1), dtype=np.float64)
    lam = np.empty(max(n, 1), dtype=np.float64)
    P = ctypes.POINTER(ctypes.c_double)
    k = _load().oracle_pagerank_adjoint(n, prp, pci, pval, pv, pr, pc, damping, tol, itermax,
                                        int(dangling), dW.ctypes.data_as(P), dv.ctypes.data_as(P),
                                        lam.ctypes.data_as(P))
    if k < 0:
        raise MemoryError("oracle_pagerank_adjoint")
    return dW[:g.nnz], dv[:n], lam[:n], int(k)
