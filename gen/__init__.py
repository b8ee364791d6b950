"""Seeded synthetic graph inputs (shared by the CUDA path's tests/bench and the oracle).

Nothing here computes a triangle count, a traversal or a rank: these functions
only build the graphs and the random vectors the method consumes.  The heavy
lifting (R-MAT descent, CSR build with dedupe) is plain C in ``gen.c``; this
module compiles it on first use and wraps it with ctypes.

Workload recipes (the paper's Table IV graphs are not available; these are the
stand-ins for their shapes):

* ``rmat(scale, ef)``: Graph500-style R-MAT, a/b/c/d = .57/.19/.19/.05,
  ``ef * 2**scale`` draws, symmetrised, self-loops and duplicates removed
  (stand-in for the paper's Kron graph).
* ``erdos_renyi(n, avg_degree)``: ``n * avg_degree / 2`` uniform endpoint pairs,
  symmetrised and deduplicated (stand-in for Urand).
* ``grid(rows, cols)``: 4-neighbour 2D grid (stand-in for the high-diameter
  Road graph).
* ``rmat_weighted_directed(scale, ef)``: directed R-MAT with weights uniform in
  (0, 1] per unique edge, row-normalised in float64 and stored as float32.
* ``rmat_batch(g)``: ``g`` independent R-MAT graphs with scale ~ U{8..16} and
  edge factor ~ U{8..32}, concatenated block-diagonally.
* ``with_pair_weights(g)``: symmetric float32 edge weights uniform in (0, 1]
  (one counter-based draw per unordered vertex pair), for single-source
  shortest paths on an undirected graph.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

DEFAULT_SEED = 20210404
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so next to it (plain gcc, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.gen_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.gen_rmat_edges.restype = None
        lib.gen_uniform_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
        lib.gen_uniform_edges.restype = None
        lib.gen_edges_to_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int,
                                         ctypes.c_int, i32p, i32p]
        lib.gen_edges_to_csr.restype = ctypes.c_int64
        lib.gen_grid_csr.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p]
        lib.gen_grid_csr.restype = ctypes.c_int64
        lib.gen_uniform_open0.argtypes = [ctypes.c_int64, ctypes.c_uint64, f64p]
        lib.gen_uniform_open0.restype = None
        lib.gen_normal.argtypes = [ctypes.c_int64, ctypes.c_uint64, f64p]
        lib.gen_normal.restype = None
        lib.gen_sources.argtypes = [ctypes.c_int32, i32p, ctypes.c_int32, ctypes.c_uint64, i32p]
        lib.gen_sources.restype = ctypes.c_int32
        lib.gen_splitmix64_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gen_splitmix64_draw.restype = ctypes.c_uint64
        lib.gen_pair_weights.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]
        lib.gen_pair_weights.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Graph:
    """Host CSR graph: int32 ``rowptr[n+1]``, int32 ``colidx[nnz]``, optional float32 ``val``."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    directed: bool = False
    val: Optional[np.ndarray] = None
    name: str = ""
    # block-diagonal batches: vertex offsets of each member graph (len g+1)
    voff: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degree(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)


def splitmix64(seed: int, k: int) -> int:
    """Draw k of the counter-mode splitmix64 stream ``seed``."""
    return int(_load().gen_splitmix64_draw(seed & (2**64 - 1), k))


def from_edges(n: int, src, dst, symmetric: bool = True, drop_self: bool = True,
               name: str = "") -> Graph:
    """CSR (sorted rows, no duplicates) from an edge list."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    e = int(src.shape[0])
    rowptr = np.zeros(n + 1, dtype=np.int32)
    colidx = np.empty(max(1, (2 if symmetric else 1) * e), dtype=np.int32)
    nnz = _load().gen_edges_to_csr(n, e, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                   int(symmetric), int(drop_self), _p(rowptr, ctypes.c_int32),
                                   _p(colidx, ctypes.c_int32))
    if nnz < 0:
        raise ValueError("edge endpoint out of range or nnz does not fit int32")
    colidx = colidx[:nnz].copy()
    return Graph(n=n, rowptr=rowptr, colidx=colidx, directed=not symmetric, name=name)


def rmat_edges(scale: int, edgefactor: int, seed: int = DEFAULT_SEED,
               a: float = 0.57, b: float = 0.19, c: float = 0.19):
    ne = edgefactor * (1 << scale)
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    _load().gen_rmat_edges(scale, ne, a, b, c, seed & (2**64 - 1), _p(src, ctypes.c_int32),
                           _p(dst, ctypes.c_int32))
    return src, dst


def rmat(scale: int, edgefactor: int = 16, seed: int = DEFAULT_SEED, directed: bool = False,
         a: float = 0.57, b: float = 0.19, c: float = 0.19) -> Graph:
    src, dst = rmat_edges(scale, edgefactor, seed, a, b, c)
    g = from_edges(1 << scale, src, dst, symmetric=not directed, drop_self=True,
                   name=f"rmat{scale}_ef{edgefactor}{'_dir' if directed else ''}")
    g.meta.update(scale=scale, edgefactor=edgefactor, seed=seed)
    return g


def erdos_renyi(n: int, avg_degree: float = 8.0, seed: int = DEFAULT_SEED) -> Graph:
    ne = int(round(n * avg_degree / 2))
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    _load().gen_uniform_edges(n, ne, seed & (2**64 - 1), _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32))
    g = from_edges(n, src, dst, symmetric=True, drop_self=True, name=f"er{n}_d{avg_degree:g}")
    g.meta.update(avg_degree=avg_degree, seed=seed)
    return g


def grid(rows: int, cols: int) -> Graph:
    n = rows * cols
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cap = 4 * n
    colidx = np.empty(max(cap, 1), dtype=np.int32)
    nnz = _load().gen_grid_csr(rows, cols, _p(rowptr, ctypes.c_int32), _p(colidx, ctypes.c_int32))
    return Graph(n=n, rowptr=rowptr, colidx=colidx[:nnz].copy(), name=f"grid{rows}x{cols}",
                 meta=dict(rows=rows, cols=cols))


def uniform_open0(count: int, seed: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gen_uniform_open0(count, seed & (2**64 - 1), _p(out, ctypes.c_double))
    return out


def normal(count: int, seed: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gen_normal(count, seed & (2**64 - 1), _p(out, ctypes.c_double))
    return out


def row_normalized_weights(g: Graph, seed: int) -> np.ndarray:
    """Weights uniform in (0,1] per stored entry (CSR order), each row scaled to sum 1 in float64."""
    w = uniform_open0(g.nnz, seed)
    deg = np.diff(g.rowptr).astype(np.int64)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    s = np.zeros(g.n, dtype=np.float64)
    np.add.at(s, rows, w)
    return w / s[rows]


def rmat_weighted_directed(scale: int, edgefactor: int = 16, seed: int = DEFAULT_SEED) -> Graph:
    g = rmat(scale, edgefactor, seed, directed=True)
    w64 = row_normalized_weights(g, seed ^ 0x5EED_0F_3E16)
    g.val = w64.astype(np.float32)
    g.meta["val64"] = w64
    g.name = f"rmat{scale}_ef{edgefactor}_dir_w"
    return g


def with_pair_weights(g: Graph, seed: int = DEFAULT_SEED) -> Graph:
    """g with float32 values uniform in (0, 1], equal on (i, j) and (j, i)."""
    val = np.empty(max(g.nnz, 1), dtype=np.float32)
    _load().gen_pair_weights(g.n, _p(g.rowptr, ctypes.c_int32), _p(g.colidx, ctypes.c_int32),
                             (seed ^ 0x55A9) & (2**64 - 1), _p(val, ctypes.c_float))
    out = Graph(n=g.n, rowptr=g.rowptr, colidx=g.colidx, directed=g.directed, val=val[:g.nnz].copy(),
                name=g.name + "_w", voff=g.voff, meta=dict(g.meta))
    return out


def sources(g: Graph, k: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """k distinct seeded random vertices with a non-empty row."""
    out = np.empty(k, dtype=np.int32)
    got = _load().gen_sources(g.n, _p(g.rowptr, ctypes.c_int32), k, seed & (2**64 - 1),
                              _p(out, ctypes.c_int32))
    return out[:got].copy()


def rmat_batch(g: int = 512, seed: int = DEFAULT_SEED, scale_lo: int = 8, scale_hi: int = 16,
               ef_lo: int = 8, ef_hi: int = 32) -> Graph:
    """g independent undirected R-MAT graphs concatenated block-diagonally.

    Member i has scale U{scale_lo..scale_hi} and edge factor U{ef_lo..ef_hi}
    (draws 2i and 2i+1 of the stream ``seed``) and its own R-MAT seed
    (draw 2g+i).  ``voff`` holds the vertex offsets of the members.
    """
    scales, efs, parts = [], [], []
    for i in range(g):
        s = scale_lo + splitmix64(seed, 2 * i) % (scale_hi - scale_lo + 1)
        ef = ef_lo + splitmix64(seed, 2 * i + 1) % (ef_hi - ef_lo + 1)
        parts.append(rmat(s, ef, splitmix64(seed, 2 * g + i)))
        scales.append(s)
        efs.append(ef)
    return concat(parts, name=f"rmat_batch{g}", meta=dict(scales=scales, efs=efs, seed=seed))


def concat(parts, name: str = "", meta: Optional[dict] = None) -> Graph:
    """Block-diagonal concatenation of undirected graphs (ids shifted by vertex offsets)."""
    voff = np.zeros(len(parts) + 1, dtype=np.int64)
    eoff = np.zeros(len(parts) + 1, dtype=np.int64)
    for i, p in enumerate(parts):
        voff[i + 1] = voff[i] + p.n
        eoff[i + 1] = eoff[i] + p.nnz
    if eoff[-1] >= 2**31 or voff[-1] >= 2**31:
        raise ValueError("batch too large for int32 CSR")
    N = int(voff[-1])
    rowptr = np.empty(N + 1, dtype=np.int32)
    colidx = np.empty(int(eoff[-1]), dtype=np.int32)
    rowptr[0] = 0
    for i, p in enumerate(parts):
        rowptr[voff[i] + 1: voff[i + 1] + 1] = p.rowptr[1:] + eoff[i]
        colidx[eoff[i]: eoff[i + 1]] = p.colidx + voff[i]
    out = Graph(n=N, rowptr=rowptr, colidx=colidx, name=name, voff=voff.astype(np.int32),
                meta=dict(meta or {}))
    out.meta["parts"] = parts
    return out


# ---- small deterministic fixtures (closed-form pins) -------------------------------------------

def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, name=f"K{n}")


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"P{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"C{n}")


def star(s: int) -> Graph:
    """K_{1,s}: centre 0, leaves 1..s."""
    leaves = np.arange(1, s + 1)
    return from_edges(s + 1, np.zeros(s, dtype=np.int64), leaves, name=f"star{s}")


def wheel(k: int) -> Graph:
    """Hub 0 joined to every vertex of the cycle 1..k."""
    c = np.arange(1, k + 1)
    src = np.concatenate([np.zeros(k, dtype=np.int64), c])
    dst = np.concatenate([c, 1 + (c % k)])
    return from_edges(k + 1, src, dst, name=f"wheel{k}")


def complete_bipartite(p: int, q: int) -> Graph:
    a, b = np.meshgrid(np.arange(p), p + np.arange(q), indexing="ij")
    return from_edges(p + q, a.ravel(), b.ravel(), name=f"K{p},{q}")


def binary_tree(n: int) -> Graph:
    v = np.arange(1, n)
    return from_edges(n, (v - 1) // 2, v, name=f"tree{n}")


def random_graph(n: int, p: float, seed: int, directed: bool = False) -> Graph:
    """G(n, p) from counter-mode draws over all ordered/unordered pairs (small n only)."""
    rng_src, rng_dst = [], []
    k = 0
    for i in range(n):
        for j in range((0 if directed else i + 1), n):
            if i == j:
                continue
            u = (splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)
            k += 1
            if u < p:
                rng_src.append(i)
                rng_dst.append(j)
    return from_edges(n, np.array(rng_src, dtype=np.int32), np.array(rng_dst, dtype=np.int32),
                      symmetric=not directed, name=f"gnp{n}_{p}")
