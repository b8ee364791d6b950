"""Python binding of liblagr.so, the GB300 masked-semiring graph library.

Argument marshalling only: every function here converts torch tensors to
device pointers, passes the current CUDA stream and calls the C entry point of
the same name declared in ``include/lagr.h``; all graph computation happens in
the library's CUDA kernels.  There is no CPU fallback: importing works without
a GPU (so the library can be inspected), but every call that reaches the device
raises when CUDA or the compiled library is unavailable.

Entry points (same names as the C ABI): ``lagr_graph_new``, ``lagr_graph_free``,
``lagr_graph_check``, ``lagr_property_AT``, ``lagr_tc``, ``lagr_tc_edges``, ``lagr_bfs``,
``lagr_bfs_multi``, ``lagr_bfs_batch64``, ``lagr_bfs_noalloc``, ``lagr_betweenness``,
``lagr_sssp``, ``lagr_connected_components``, ``lagr_pagerank``, ``lagr_pagerank_backward``,
``lagr_batch_plan`` / ``lagr_batch_run`` / ``lagr_batch_free``, plus the
``PageRankFunction`` autograd wrapper.
"""
from __future__ import annotations

import ctypes
import os
import warnings
from typing import Optional, Sequence

from . import build as _build

LIB_PATH = _build.LIB

LAGR_MSG_LEN = 256
LAGR_OK = 0
LAGR_ERR_NULL_POINTER = -1
LAGR_ERR_INVALID_VALUE = -2
LAGR_ERR_INVALID_GRAPH = -3
LAGR_ERR_PROPERTY_MISSING = -4
LAGR_ERR_OUT_OF_MEMORY = -5
LAGR_ERR_CUDA = -6
LAGR_ERR_TIMEOUT = -7
LAGR_ERR_DEVICE_CHECK = -8
LAGR_ERR_TOO_LARGE = -9
LAGR_WARN_NOT_CONVERGED = 1

LAGR_UNDIRECTED = 0
LAGR_DIRECTED = 1
LAGR_TC_AUTO, LAGR_TC_SORT, LAGR_TC_NOSORT = 0, 1, 2
LAGR_BFS_PUSH_ONLY, LAGR_BFS_PULL_ONLY = 1, 2
LAGR_PR_GAP, LAGR_PR_DANGLING, LAGR_PR_WEIGHTED, LAGR_PR_WARM_START = 0, 1, 2, 4


class LagrError(RuntimeError):
    def __init__(self, code: int, msg: str, func: str):
        super().__init__(f"{func} failed with {code}: {msg}")
        self.code = code


class LagrWarning(UserWarning):
    pass


class _GraphStruct(ctypes.Structure):
    """Mirror of lagr_graph_struct (include/lagr.h); the struct is not opaque (Sec. II-A)."""
    _fields_ = [
        ("n", ctypes.c_int32),
        ("nnz", ctypes.c_int64),
        ("kind", ctypes.c_int32),
        ("rowptr", ctypes.c_void_p),
        ("colidx", ctypes.c_void_p),
        ("val", ctypes.c_void_p),
        ("at_rowptr", ctypes.c_void_p),
        ("at_colidx", ctypes.c_void_p),
        ("at_val", ctypes.c_void_p),
        ("at_owned", ctypes.c_int32),
        ("row_degree", ctypes.c_void_p),
        ("u_dplus", ctypes.c_void_p),
        ("u_colidx", ctypes.c_void_p),
        ("u_order", ctypes.c_int32),
        ("a_pattern_is_symmetric", ctypes.c_int32),
        ("ndiag", ctypes.c_int64),
        ("last_levels", ctypes.c_int32),
        ("last_push_levels", ctypes.c_int32),
        ("last_pull_levels", ctypes.c_int32),
        ("last_iters", ctypes.c_int32),
        ("last_resid", ctypes.c_double),
        ("priv", ctypes.c_void_p),
    ]


_G = ctypes.POINTER(_GraphStruct)
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f32 = ctypes.c_float
_str = ctypes.c_char_p

_SIGNATURES = {
    "lagr_version": ([], ctypes.c_char_p),
    "lagr_kernel_launches": ([], ctypes.c_uint64),
    "lagr_timing_enable": ([ctypes.c_int], ctypes.c_int),
    "lagr_timing_read": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)], ctypes.c_int),
    "lagr_timing_reset": ([], ctypes.c_int),
    "lagr_set_allocator": ([_vp, _vp, _vp], ctypes.c_int),
    "lagr_release_memory": ([ctypes.c_uint64, _str], ctypes.c_int),
    "lagr_graph_new": ([ctypes.POINTER(_G), _i32, _i64, _vp, _vp, _vp, _i32, _str], ctypes.c_int),
    "lagr_graph_free": ([ctypes.POINTER(_G), _vp, _str], ctypes.c_int),
    "lagr_delete_properties": ([_G, _vp, _str], ctypes.c_int),
    "lagr_graph_check": ([_G, _vp, _str], ctypes.c_int),
    "lagr_property_AT": ([_G, _vp, _str], ctypes.c_int),
    "lagr_property_row_degree": ([_G, _vp, _str], ctypes.c_int),
    "lagr_tc": ([ctypes.POINTER(ctypes.c_uint64), _G, _i32, _vp, _str], ctypes.c_int),
    "lagr_bfs": ([_vp, _vp, ctypes.POINTER(_i32), _G, _i32, _i32, _vp, _str], ctypes.c_int),
    "lagr_bfs_multi": ([_vp, _vp, _vp, _G, _vp, _i32, _i32, _vp, _str], ctypes.c_int),
    "lagr_bfs_batch64": ([_vp, _G, ctypes.POINTER(_i32), _i32, _vp, _str], ctypes.c_int),
    "lagr_bfs_noalloc": ([_vp, _vp, ctypes.POINTER(_i32), _i32, _i64, _vp, _vp, _i32, _vp, _str], ctypes.c_int),
    "lagr_pagerank": ([_vp, ctypes.POINTER(_i32), _G, _f32, _f32, _i32, _vp, _i32, _vp, _str], ctypes.c_int),
    "lagr_pagerank_backward": ([_vp, _vp, ctypes.POINTER(_i32), _vp, _vp, _G, _f32, _f32, _i32, _vp, _i32, _vp,
                                _str], ctypes.c_int),
    "lagr_batch_plan": ([ctypes.POINTER(_vp), _i32, ctypes.POINTER(_i32), _i32, _i64, _vp, _vp, _f32, _i32, _i32,
                         _str, _vp, _str], ctypes.c_int),
    "lagr_batch_run": ([_vp, _vp, _vp, _vp, _str], ctypes.c_int),
    "lagr_batch_tile": ([ctypes.POINTER(_i32), _vp], ctypes.c_int),
    "lagr_batch_free": ([ctypes.POINTER(_vp), _vp, _str], ctypes.c_int),
    "lagr_debug_tc_capacity": ([_i64, _i64], ctypes.c_int),
    "lagr_tc_edges": ([_vp, ctypes.POINTER(ctypes.c_uint64), _G, _i32, _vp, _str], ctypes.c_int),
    "lagr_betweenness": ([_vp, ctypes.POINTER(_i32), _G, ctypes.POINTER(_i32), _i32, _vp, _str], ctypes.c_int),
    "lagr_sssp": ([_vp, ctypes.POINTER(_i32), _G, _i32, _f32, _vp, _str], ctypes.c_int),
    "lagr_connected_components": ([_vp, ctypes.POINTER(_i32), _G, _vp, _str], ctypes.c_int),
}

_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load liblagr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_2104_01661_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGNATURES)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("liblagr needs a CUDA device; there is no CPU fallback")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(rc: int, msg, func: str):
    text = msg.value.decode(errors="replace") if msg is not None else ""
    if rc < 0:
        raise LagrError(rc, text, func)
    if rc > 0:
        warnings.warn(f"{func}: {text}", LagrWarning, stacklevel=3)
    return rc


def _dev(t, dtype, name):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t


class Graph:
    """A lagr_graph over borrowed device CSR tensors (kept alive by this object)."""

    def __init__(self, rowptr, colidx, val=None, directed: bool = False, stream=None):
        torch = _torch()
        self.rowptr = _dev(rowptr, torch.int32, "rowptr")
        self.colidx = _dev(colidx, torch.int32, "colidx")
        self.val = _dev(val, torch.float32, "val")
        self.n = int(rowptr.numel()) - 1
        self.nnz = int(colidx.numel())
        self.directed = directed
        self._stream = stream
        lib = load_library()
        self.handle = _G()
        msg = ctypes.create_string_buffer(LAGR_MSG_LEN)
        rc = lib.lagr_graph_new(ctypes.byref(self.handle), self.n, self.nnz, _ptr(self.rowptr),
                                _ptr(self.colidx), _ptr(self.val),
                                LAGR_DIRECTED if directed else LAGR_UNDIRECTED, msg)
        _check(rc, msg, "lagr_graph_new")

    @classmethod
    def from_host(cls, g, device="cuda", with_values: bool = True):
        """From a gen.Graph (host numpy CSR)."""
        torch = _torch()
        rp = torch.from_numpy(g.rowptr).to(device)
        ci = torch.from_numpy(g.colidx).to(device)
        val = torch.from_numpy(g.val).to(device) if (with_values and g.val is not None) else None
        return cls(rp, ci, val, directed=g.directed)

    @property
    def struct(self) -> _GraphStruct:
        return self.handle.contents

    def free(self):
        if getattr(self, "handle", None) and self.handle:
            msg = ctypes.create_string_buffer(LAGR_MSG_LEN)
            lib = load_library()
            lib.lagr_graph_free(ctypes.byref(self.handle), _stream(self._stream), msg)
            self.handle = _G()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _msg():
    return ctypes.create_string_buffer(LAGR_MSG_LEN)


def lagr_graph_check(G: Graph, stream=None):
    msg = _msg()
    return _check(load_library().lagr_graph_check(G.handle, _stream(stream), msg), msg, "lagr_graph_check")


def lagr_property_AT(G: Graph, stream=None):
    msg = _msg()
    return _check(load_library().lagr_property_AT(G.handle, _stream(stream), msg), msg, "lagr_property_AT")


def lagr_delete_properties(G: Graph, stream=None):
    msg = _msg()
    return _check(load_library().lagr_delete_properties(G.handle, _stream(stream), msg), msg,
                  "lagr_delete_properties")


def lagr_tc(G: Graph, method: int = LAGR_TC_AUTO, stream=None) -> int:
    """Triangle count (Alg. 6); synchronises the stream."""
    out = ctypes.c_uint64(0)
    msg = _msg()
    _check(load_library().lagr_tc(ctypes.byref(out), G.handle, method, _stream(stream), msg), msg, "lagr_tc")
    return int(out.value)


def lagr_tc_edges(G: Graph, method: int = LAGR_TC_AUTO, c=None, stream=None):
    """Triangle count with C<s(L)> kept (Alg. 6, unfused).  Returns (c uint32-as-int32 [nnz], t)."""
    torch = _torch()
    if c is None:
        c = torch.empty(G.nnz, dtype=torch.int32, device=G.rowptr.device)
    _dev(c, torch.int32, "c")
    if c.numel() < G.nnz:
        raise ValueError(f"c has {c.numel()} elements, the graph {G.nnz} entries")
    t = ctypes.c_uint64(0)
    msg = _msg()
    rc = load_library().lagr_tc_edges(_ptr(c), ctypes.byref(t), G.handle, method, _stream(stream), msg)
    _check(rc, msg, "lagr_tc_edges")
    return c, int(t.value)


def lagr_betweenness(G: Graph, sources: Sequence[int], centrality=None, stream=None):
    """Batched betweenness centrality (Alg. 3) from at most 64 sources, float64.  Returns
    (centrality [n], levels)."""
    torch = _torch()
    if centrality is None:
        centrality = torch.empty(G.n, dtype=torch.float64, device=G.rowptr.device)
    _dev(centrality, torch.float64, "centrality")
    k = len(sources)
    src = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in sources])
    levels = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_betweenness(_ptr(centrality), ctypes.byref(levels), G.handle, src, k,
                                         _stream(stream), msg)
    _check(rc, msg, "lagr_betweenness")
    return centrality, int(levels.value)


def lagr_sssp(G: Graph, src: int, delta: float, dist=None, stream=None):
    """Single-source shortest paths by delta-stepping (Alg. 5) over the graph's float32 values.
    Returns (dist [n] float32, +inf when unreachable; buckets)."""
    torch = _torch()
    if dist is None:
        dist = torch.empty(G.n, dtype=torch.float32, device=G.rowptr.device)
    _dev(dist, torch.float32, "dist")
    b = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_sssp(_ptr(dist), ctypes.byref(b), G.handle, int(src), float(delta), _stream(stream),
                                  msg)
    _check(rc, msg, "lagr_sssp")
    return dist, int(b.value)


def lagr_connected_components(G: Graph, component=None, stream=None):
    """Connected components by FastSV (Alg. 7): component[u] = the smallest id of u's component.
    Returns (component [n] int32, rounds)."""
    torch = _torch()
    if component is None:
        component = torch.empty(G.n, dtype=torch.int32, device=G.rowptr.device)
    _dev(component, torch.int32, "component")
    r = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_connected_components(_ptr(component), ctypes.byref(r), G.handle, _stream(stream), msg)
    _check(rc, msg, "lagr_connected_components")
    return component, int(r.value)


def lagr_bfs(G: Graph, src: int, flags: int = 0, level=None, parent=None, want_level: bool = True,
             want_parent: bool = True, stream=None):
    """Parents BFS (Alg. 1/2).  Returns (level, parent, depth); outputs may be passed in."""
    torch = _torch()
    if want_level and level is None:
        level = torch.empty(G.n, dtype=torch.int32, device=G.rowptr.device)
    if want_parent and parent is None:
        parent = torch.empty(G.n, dtype=torch.int32, device=G.rowptr.device)
    _dev(level, torch.int32, "level")
    _dev(parent, torch.int32, "parent")
    depth = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_bfs(_ptr(level), _ptr(parent), ctypes.byref(depth), G.handle, int(src), flags,
                                 _stream(stream), msg)
    _check(rc, msg, "lagr_bfs")
    return level, parent, int(depth.value)


LAGR_BFS_MULTI_MAX = 64


def lagr_bfs_multi(G: Graph, srcs, flags: int = 0, level=None, parent=None, want_level: bool = True,
                   want_parent: bool = True, stream=None):
    """Independent parents BFS from each of `srcs` (at most 64), interleaved on side streams.
    Returns (level [k, n], parent [k, n], depths); outputs may be passed in."""
    torch = _torch()
    srcs = [int(x) for x in srcs]
    k = len(srcs)
    if want_level and level is None:
        level = torch.empty((k, G.n), dtype=torch.int32, device=G.rowptr.device)
    if want_parent and parent is None:
        parent = torch.empty((k, G.n), dtype=torch.int32, device=G.rowptr.device)
    for t, name in ((level, "level"), (parent, "parent")):
        _dev(t, torch.int32, name)
        if t is not None and tuple(t.shape) != (k, G.n):
            raise ValueError(f"{name} must have shape ({k}, {G.n})")
    src = (ctypes.c_int32 * max(k, 1))(*srcs)
    depth = (ctypes.c_int32 * max(k, 1))()
    msg = _msg()
    rc = load_library().lagr_bfs_multi(_ptr(level), _ptr(parent), depth, G.handle, src, k, flags,
                                       _stream(stream), msg)
    _check(rc, msg, "lagr_bfs_multi")
    return level, parent, [int(depth[i]) for i in range(k)]


LAGR_BFS_NOALLOC_MAX_N = 1 << 21


def lagr_bfs_noalloc(rowptr, colidx, src: int, level, parent, stream=None):
    """Parents BFS for callers that cannot allocate device memory: the caller passes the
    undirected graph's device CSR and the output tensors (either may be None); the library uses
    only its fixed built-in work array (graphs of at most LAGR_BFS_NOALLOC_MAX_N vertices) and
    allocates nothing.  Calls must not overlap on one device.  Returns the depth."""
    torch = _torch()
    _dev(rowptr, torch.int32, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    _dev(level, torch.int32, "level")
    _dev(parent, torch.int32, "parent")
    n = int(rowptr.numel()) - 1
    for t, name in ((colidx, "colidx"), (level, "level"), (parent, "parent")):
        if t is not None and t.device != rowptr.device:
            raise ValueError(f"{name} is on {t.device}, rowptr on {rowptr.device}")
    for t, name in ((level, "level"), (parent, "parent")):
        if t is not None and t.numel() < n:
            raise ValueError(f"{name} has {t.numel()} elements, the graph {n} vertices")
    depth = ctypes.c_int32(0)
    msg = _msg()
    with torch.cuda.device(rowptr.device):  # the built-in work array of rowptr's device
        rc = load_library().lagr_bfs_noalloc(_ptr(level), _ptr(parent), ctypes.byref(depth), n,
                                             int(colidx.numel()), _ptr(rowptr), _ptr(colidx), int(src),
                                             _stream(stream), msg)
    _check(rc, msg, "lagr_bfs_noalloc")
    return int(depth.value)


def lagr_bfs_batch64(G: Graph, sources: Sequence[int], level=None, stream=None):
    """k <= 64 BFS at once; returns level [k, n] (int32)."""
    torch = _torch()
    k = len(sources)
    if level is None:
        level = torch.empty((k, G.n), dtype=torch.int32, device=G.rowptr.device)
    _dev(level, torch.int32, "level")
    src = (ctypes.c_int32 * max(k, 1))(*[int(s) for s in sources])
    msg = _msg()
    rc = load_library().lagr_bfs_batch64(_ptr(level), G.handle, src, k, _stream(stream), msg)
    _check(rc, msg, "lagr_bfs_batch64")
    return level


def lagr_pagerank(G: Graph, damping: float = 0.85, tol: float = 1e-7, itermax: int = 100, teleport=None,
                  flags: int = 0, rank=None, stream=None):
    """PageRank (Alg. 4) in float32.  Returns (rank, iterations)."""
    torch = _torch()
    if rank is None:
        rank = torch.empty(G.n, dtype=torch.float32, device=G.rowptr.device)
    _dev(rank, torch.float32, "rank")
    _dev(teleport, torch.float32, "teleport")
    iters = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_pagerank(_ptr(rank), ctypes.byref(iters), G.handle, damping, tol, itermax,
                                      _ptr(teleport), flags, _stream(stream), msg)
    _check(rc, msg, "lagr_pagerank")
    return rank, int(iters.value)


def lagr_pagerank_backward(G: Graph, dL_drank, rank=None, damping: float = 0.85, tol: float = 1e-7,
                           itermax: int = 100, teleport=None, flags: int = LAGR_PR_WEIGHTED, want_dw: bool = True,
                           want_dteleport: bool = True, stream=None):
    """Adjoint of the weighted PageRank fixed point.  Returns (dL/dw [nnz], dL/dteleport [n], iterations)."""
    torch = _torch()
    dev = G.rowptr.device
    dw = torch.empty(G.nnz, dtype=torch.float32, device=dev) if want_dw else None
    dv = torch.empty(G.n, dtype=torch.float32, device=dev) if want_dteleport else None
    _dev(dL_drank, torch.float32, "dL_drank")
    _dev(rank, torch.float32, "rank")
    _dev(teleport, torch.float32, "teleport")
    iters = ctypes.c_int32(0)
    msg = _msg()
    rc = load_library().lagr_pagerank_backward(_ptr(dw), _ptr(dv), ctypes.byref(iters), _ptr(dL_drank),
                                               _ptr(rank), G.handle, damping, tol, itermax, _ptr(teleport),
                                               flags | LAGR_PR_WEIGHTED, _stream(stream), msg)
    _check(rc, msg, "lagr_pagerank_backward")
    return dw, dv, int(iters.value)


class Batch:
    """lagr_batch_plan / lagr_batch_run over a block-diagonal concatenation of g undirected graphs."""

    def __init__(self, voff, rowptr, colidx, damping: float = 0.85, iters: int = 20, tile: int = 0,
                 tune_cache: Optional[str] = None, stream=None):
        torch = _torch()
        self.rowptr = _dev(rowptr, torch.int32, "rowptr")
        self.colidx = _dev(colidx, torch.int32, "colidx")
        vo = [int(x) for x in voff]
        self.g = len(vo) - 1
        self.N = int(rowptr.numel()) - 1
        self._voff = (ctypes.c_int32 * len(vo))(*vo)
        self._stream = stream
        self.handle = ctypes.c_void_p()
        msg = _msg()
        rc = load_library().lagr_batch_plan(ctypes.byref(self.handle), self.g, self._voff, self.N,
                                            int(colidx.numel()), _ptr(self.rowptr), _ptr(self.colidx), damping,
                                            iters, tile, tune_cache.encode() if tune_cache else None,
                                            _stream(stream), msg)
        _check(rc, msg, "lagr_batch_plan")

    @property
    def tile(self) -> int:
        t = ctypes.c_int32(0)
        load_library().lagr_batch_tile(ctypes.byref(t), self.handle)
        return int(t.value)

    def run(self, ntri=None, rank=None, stream=None):
        """Replay the captured pass; returns (ntri uint64-as-int64 [g], rank float32 [N])."""
        torch = _torch()
        dev = self.rowptr.device
        if ntri is None:
            ntri = torch.empty(self.g, dtype=torch.int64, device=dev)
        if rank is None:
            rank = torch.empty(self.N, dtype=torch.float32, device=dev)
        msg = _msg()
        rc = load_library().lagr_batch_run(_ptr(ntri), _ptr(rank), self.handle, _stream(stream), msg)
        _check(rc, msg, "lagr_batch_run")
        return ntri, rank

    def free(self):
        if getattr(self, "handle", None) and self.handle.value:
            msg = _msg()
            load_library().lagr_batch_free(ctypes.byref(self.handle), _stream(self._stream), msg)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _pagerank_function():
    import torch

    class PageRankFunction(torch.autograd.Function):
        """r = PageRank(W, v) (weighted form, float32) with the hand-written adjoint as backward.

        forward(rowptr, colidx, w, teleport, damping, tol, itermax, flags, directed, adjoint_tol) -> r.
        Gradients flow to the edge weights w (CSR order) and the teleport vector.  Only r is
        saved; the backward solves the transposed fixed point with the same gather kernels, to a
        relative L1 change below adjoint_tol.
        """

        @staticmethod
        def forward(ctx, rowptr, colidx, w, teleport, damping=0.85, tol=1e-7, itermax=100, flags=0,
                    directed=True, adjoint_tol=1e-6):
            G = Graph(rowptr, colidx, w.detach().contiguous(), directed=directed)
            tp = None if teleport is None else teleport.detach().contiguous()
            r, _ = lagr_pagerank(G, damping, tol, itermax, tp, flags | LAGR_PR_WEIGHTED)
            G.free()
            ctx.save_for_backward(rowptr, colidx, w, r, teleport if teleport is not None else r.new_empty(0))
            ctx.has_teleport = teleport is not None
            ctx.cfg = (damping, adjoint_tol, itermax, flags, directed)
            return r

        @staticmethod
        def backward(ctx, grad_r):
            rowptr, colidx, w, r, teleport = ctx.saved_tensors
            damping, tol, itermax, flags, directed = ctx.cfg
            G = Graph(rowptr, colidx, w.detach().contiguous(), directed=directed)
            tp = teleport if ctx.has_teleport else None
            dw, dv, _ = lagr_pagerank_backward(G, grad_r.contiguous().float(), r, damping, tol, itermax, tp,
                                               flags | LAGR_PR_WEIGHTED, want_dw=ctx.needs_input_grad[2],
                                               want_dteleport=ctx.has_teleport and ctx.needs_input_grad[3])
            G.free()
            return None, None, dw, dv, None, None, None, None, None, None

    return PageRankFunction


def pagerank_autograd(rowptr, colidx, w, teleport=None, damping=0.85, tol=1e-7, itermax=100, flags=0,
                      directed=True, adjoint_tol=1e-6):
    """Differentiable weighted PageRank (see PageRankFunction).  The forward stops at an L1 change
    below ``tol`` (Alg. 4), the adjoint at a relative L1 change below ``adjoint_tol``."""
    return _pagerank_function().apply(rowptr, colidx, w, teleport, damping, tol, itermax, flags, directed,
                                      adjoint_tol)


def kernel_launches() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(load_library().lagr_kernel_launches())


TIMED_KERNELS = ("pr_gather", "tc_count_cta", "tc_count_warp", "bfs_push_small", "bfs_push_lb", "bfs_pull")


def timing_enable(on: bool = True) -> None:
    """Record CUDA events around every later launch of the timed hot kernels (or stop)."""
    load_library().lagr_timing_enable(1 if on else 0)


def timing_reset() -> None:
    rc = load_library().lagr_timing_reset()
    if rc < 0:
        raise LagrError(rc, "an event failed", "lagr_timing_reset")


def timing_read(kernel: str):
    """(total device ms, launches) of a timed kernel since the last reset."""
    ms = ctypes.c_double()
    cnt = _i64()
    rc = load_library().lagr_timing_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(cnt))
    if rc < 0:
        raise LagrError(rc, f"unknown kernel {kernel!r} or an event failed", "lagr_timing_read")
    return float(ms.value), int(cnt.value)


def lagr_release_memory(keep_bytes: int = 0) -> None:
    """Trim the library's device memory pools to ``keep_bytes`` of free memory each."""
    msg = _msg()
    _check(load_library().lagr_release_memory(int(keep_bytes), msg), msg, "lagr_release_memory")


def version() -> str:
    return load_library().lagr_version().decode()
