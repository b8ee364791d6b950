"""The C ABI without a GPU: the library loads, exports every entry point include/lagr.h declares,
the ctypes mirror of lagr_graph_struct matches the C layout, and argument validation that happens
before any device work returns the documented codes and messages."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2104_01661_gb300 as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lagr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2104_01661_gb300 import build
    build.build()
    return L.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lagr_[A-Za-z0-9_]+)\s*\(", text)) - {"lagr_alloc_fn", "lagr_free_fn"})


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(L.exported_symbols())
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lagr_\w+)", out))
    assert set(names) <= exported


def test_version(lib):
    assert "sm_103a" in L.version()


def test_struct_layout_matches_c(tmp_path):
    fields = [f for f, _ in L._GraphStruct._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"lagr.h\"\nint main(void){\n"
                   "printf(\"%zu\\n\", sizeof(lagr_graph_struct));\n" +
                   "".join(f"printf(\"%zu\\n\", offsetof(lagr_graph_struct, {f}));\n" for f in fields) +
                   "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == ctypes.sizeof(L._GraphStruct)
    for f, off in zip(fields, vals[1:]):
        assert getattr(L._GraphStruct, f).offset == off, f


def _new(lib, n, nnz, rp, ci, kind=L.LAGR_UNDIRECTED):
    G = L._G()
    msg = ctypes.create_string_buffer(L.LAGR_MSG_LEN)
    rc = lib.lagr_graph_new(ctypes.byref(G), n, nnz, rp, ci, None, kind, msg)
    return rc, G, msg.value.decode()


FAKE = ctypes.c_void_p(0x1000)  # never dereferenced: these calls fail validation first


def test_graph_new_validation(lib):
    msg = ctypes.create_string_buffer(L.LAGR_MSG_LEN)
    assert lib.lagr_graph_new(None, 1, 0, FAKE, FAKE, None, 0, msg) == L.LAGR_ERR_NULL_POINTER
    assert _new(lib, -1, 0, FAKE, FAKE)[0] == L.LAGR_ERR_INVALID_VALUE
    assert _new(lib, 4, -5, FAKE, FAKE)[0] == L.LAGR_ERR_INVALID_VALUE
    rc, _, text = _new(lib, 4, 2**31, FAKE, FAKE)
    assert rc == L.LAGR_ERR_TOO_LARGE and "int32" in text
    assert _new(lib, 4, 4, FAKE, FAKE, kind=7)[0] == L.LAGR_ERR_INVALID_VALUE
    assert _new(lib, 4, 4, None, FAKE)[0] == L.LAGR_ERR_NULL_POINTER
    rc, G, text = _new(lib, 4, 4, FAKE, FAKE)
    assert rc == 0 and text == ""
    s = G.contents
    assert (s.n, s.nnz, s.kind, s.ndiag, s.u_order) == (4, 4, 0, -1, -1)
    assert s.a_pattern_is_symmetric == 1 and not s.at_rowptr
    assert lib.lagr_graph_free(ctypes.byref(G), None, msg) == 0
    assert not G


def test_entry_point_validation(lib):
    msg = ctypes.create_string_buffer(L.LAGR_MSG_LEN)
    _, G, _ = _new(lib, 4, 4, FAKE, FAKE)
    _, D, _ = _new(lib, 4, 4, FAKE, FAKE, kind=L.LAGR_DIRECTED)
    out = ctypes.c_uint64()
    assert lib.lagr_tc(None, G, 0, None, msg) == L.LAGR_ERR_NULL_POINTER
    assert lib.lagr_tc(ctypes.byref(out), G, 9, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_tc(ctypes.byref(out), D, 0, None, msg) == L.LAGR_ERR_INVALID_GRAPH
    assert b"undirected" in msg.value
    assert lib.lagr_bfs(None, None, None, G, 4, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs(None, None, None, G, -1, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs(None, None, None, G, 0, 3, None, msg) == L.LAGR_ERR_INVALID_VALUE
    src = (ctypes.c_int32 * 2)(0, 1)
    assert lib.lagr_bfs_multi(None, None, None, G, None, 2, 0, None, msg) == L.LAGR_ERR_NULL_POINTER
    assert lib.lagr_bfs_multi(None, None, None, G, src, 0, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs_multi(None, None, None, G, src, 65, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs_multi(None, None, None, G, src, 2, 3, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs_multi(None, None, None, G, (ctypes.c_int32 * 2)(0, 4), 2, 0, None, msg) == \
        L.LAGR_ERR_INVALID_VALUE
    assert b"out of range" in msg.value
    assert lib.lagr_bfs_batch64(FAKE, G, src, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs_batch64(FAKE, G, src, 65, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_bfs_batch64(FAKE, D, src, 2, None, msg) == L.LAGR_ERR_INVALID_GRAPH
    bad = (ctypes.c_int32 * 2)(0, 9)
    assert lib.lagr_bfs_batch64(FAKE, G, bad, 2, None, msg) == L.LAGR_ERR_INVALID_VALUE
    it = ctypes.c_int32()
    for damping in (0.0, 1.0, -0.5, float("nan")):
        assert lib.lagr_pagerank(FAKE, ctypes.byref(it), G, damping, 1e-7, 10, None, 0, None, msg) == \
            L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_pagerank(None, None, G, 0.85, 1e-7, 10, None, 0, None, msg) == L.LAGR_ERR_NULL_POINTER
    assert lib.lagr_pagerank(FAKE, None, G, 0.85, -1.0, 10, None, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_pagerank(FAKE, None, G, 0.85, 1e-7, 0, None, 0, None, msg) == L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_pagerank(FAKE, None, G, 0.85, 1e-7, 10, None, 64, None, msg) == L.LAGR_ERR_INVALID_VALUE
    # weighted form without values
    assert lib.lagr_pagerank(FAKE, None, G, 0.85, 1e-7, 10, None, L.LAGR_PR_WEIGHTED, None, msg) == \
        L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_pagerank_backward(None, None, None, None, None, G, 0.85, 1e-7, 10, None, 2, None, msg) == \
        L.LAGR_ERR_NULL_POINTER
    assert lib.lagr_pagerank_backward(None, None, None, FAKE, None, G, 0.85, 1e-7, 10, None, 0, None, msg) == \
        L.LAGR_ERR_INVALID_VALUE
    B = ctypes.c_void_p()
    voff = (ctypes.c_int32 * 3)(0, 2, 2)
    assert lib.lagr_batch_plan(ctypes.byref(B), 2, voff, 2, 2, FAKE, FAKE, 0.85, 5, 0, None, None, msg) == \
        L.LAGR_ERR_INVALID_VALUE
    voff = (ctypes.c_int32 * 3)(0, 1, 3)
    assert lib.lagr_batch_plan(ctypes.byref(B), 2, voff, 2, 2, FAKE, FAKE, 0.85, 5, 0, None, None, msg) == \
        L.LAGR_ERR_INVALID_VALUE
    assert lib.lagr_set_allocator(FAKE, None, None) == L.LAGR_ERR_NULL_POINTER
    assert lib.lagr_graph_free(ctypes.byref(G), None, msg) == 0
    assert lib.lagr_graph_free(ctypes.byref(D), None, msg) == 0


def test_binding_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA"):
        L.Graph(torch.zeros(2, dtype=torch.int32), torch.zeros(1, dtype=torch.int32))


def test_timing_api_host_side(lib):
    import ctypes
    ms, cnt = ctypes.c_double(-1.0), ctypes.c_int64(-1)
    assert lib.lagr_timing_reset() == 0
    assert lib.lagr_timing_read(b"no_such_kernel", ctypes.byref(ms), ctypes.byref(cnt)) == -2
    assert lib.lagr_timing_read(None, ctypes.byref(ms), ctypes.byref(cnt)) == -1
    for name in (b"pr_gather", b"tc_count_cta", b"tc_count_warp", b"bfs_push_small", b"bfs_push_lb", b"bfs_pull"):
        assert lib.lagr_timing_read(name, ctypes.byref(ms), ctypes.byref(cnt)) == 0
        assert ms.value == 0.0 and cnt.value == 0
    assert lib.lagr_timing_enable(1) == 0 and lib.lagr_timing_enable(0) == 0


def test_release_memory_without_pools(lib):
    msg = ctypes.create_string_buffer(L.LAGR_MSG_LEN)
    msg.value = b"stale"
    assert lib.lagr_release_memory(0, msg) == 0 and msg.value == b""
    assert lib.lagr_release_memory(1 << 40, None) == 0


def test_every_declaration_cites_its_passage():
    # each entry point's comment names the passage of the paper that defines it (or says there is none)
    text = open(HEADER).read()
    pat = re.compile(r"(/\*(?:(?!\*/).)*\*/)\s*(?:#define[^\n]*\n\s*)*((?:typedef[^;]*;\s*)*)"
                     r"(?:[A-Za-z_][\w \*]*?)\b(lagr_[A-Za-z0-9_]+)\s*\(", re.S)
    seen = {}
    for m in pat.finditer(text):
        comment = re.sub(r"\s*\n\s*\*\s*", " ", m.group(1))
        seen[m.group(3)] = bool(re.search(r"Alg\. ?\d|Sec\. ?[IVX]|Table [IVX]|no (paper )?counterpart", comment,
                                          re.I))
    assert len(seen) >= 15
    assert all(seen.values()), [k for k, v in seen.items() if not v]
