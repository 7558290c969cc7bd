"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function include/cellgraph.h declares, rejects
bad arguments before touching a device, and answers workspace-size queries.
Also checks that the product path never reaches the oracle."""
import ctypes
import os
import re

import pytest

from paper_1503_06029_gb300 import build as libbuild
from paper_1503_06029_gb300 import cellgraph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cellgraph.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return cellgraph.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cg_pack_signs", "cg_dedup_cells", "cg_neighbors_h1", "cg_build"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in cellgraph.h but not exported"
    assert set(cellgraph.EXPORTS) <= set(names)


def test_missing_library_raises(tmp_path):
    saved = cellgraph._lib
    cellgraph._lib = None
    try:
        with pytest.raises(cellgraph.CellGraphError):
            cellgraph.load_library(str(tmp_path / "nope.so"))
    finally:
        cellgraph._lib = saved


def test_invalid_arguments_rejected_on_host(lib):
    P = ctypes.c_void_p
    # d = 7 is out of range: rejected before any CUDA call
    st = lib.cg_pack_signs(P(1), 10, 7, P(1), P(1), 16, 64, P(1), None)
    assert st == cellgraph.ERR_INVALID_ARG
    assert b"d must" in lib.cg_last_error()
    st = lib.cg_pack_signs(P(1), 10, 3, P(1), P(1), 16, 48, P(1), None)
    assert st == cellgraph.ERR_INVALID_ARG
    st = lib.cg_pack_signs(P(1), 10, 3, P(1), P(1), 0, 64, P(1), None)
    assert st == cellgraph.ERR_INVALID_ARG
    st = lib.cg_pack_signs(P(1), 10, 3, P(1), P(1), 5000, 64, P(1), None)
    assert st == cellgraph.ERR_INVALID_ARG
    st = lib.cg_pack_signs(None, 10, 3, P(1), P(1), 16, 64, P(1), None)
    assert st == cellgraph.ERR_INVALID_ARG
    need = ctypes.c_size_t(0)
    st = lib.cg_neighbors_h1(P(1), 10, 16, 64, P(1), 10, None, 9, None, ctypes.byref(need), None)
    assert st == cellgraph.ERR_INVALID_ARG
    # ALLPAIRS is quadratic: refused above 2^18 cells, before any CUDA call
    st = lib.cg_neighbors_h1(P(1), (1 << 18) + 1, 16, 64, P(1), 10, None,
                             cellgraph.STRATEGY["allpairs"], None, ctypes.byref(need), None)
    assert st == cellgraph.ERR_INVALID_ARG
    assert b"ALLPAIRS" in lib.cg_last_error()
    st = lib.cg_neighbors_h1(P(1), 1 << 18, 16, 64, P(1), 10, None,
                             cellgraph.STRATEGY["allpairs"], None, ctypes.byref(need), None)
    assert st == 0 and need.value > 0  # the workspace query itself is fine
    st = lib.cg_build(None, P(1), 10, 3, P(1), P(1), 16, 64, P(1), 1, None, P(1), 1, None, None)
    assert st == cellgraph.ERR_INVALID_ARG


@pytest.mark.parametrize("ell", [16, 64, 65, 1024])
def test_workspace_queries(lib, ell):
    need = ctypes.c_size_t(0)
    for n in (0, 1, 1000, 1 << 20):
        st = lib.cg_dedup_cells(ctypes.c_void_p(1), n, ell, 64, None, 0, None, None, None,
                                ctypes.byref(need), None)
        assert st == 0 and need.value > 0
        small = need.value
        st = lib.cg_neighbors_h1(ctypes.c_void_p(1), n, ell, 64, None, 0, None, 0, None,
                                 ctypes.byref(need), None)
        assert st == 0 and need.value > 0
    # workspace grows with n
    lib.cg_dedup_cells(ctypes.c_void_p(1), 10, ell, 64, None, 0, None, None, None,
                       ctypes.byref(need), None)
    assert need.value < small


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1503_06029_gb300")
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pat.search(text), f
                assert "cg_oracle" not in text and "libcgoracle" not in text, f


def test_oracle_and_library_share_no_sources():
    ora = open(os.path.join(ROOT, "oracle", "cg_oracle.cpp")).read()
    assert "#include \"" not in ora  # only standard headers
    for f in os.listdir(os.path.join(ROOT, "paper_1503_06029_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_1503_06029_gb300", "csrc", f)).read()


def test_path_to_follows_parents():
    """cellgraph.path_to walks a BFS parent array back to the source (host
    logic, no device): a path, the source itself, and an unreachable cell."""
    import numpy as np

    parent = np.array([-1, 0, 1, 1, 3, -1, 5], np.int32)  # 0-1-3-4 and 1-2; 5-6 apart
    assert cellgraph.path_to(parent, 0, 4) == [0, 1, 3, 4]
    assert cellgraph.path_to(parent, 0, 2) == [0, 1, 2]
    assert cellgraph.path_to(parent, 0, 0) == [0]
    assert cellgraph.path_to(parent, 0, 6) == []  # its tree ends at 5, not at the source


def test_bfs_arguments_rejected_on_host(lib):
    P = ctypes.c_void_p
    need = ctypes.c_size_t(0)
    assert lib.cg_bfs(P(1), 4, 0, 0, P(1), None, None, None, None, ctypes.byref(need),
                      None) == cellgraph.ERR_INVALID_ARG  # no cells
    assert lib.cg_bfs(P(1), -1, 5, 0, P(1), None, None, None, None, ctypes.byref(need),
                      None) == cellgraph.ERR_INVALID_ARG  # negative edge count
    assert lib.cg_bfs(P(1), 4, 5, 0, P(1), None, None, None, None, ctypes.byref(need),
                      None) == 0 and need.value > 0  # workspace query
    assert lib.cg_bfs(P(1), 4, 5, 9, P(1), None, None, None, P(1), ctypes.byref(need),
                      None) == cellgraph.ERR_INVALID_ARG  # source out of range
