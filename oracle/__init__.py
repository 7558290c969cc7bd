"""CPU oracle for the cell-graph hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never touches it, and it shares no code with them.

The arithmetic lives in ``cg_oracle.cpp`` (plain single-threaded C++17); this
module compiles it with g++ on first use and marshals numpy arrays through
ctypes. Every function follows the paper "Massively Parallel Construction of
the Cell Graph":

* ``pack_signs``  §2.1 / Figure 1: bit i = [a_i . p >= b_i], exact.
* ``pack_signs_quadric``  §2.1 with curved boundaries: bit i = [q_i(p) +
                  a_i . p >= b_i], q_i an integer quadratic form, exact.
* ``dedup``       §3.2: sort the vectors and drop duplicates.
* ``neighbors``   §2.2 definition of G_X, searched as in Algorithm 4
                  (flip one bit, look the result up).
* ``heuristic``   §3.1, Algorithms 1-2: pivot distances, inequality (⋆),
                  segment-wise comparison of the remaining pairs.
* ``tree``        §3.2, Algorithms 3-4: the 2^r-ary search tree and its walk.
* ``bfs``         §6 (paths in the cell graph): textbook queue BFS distances.
* ``build``       the three steps for one scene.

Pins (tests that tie these functions to something other than themselves) are in
``tests/test_oracle_pins.py``; none of the functions is left unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.cpp")
_LIB = os.path.join(_HERE, "libcgoracle.so")
_lock = threading.Lock()
_lib = None


def compile_library(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libcgoracle.so`` (g++, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(compile_library())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            lib.cgo_pack_signs.argtypes = [P, I64, I, P, P, I, I, P]
            lib.cgo_pack_signs_quadric.argtypes = [P, I64, I, P, P, P, I, I, P]
            lib.cgo_dedup.argtypes = [P, I64, I, I, P, P, P]
            lib.cgo_neighbors_h1_rows.argtypes = [P, I64, I, I, P, I64, P, I64, P]
            lib.cgo_neighbors_h1.argtypes = [P, I64, I, I, P, I64, P]
            lib.cgo_tree.argtypes = [P, I64, I, I, I, I, P, I, P, I64, P]
            lib.cgo_tree_digits.argtypes = [P, I64, I, I, I, I, P]
            lib.cgo_heuristic.argtypes = [P, I64, I, I, I, I, I, P, I64, P, P]
            lib.cgo_bfs.argtypes = [P, I64, I64, I64, P]
            for f in (lib.cgo_pack_signs, lib.cgo_pack_signs_quadric, lib.cgo_dedup, lib.cgo_neighbors_h1_rows,
                      lib.cgo_neighbors_h1, lib.cgo_tree, lib.cgo_tree_digits,
                      lib.cgo_heuristic, lib.cgo_bfs):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def words(ell: int, word_bits: int) -> int:
    return (ell + word_bits - 1) // word_bits


def _wtype(word_bits: int):
    if word_bits == 64:
        return np.uint64
    if word_bits == 32:
        return np.uint32
    raise ValueError("word_bits must be 32 or 64")


def _ptr(x: np.ndarray):
    return ctypes.c_void_p(x.ctypes.data)


def pack_signs(pts, a, b, word_bits: int = 64) -> np.ndarray:
    """Packed sign vectors, shape [N, ceil(l/word_bits)] of uint32/uint64."""
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int64)
    n, d = pts.shape
    ell = a.shape[0]
    assert a.shape[1] == d and b.shape == (ell,)
    keys = np.zeros((n, words(ell, word_bits)), dtype=_wtype(word_bits))
    rc = lib.cgo_pack_signs(_ptr(pts), n, d, _ptr(a), _ptr(b), ell, word_bits, _ptr(keys))
    if rc:
        raise RuntimeError(f"cgo_pack_signs failed: {rc}")
    return keys


def pack_signs_quadric(pts, q, a, b, word_bits: int = 64) -> np.ndarray:
    """Packed sign vectors of quadric constraints (bit i = [sum_{j<=k}
    q[i, jk] p_j p_k + a[i] . p >= b[i]], exact), shape [N, ceil(l/word_bits)].
    ``q`` int32 [l, d(d+1)/2]: monomial coefficients, (j, k) with j <= k in
    row-major order."""
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int64)
    n, d = pts.shape
    ell = a.shape[0]
    assert a.shape[1] == d and b.shape == (ell,) and q.shape == (ell, d * (d + 1) // 2)
    keys = np.zeros((n, words(ell, word_bits)), dtype=_wtype(word_bits))
    rc = lib.cgo_pack_signs_quadric(_ptr(pts), n, d, _ptr(q), _ptr(a), _ptr(b), ell, word_bits,
                                    _ptr(keys))
    if rc:
        raise RuntimeError(f"cgo_pack_signs_quadric failed: {rc}")
    return keys


def build_quadric(pts, q, a, b, word_bits: int = 64):
    """(cells, edges) of one scene of quadric constraints."""
    keys = pack_signs_quadric(pts, q, a, b, word_bits)
    ell = np.asarray(a).shape[0]
    cells = dedup(keys, ell, word_bits)
    return cells, neighbors(cells, ell, word_bits)


def dedup(keys, ell: int, word_bits: int = 64, point_cell: bool = False):
    """Sorted unique cells [U, W]; with ``point_cell`` also the cell number of
    every input vector."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=_wtype(word_bits))
    n = keys.shape[0]
    w = words(ell, word_bits)
    assert keys.shape == (n, w)
    cells = np.zeros((max(n, 1), w), dtype=keys.dtype)
    nc = ctypes.c_int64(0)
    pc = np.zeros(max(n, 1), dtype=np.uint32) if point_cell else None
    rc = lib.cgo_dedup(_ptr(keys), n, ell, word_bits, _ptr(cells), ctypes.byref(nc),
                       _ptr(pc) if pc is not None else None)
    if rc:
        raise RuntimeError(f"cgo_dedup failed: {rc}")
    cells = cells[: nc.value].copy()
    if point_cell:
        return cells, pc[:n].copy()
    return cells


def neighbors(cells, ell: int, word_bits: int = 64, rows=None) -> np.ndarray:
    """Edges (i, j), i < j, of the cell graph over sorted unique ``cells``, as
    uint32[E, 2] in lexicographic order. With ``rows``, only edges whose first
    endpoint is in ``rows`` (in the order of ``rows``)."""
    lib = _load()
    cells = np.ascontiguousarray(cells, dtype=_wtype(word_bits))
    u = cells.shape[0]
    assert cells.shape[1] == words(ell, word_bits)
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n_rows = u if rows_arr is None else rows_arr.shape[0]
    cap = max(1, n_rows * ell // 2 + 1) if ell <= 64 else max(1, n_rows * 4)
    while True:
        edges = np.zeros((cap, 2), dtype=np.uint32)
        ne = ctypes.c_int64(0)
        rc = lib.cgo_neighbors_h1_rows(_ptr(cells), u, ell, word_bits,
                                       _ptr(rows_arr) if rows_arr is not None else None,
                                       n_rows, _ptr(edges), cap, ctypes.byref(ne))
        if rc == -2:
            cap = ne.value
            continue
        if rc:
            raise RuntimeError(f"cgo_neighbors_h1 failed: {rc}")
        return edges[: ne.value].copy()


def heuristic(cells, ell: int, word_bits: int = 64, h: int = 4, w: int = 32,
              as_printed: bool = False):
    """Edges by the heuristic of §3.1 (Algorithms 1-2) with the first h cells
    as pivots and w-segment comparison: (edges uint32[E][2], pairs that passed
    the pivot test). as_printed applies Algorithm 2's test as printed ("> 1"),
    which the oracle reads as inverted."""
    lib = _load()
    cells = np.ascontiguousarray(cells)
    u = cells.shape[0]
    ne, nt = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.cgo_heuristic(_ptr(cells), u, ell, word_bits, h, w, int(as_printed), None, 0,
                           ctypes.byref(ne), ctypes.byref(nt))
    if rc not in (0, -2):
        raise RuntimeError(f"cgo_heuristic failed: {rc}")
    out = np.zeros((ne.value, 2), np.uint32)
    rc = lib.cgo_heuristic(_ptr(cells), u, ell, word_bits, h, w, int(as_printed), _ptr(out),
                           ne.value, ctypes.byref(ne), ctypes.byref(nt))
    if rc != 0:
        raise RuntimeError(f"cgo_heuristic failed: {rc}")
    return out, int(nt.value)


def bfs(edges, n_cells: int, source: int) -> np.ndarray:
    """Shortest-path distances (in edges) from cell `source` over the
    undirected edge list, -1 for unreachable cells (int32[n_cells])."""
    lib = _load()
    edges = np.ascontiguousarray(edges, dtype=np.uint32).reshape(-1, 2)
    dist = np.zeros(n_cells, np.int32)
    rc = lib.cgo_bfs(_ptr(edges), edges.shape[0], n_cells, source, _ptr(dist))
    if rc != 0:
        raise RuntimeError(f"cgo_bfs failed: {rc}")
    return dist


def tree(cells, ell: int, word_bits: int = 64, r: int = 8, order: int = 0, edges: bool = True):
    """The search tree of §3.2 over sorted unique ``cells``: node counts per
    level (index 0 is the root) and, with ``edges``, the edges found by the
    Algorithm 4 walk (uint32[E, 2], same order as ``neighbors``). ``order`` 0
    is the paper's digit recoding (Figure 2), 1 the value-order recoding."""
    lib = _load()
    cells = np.ascontiguousarray(cells, dtype=_wtype(word_bits))
    u = cells.shape[0]
    L = (ell + r - 1) // r
    counts = np.zeros(L + 1, dtype=np.int64)
    if not edges:
        rc = lib.cgo_tree(_ptr(cells), u, ell, word_bits, r, order, _ptr(counts), L + 1, None, 0,
                          ctypes.byref(ctypes.c_int64(0)))
        if rc:
            raise RuntimeError(f"cgo_tree failed: {rc}")
        return counts
    cap = max(1, u * min(ell, 64) // 2 + 1) if ell <= 64 else max(1, u * 4)
    while True:
        out = np.zeros((cap, 2), dtype=np.uint32)
        ne = ctypes.c_int64(0)
        rc = lib.cgo_tree(_ptr(cells), u, ell, word_bits, r, order, _ptr(counts), L + 1, _ptr(out),
                          cap, ctypes.byref(ne))
        if rc == -2:
            cap = ne.value
            continue
        if rc:
            raise RuntimeError(f"cgo_tree failed: {rc}")
        return counts, out[: ne.value].copy()


def tree_digits(cells, ell: int, word_bits: int = 64, r: int = 8, order: int = 0) -> np.ndarray:
    """Digit recoding used by ``tree``: uint32[U, ceil(l / r)]."""
    lib = _load()
    cells = np.ascontiguousarray(cells, dtype=_wtype(word_bits))
    u = cells.shape[0]
    L = (ell + r - 1) // r
    out = np.zeros((max(u, 1), L), dtype=np.uint32)
    rc = lib.cgo_tree_digits(_ptr(cells), u, ell, word_bits, r, order, _ptr(out))
    if rc:
        raise RuntimeError(f"cgo_tree_digits failed: {rc}")
    return out[:u].copy()


def build(pts, a, b, word_bits: int = 64):
    """(cells, edges) of one scene: pack, dedup, neighbours."""
    keys = pack_signs(pts, a, b, word_bits)
    cells = dedup(keys, np.asarray(a).shape[0], word_bits)
    edges = neighbors(cells, np.asarray(a).shape[0], word_bits)
    return cells, edges
