"""ctypes binding of libcellgraph.so (C-ABI in include/cellgraph.h).

Argument marshalling only: every step runs in the CUDA library. Tensors are
torch CUDA tensors (device memory and the current stream come from torch);
vectors use int64 tensors for 64-bit words and int32 tensors for 32-bit words
(the bits are the unsigned words of the C-ABI), edges are int32 [E, 2] holding
the uint32 cell numbers.

There is no CPU fallback: if the library is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcellgraph.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_CAPACITY = 3
ERR_OOM = 4
ERR_CUDA = 5
ERR_TIMEOUT = 6
ERR_INTERNAL = 7

STRATEGY = {"auto": 0, "hash": 1, "sorted": 2, "pivot": 3, "tree": 4, "halves": 5,
            "allpairs": 6}
STRATEGY_NAME = {v: k for k, v in STRATEGY.items()}
TUNE_BUCKETS = 7
TUNE_LIMITS = (16, 32, 64, 128, 256, 1024, 4096)

EXPORTS = [
    "cg_last_error", "cg_version", "cg_launch_count", "cg_pack_signs", "cg_dedup_cells",
    "cg_neighbors_h1", "cg_ctx_create", "cg_ctx_destroy", "cg_ctx_pool_bytes", "cg_build",
    "cg_build_host", "cg_ctx_set_timing", "cg_ctx_stage_times", "cg_build_batch",
    "cg_server_create", "cg_server_submit", "cg_server_poll", "cg_server_wait",
    "cg_server_result_get", "cg_server_copy", "cg_server_release", "cg_server_get_stats",
    "cg_server_inject_alloc_failures", "cg_server_destroy", "cg_tune_bucket", "cg_ctx_tune_get",
    "cg_ctx_tune_set", "cg_ctx_autotune", "cg_server_use_tuning", "cg_build_dev", "cg_bfs",
    "cg_set_wait_limit", "cg_pack_signs_quadric",
]

REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class CgScene(ctypes.Structure):
    """struct cg_scene (include/cellgraph.h)."""
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("ell", ctypes.c_int)]


class CgBatchOut(ctypes.Structure):
    """struct cg_batch_out (include/cellgraph.h)."""
    _fields_ = [("cells", ctypes.c_void_p), ("cells_cap", ctypes.c_int64),
                ("edges", ctypes.c_void_p), ("edges_cap", ctypes.c_int64),
                ("n_cells", ctypes.c_void_p), ("n_edges", ctypes.c_void_p),
                ("cells_offset", ctypes.c_void_p), ("edges_offset", ctypes.c_void_p)]


class CgTuneParams(ctypes.Structure):
    """struct cg_tune_params (include/cellgraph.h)."""
    _fields_ = [("strategy", ctypes.c_int), ("pivots", ctypes.c_int),
                ("sign_kernel", ctypes.c_int)]


class CgServerResult(ctypes.Structure):
    """struct cg_server_result (include/cellgraph.h)."""
    _fields_ = [("status", ctypes.c_int), ("n_cells", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("words", ctypes.c_int),
                ("cells", ctypes.c_void_p), ("edges", ctypes.c_void_p),
                ("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("retries", ctypes.c_int)]


class CgServerStats(ctypes.Structure):
    """struct cg_server_stats (include/cellgraph.h)."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("retried", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("max_running", ctypes.c_int), ("groups", ctypes.c_int64),
                ("grouped", ctypes.c_int64)]


class CellGraphError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libcellgraph.so (raises if it is missing) and declares signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise CellGraphError(-1, f"{path} is not built (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I64, I, S = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        PI64 = ctypes.POINTER(ctypes.c_int64)
        PS = ctypes.POINTER(ctypes.c_size_t)
        lib.cg_last_error.restype = ctypes.c_char_p
        lib.cg_version.restype = ctypes.c_char_p
        lib.cg_launch_count.restype = ctypes.c_uint64
        lib.cg_pack_signs.argtypes = [P, I64, I, P, P, I, I, P, P]
        lib.cg_dedup_cells.argtypes = [P, I64, I, I, P, I64, PI64, P, P, PS, P]
        lib.cg_neighbors_h1.argtypes = [P, I64, I, I, P, I64, PI64, I, P, PS, P]
        lib.cg_ctx_create.argtypes = [ctypes.POINTER(P), I]
        lib.cg_ctx_destroy.argtypes = [P]
        lib.cg_ctx_pool_bytes.argtypes = [P, PS]
        build_args = [P, P, I64, I, P, P, I, I, P, I64, PI64, P, I64, PI64, P]
        lib.cg_build.argtypes = build_args
        lib.cg_build_host.argtypes = build_args
        lib.cg_build_batch.argtypes = [P, P, I, P, P]
        lib.cg_build_dev.argtypes = [P, P, I64, I, P, P, I, I, P, I64, P, I64, P, P]
        lib.cg_ctx_set_timing.argtypes = [P, I]
        lib.cg_ctx_stage_times.argtypes = [P, P, P, I, ctypes.POINTER(ctypes.c_int), PI64]
        lib.cg_server_create.argtypes = [I, S, I, ctypes.POINTER(P)]
        lib.cg_server_submit.argtypes = [P, P, I, PI64]
        lib.cg_server_poll.argtypes = [P, I64, ctypes.POINTER(ctypes.c_int)]
        lib.cg_server_wait.argtypes = [P, I64, ctypes.c_double]
        lib.cg_server_result_get.argtypes = [P, I64, P]
        lib.cg_server_copy.argtypes = [P, I64, P, I64, P, I64]
        lib.cg_server_release.argtypes = [P, I64]
        lib.cg_server_get_stats.argtypes = [P, P]
        lib.cg_server_inject_alloc_failures.argtypes = [P, I]
        lib.cg_server_destroy.argtypes = [P]
        lib.cg_tune_bucket.argtypes = [I]
        lib.cg_ctx_tune_get.argtypes = [P, I, P]
        lib.cg_ctx_tune_set.argtypes = [P, I, P]
        lib.cg_ctx_autotune.argtypes = [P, P, I, I, P]
        lib.cg_server_use_tuning.argtypes = [P, P]
        lib.cg_bfs.argtypes = [P, I64, I64, I64, P, P, PI64, PI64, P, PS, P]
        lib.cg_set_wait_limit.argtypes = [I64]
        lib.cg_pack_signs_quadric.argtypes = [P, I64, I, P, P, P, I, I, P, P]
        for name in EXPORTS[3:]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != OK:
        raise CellGraphError(st, load_library().cg_last_error().decode())


def version() -> str:
    return load_library().cg_version().decode()


def launch_count() -> int:
    return int(load_library().cg_launch_count())


def set_wait_limit(polls: int) -> None:
    """Test control: bounded device-side waits of kernels launched afterwards
    give up after ``polls`` polls (0: before the first one); a negative value
    restores the built-in limits."""
    _check(load_library().cg_set_wait_limit(int(polls)))


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)


def words(ell: int, word_bits: int) -> int:
    return (ell + word_bits - 1) // word_bits


def word_dtype(word_bits: int):
    torch = _torch()
    if word_bits == 64:
        return torch.int64
    if word_bits == 32:
        return torch.int32
    raise ValueError("word_bits must be 32 or 64")


def pack_signs(pts, a, b, word_bits: int = 64, out=None, stream=None):
    """Sign vectors of the points (§2.1): returns [N, W] words on the device."""
    torch = _torch()
    lib = load_library()
    n, d = pts.shape
    ell = a.shape[0]
    if out is None:
        out = torch.empty((n, words(ell, word_bits)), dtype=word_dtype(word_bits),
                          device=pts.device)
    _check(lib.cg_pack_signs(_dev(pts, torch.int32, "pts"), n, d, _dev(a, torch.int32, "a"),
                             _dev(b, torch.int64, "b"), ell, word_bits,
                             _dev(out, word_dtype(word_bits), "keys"), _stream_ptr(stream)))
    return out


def pack_signs_quadric(pts, q, a, b, word_bits: int = 64, out=None, stream=None):
    """Sign vectors of quadric constraints (§2.1 with curved boundaries):
    bit i = [sum_{j<=k} q[i, jk] p_j p_k + a[i] . p >= b[i]], exact. ``q`` is
    int32 [l, d(d+1)/2] (monomial coefficients, (j, k) with j <= k in
    row-major order). Returns [N, W] words on the device."""
    torch = _torch()
    lib = load_library()
    n, d = pts.shape
    ell = a.shape[0]
    if out is None:
        out = torch.empty((n, words(ell, word_bits)), dtype=word_dtype(word_bits),
                          device=pts.device)
    _check(lib.cg_pack_signs_quadric(
        _dev(pts, torch.int32, "pts"), n, d, _dev(q, torch.int32, "q"),
        _dev(a, torch.int32, "a"), _dev(b, torch.int64, "b"), ell, word_bits,
        _dev(out, word_dtype(word_bits), "keys"), _stream_ptr(stream)))
    return out


def build_quadric(pts, q, a, b, word_bits: int = 64, strategy: str = "auto", stream=None):
    """Cells and edges of a scene of quadric constraints: cg_pack_signs_quadric,
    cg_dedup_cells and cg_neighbors_h1 in turn (device tensors in and out)."""
    ell = a.shape[0]
    keys = pack_signs_quadric(pts, q, a, b, word_bits, stream=stream)
    cells = dedup_cells(keys, ell, word_bits, stream=stream)
    return cells, neighbors_h1(cells, ell, word_bits, strategy=strategy, stream=stream)


def dedup_cells(keys, ell: int, word_bits: int = 64, point_cell: bool = False, stream=None):
    """Sorted distinct vectors (§3.2); optionally the cell number of every row."""
    torch = _torch()
    lib = load_library()
    n = keys.shape[0]
    kp = _dev(keys, word_dtype(word_bits), "keys")
    need = ctypes.c_size_t(0)
    st = ctypes.c_void_p(None)
    _check(lib.cg_dedup_cells(kp, n, ell, word_bits, None, 0, None, None, None,
                              ctypes.byref(need), st))
    ws = torch.empty(need.value, dtype=torch.uint8, device=keys.device)
    cells = torch.empty((max(n, 1), words(ell, word_bits)), dtype=word_dtype(word_bits),
                        device=keys.device)
    pc = torch.empty(max(n, 1), dtype=torch.int32, device=keys.device) if point_cell else None
    nc = ctypes.c_int64(0)
    _check(lib.cg_dedup_cells(kp, n, ell, word_bits, _dev(cells, word_dtype(word_bits), "cells"),
                              cells.shape[0], ctypes.byref(nc),
                              _dev(pc, torch.int32, "point_cell") if pc is not None else None,
                              ctypes.c_void_p(ws.data_ptr()), ctypes.byref(need),
                              _stream_ptr(stream)))
    cells = cells[: nc.value]
    if point_cell:
        return cells, pc[:n]
    return cells


def neighbors_h1(cells, ell: int, word_bits: int = 64, strategy: str = "auto", edges_cap=None,
                 stream=None):
    """Edges (i, j), i < j, of the cell graph over sorted distinct ``cells``
    (§2.2, Algorithm 4), as an int32 [E, 2] device tensor."""
    torch = _torch()
    lib = load_library()
    u = cells.shape[0]
    cp = _dev(cells, word_dtype(word_bits), "cells")
    need = ctypes.c_size_t(0)
    _check(lib.cg_neighbors_h1(cp, u, ell, word_bits, None, 0, None, STRATEGY[strategy], None,
                               ctypes.byref(need), ctypes.c_void_p(None)))
    ws = torch.empty(need.value, dtype=torch.uint8, device=cells.device)
    cap = edges_cap if edges_cap is not None else max(1, u * min(ell, 64) // 2 + 1)
    while True:
        edges = torch.empty((cap, 2), dtype=torch.int32, device=cells.device)
        ne = ctypes.c_int64(0)
        rc = lib.cg_neighbors_h1(cp, u, ell, word_bits, _dev(edges, torch.int32, "edges"), cap,
                                 ctypes.byref(ne), STRATEGY[strategy],
                                 ctypes.c_void_p(ws.data_ptr()), ctypes.byref(need),
                                 _stream_ptr(stream))
        if rc == ERR_CAPACITY:
            cap = ne.value
            continue
        _check(rc)
        return edges[: ne.value]


def bfs(edges, n_cells: int, source: int, parent: bool = True, stream=None):
    """Breadth-first search on the cell graph from cell ``source`` (a path in
    G_X is an approximate motion plan, §6). ``edges``: the int32 [E, 2] device
    tensor of ``neighbors_h1`` / ``Context.build``. Returns (dist, parent,
    n_reached, depth): int32 [n_cells] device tensors (dist -1 when
    unreachable; parent None unless asked for, -1 for the source)."""
    torch = _torch()
    lib = load_library()
    e = edges.reshape(-1, 2)
    ep = _dev(e, torch.int32, "edges") if e.shape[0] > 0 else ctypes.c_void_p(None)
    need = ctypes.c_size_t(0)
    _check(lib.cg_bfs(ep, e.shape[0], n_cells, source, None, None, None, None, None,
                      ctypes.byref(need), ctypes.c_void_p(None)))
    dev = edges.device
    ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
    dist = torch.empty(n_cells, dtype=torch.int32, device=dev)
    par = torch.empty(n_cells, dtype=torch.int32, device=dev) if parent else None
    reached, depth = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.cg_bfs(ep, e.shape[0], n_cells, source, ctypes.c_void_p(dist.data_ptr()),
                      ctypes.c_void_p(par.data_ptr()) if parent else None,
                      ctypes.byref(reached), ctypes.byref(depth),
                      ctypes.c_void_p(ws.data_ptr()), ctypes.byref(need), _stream_ptr(stream)))
    return dist, par, int(reached.value), int(depth.value)


def path_to(parent, source: int, target: int):
    """Cells on the BFS tree's path from ``source`` to ``target`` (host list),
    following a ``bfs`` parent array; empty when target was not reached."""
    par = parent.cpu().numpy() if hasattr(parent, "cpu") else parent
    out = [int(target)]
    for _ in range(len(par)):
        p = int(par[out[-1]])
        if p < 0:
            break
        out.append(p)
    return out[::-1] if out[-1] == int(source) else []


def arrangement_cells_bound(n: int, d: int, ell: int) -> int:
    """min(n, sum_{k<=d} C(l, k)): the number of cells of l hyperplanes in
    R^d, used only as a first guess for output sizes."""
    return max(1, min(n, sum(math.comb(ell, k) for k in range(d + 1))))


class Context:
    """A library context (device pool, pinned count words, learned sizes) plus
    output-capacity bookkeeping for ``build``."""

    def __init__(self, device: int = 0):
        self._lib = load_library()
        self._h = ctypes.c_void_p(None)
        _check(self._lib.cg_ctx_create(ctypes.byref(self._h), device))
        self.device = device
        self._caps = {}
        self._bufs = {}

    def close(self):
        if self._h:
            self._lib.cg_ctx_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pool_bytes(self) -> int:
        v = ctypes.c_size_t(0)
        _check(self._lib.cg_ctx_pool_bytes(self._h, ctypes.byref(v)))
        return v.value

    def set_timing(self, enable: bool):
        _check(self._lib.cg_ctx_set_timing(self._h, int(enable)))

    def stage_times(self):
        """({stage name: total ms}, number of builds) since timing was enabled."""
        cap = 16
        ms = (ctypes.c_double * cap)()
        names = (ctypes.c_char_p * cap)()
        n = ctypes.c_int(0)
        builds = ctypes.c_int64(0)
        _check(self._lib.cg_ctx_stage_times(self._h, ctypes.cast(ms, ctypes.c_void_p),
                                            ctypes.cast(names, ctypes.c_void_p), cap,
                                            ctypes.byref(n), ctypes.byref(builds)))
        return {names[k].decode(): float(ms[k]) for k in range(min(n.value, cap))}, builds.value

    def _initial_caps(self, n, d, ell):
        u = arrangement_cells_bound(n, d, ell)
        return max(1, u), max(1, u * min(ell, 64) // 2)

    def build(self, pts, a, b, word_bits: int = 64, stream=None, outputs=None):
        """Cells and edges of one scene (device tensors in, device tensors out).
        ``outputs`` may pass preallocated (cells, edges) buffers."""
        torch = _torch()
        n, d = pts.shape
        ell = a.shape[0]
        key = (n, d, ell, word_bits)
        ccap, ecap = self._caps.get(key) or self._initial_caps(n, d, ell)
        args = (_dev(pts, torch.int32, "pts"), n, d, _dev(a, torch.int32, "a"),
                _dev(b, torch.int64, "b"), ell, word_bits)
        while True:
            if outputs is not None and outputs[0].shape[0] >= ccap and outputs[1].shape[0] >= ecap:
                cells, edges = outputs
                ccap, ecap = cells.shape[0], edges.shape[0]
            else:
                cells = torch.empty((ccap, words(ell, word_bits)), dtype=word_dtype(word_bits),
                                    device=pts.device)
                edges = torch.empty((ecap, 2), dtype=torch.int32, device=pts.device)
            nc = ctypes.c_int64(0)
            ne = ctypes.c_int64(0)
            rc = self._lib.cg_build(self._h, *args, _dev(cells, word_dtype(word_bits), "cells"),
                                    ccap, ctypes.byref(nc), _dev(edges, torch.int32, "edges"),
                                    ecap, ctypes.byref(ne), _stream_ptr(stream))
            if rc == ERR_CAPACITY:
                ccap, ecap = max(ccap, nc.value), max(ecap, ne.value)
                self._caps[key] = (ccap, ecap)
                outputs = None
                continue
            _check(rc)
            self._caps[key] = (max(ccap, nc.value), max(ecap, ne.value))
            return cells[: nc.value], edges[: ne.value]

    def build_dev(self, pts, a, b, cells, edges, counts, word_bits: int = 64, stream=None):
        """Enqueues one build without waiting (cg_build_dev): results go to the
        given device buffers, and counts (int64 [3] device tensor) receives U,
        E and a status once the stream reaches it. Capturable in a CUDA graph
        after a first call of the same size."""
        torch = _torch()
        n, d = pts.shape
        ell = a.shape[0]
        _check(self._lib.cg_build_dev(
            self._h, _dev(pts, torch.int32, "pts"), n, d, _dev(a, torch.int32, "a"),
            _dev(b, torch.int64, "b"), ell, word_bits, _dev(cells, word_dtype(word_bits), "cells"),
            cells.shape[0], _dev(edges, torch.int32, "edges"), edges.shape[0],
            _dev(counts, torch.int64, "counts"), _stream_ptr(stream)))

    def build_batch(self, scenes, stream=None, as_views: bool = True):
        """Cells and edges of many independent scenes in one batched call.
        ``scenes``: sequence of (pts, a, b) CUDA tensors. Returns a list of
        (cells int64 [U, W], edges int32 [E, 2]) views, W = ceil(l/64), cell
        numbers scene-local. The views share output buffers that the context
        reuses for the next batch of the same scenes (which then replays a
        captured CUDA graph): copy results that must outlive that call.
        With ``as_views=False`` returns (cells, edges, cells_offset,
        edges_offset) instead: the whole output buffers and the per-scene
        offsets (words / edges), without building per-scene views."""
        torch = _torch()
        S = len(scenes)
        if S == 0:
            return []
        # The scene descriptors of the last batch are reused when the same
        # tensors come again (the cache holds them, so they stay alive).
        ids = tuple(id(t) for sc in scenes for t in sc)
        cached = getattr(self, "_batch_desc", None)
        if cached is not None and cached[0] == ids:
            _, arr, dev, words_total, edges_total, ws, key, _keep = cached
        else:
            arr = (CgScene * S)()
            dev = None
            words_total = edges_total = 0
            ws = []
            for i, (pts, a, b) in enumerate(scenes):
                n, d = pts.shape
                ell = a.shape[0]
                arr[i] = CgScene(_dev(pts, torch.int32, "pts").value, n, d,
                                 _dev(a, torch.int32, "a").value, _dev(b, torch.int64, "b").value,
                                 ell)
                dev = pts.device
                u = arrangement_cells_bound(n, d, ell)
                ws.append(words(ell, 64))
                words_total += u * ws[-1]
                edges_total += 4 * u
            key = ("batch", tuple((int(x.n), int(x.d), int(x.ell)) for x in arr))
            self._batch_desc = (ids, arr, dev, words_total, edges_total, ws, key,
                                [t for sc in scenes for t in sc])
        ccap, ecap = self._caps.get(key, (max(1, words_total), max(1, edges_total)))
        n_cells = np.zeros(S, dtype=np.int64)
        n_edges = np.zeros(S, dtype=np.int64)
        coff = np.zeros(S + 1, dtype=np.int64)
        eoff = np.zeros(S + 1, dtype=np.int64)
        while True:
            bufs = self._bufs.get(key)
            if bufs is None or bufs[0].shape[0] < ccap or bufs[1].shape[0] < ecap:
                bufs = (torch.empty(ccap, dtype=torch.int64, device=dev),
                        torch.empty((ecap, 2), dtype=torch.int32, device=dev))
                self._bufs[key] = bufs
            cells, edges = bufs
            ccap, ecap = cells.shape[0], edges.shape[0]
            out = CgBatchOut(cells.data_ptr(), ccap, edges.data_ptr(), ecap,
                             n_cells.ctypes.data, n_edges.ctypes.data, coff.ctypes.data,
                             eoff.ctypes.data)
            rc = self._lib.cg_build_batch(self._h, ctypes.cast(arr, ctypes.c_void_p), S,
                                          ctypes.byref(out), _stream_ptr(stream))
            if rc == ERR_CAPACITY:
                ccap, ecap = max(ccap, int(coff[S])), max(ecap, int(eoff[S]))
                self._caps[key] = (ccap, ecap)
                continue
            _check(rc)
            self._caps[key] = (max(ccap, int(coff[S])), max(ecap, int(eoff[S])))
            if not as_views:
                return cells, edges, coff.copy(), eoff.copy()
            res = []
            for i in range(S):
                c = cells[coff[i]: coff[i + 1]].view(-1, ws[i])
                res.append((c, edges[eoff[i]: eoff[i + 1]]))
            return res

    # ---- tuning (cg_ctx_tune_* / cg_ctx_autotune) ----
    def tune_get(self, bucket: int) -> dict:
        p = CgTuneParams()
        _check(self._lib.cg_ctx_tune_get(self._h, bucket, ctypes.byref(p)))
        return {"strategy": STRATEGY_NAME[p.strategy], "pivots": p.pivots,
                "sign_kernel": p.sign_kernel}

    def tune_set(self, bucket: int, strategy: str = "hash", pivots: int = 4,
                 sign_kernel: int = 0):
        """Setting of one bucket of l (cg_ctx_tune_set). sign_kernel: 0 the
        library's choice, 1 tensor cores, 2 fp32 filter behind the box grid,
        3 fp32 filter on every constraint (see cg_tune_params)."""
        p = CgTuneParams(STRATEGY[strategy], pivots, sign_kernel)
        _check(self._lib.cg_ctx_tune_set(self._h, bucket, ctypes.byref(p)))

    def tuning(self) -> list:
        return [self.tune_get(b) for b in range(TUNE_BUCKETS)]

    def autotune(self, scenes, reps: int = 2) -> dict:
        """Times the candidate settings on the given (pts, a, b) CUDA-tensor
        scenes, per bucket of l, and keeps the fastest in the context. Returns
        {bucket: {"setting": ..., "ms": best ms per pass}} for the buckets
        that had scenes."""
        torch = _torch()
        S = len(scenes)
        arr = (CgScene * max(1, S))()
        for i, (pts, a, b) in enumerate(scenes):
            n, d = pts.shape
            arr[i] = CgScene(_dev(pts, torch.int32, "pts").value, n, d,
                             _dev(a, torch.int32, "a").value, _dev(b, torch.int64, "b").value,
                             a.shape[0])
        ms = (ctypes.c_double * TUNE_BUCKETS)()
        _check(self._lib.cg_ctx_autotune(self._h, ctypes.cast(arr, ctypes.c_void_p), S, reps, ms))
        return {b: {"setting": self.tune_get(b), "ms": ms[b]} for b in range(TUNE_BUCKETS)
                if ms[b] > 0}

    def save_tuning(self, path: str, gpu_name: str):
        """Writes the context's tuning to a JSON cache keyed by GPU name."""
        import json

        data = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
        data[gpu_name] = {str(b): t for b, t in enumerate(self.tuning())}
        with open(path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)

    def load_tuning(self, path: str, gpu_name: str) -> bool:
        """Applies the tuning cached for gpu_name; False when there is none."""
        import json

        if not os.path.exists(path):
            return False
        with open(path) as f:
            entry = json.load(f).get(gpu_name)
        if not entry:
            return False
        for b, t in entry.items():
            self.tune_set(int(b), t["strategy"], int(t["pivots"]), int(t["sign_kernel"]))
        return True

    def build_host(self, pts: np.ndarray, a: np.ndarray, b: np.ndarray, word_bits: int = 64,
                   stream=None, outputs=None):
        """Same as ``build`` with numpy arrays in and out (the C-ABI copies)."""
        pts = np.ascontiguousarray(pts, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.int32)
        b = np.ascontiguousarray(b, dtype=np.int64)
        n, d = pts.shape
        ell = a.shape[0]
        key = ("host", n, d, ell, word_bits)
        ccap, ecap = self._caps.get(key) or self._initial_caps(n, d, ell)
        wdt = np.uint64 if word_bits == 64 else np.uint32
        while True:
            if outputs is not None and outputs[0].shape[0] >= ccap and outputs[1].shape[0] >= ecap:
                cells, edges = outputs
                ccap, ecap = cells.shape[0], edges.shape[0]
            else:
                cells = np.empty((ccap, words(ell, word_bits)), dtype=wdt)
                edges = np.empty((ecap, 2), dtype=np.uint32)
            nc = ctypes.c_int64(0)
            ne = ctypes.c_int64(0)
            s = _stream_ptr(stream) if stream is not None or _torch().cuda.is_available() else None
            rc = self._lib.cg_build_host(
                self._h, ctypes.c_void_p(pts.ctypes.data), n, d, ctypes.c_void_p(a.ctypes.data),
                ctypes.c_void_p(b.ctypes.data), ell, word_bits, ctypes.c_void_p(cells.ctypes.data),
                ccap, ctypes.byref(nc), ctypes.c_void_p(edges.ctypes.data), ecap,
                ctypes.byref(ne), s)
            if rc == ERR_CAPACITY:
                ccap, ecap = max(ccap, nc.value), max(ecap, ne.value)
                self._caps[key] = (ccap, ecap)
                outputs = None
                continue
            _check(rc)
            self._caps[key] = (max(ccap, nc.value), max(ecap, ne.value))
            return cells[: nc.value], edges[: ne.value]


class Server:
    """Request server (cg_server_* in include/cellgraph.h): scenes are queued,
    admitted under an HBM budget as slots free up, and built concurrently on
    the device; results stay device-resident until released.

    ``submit`` takes numpy arrays (host inputs, copied by the server after
    admission; pinned memory makes the copies asynchronous) or CUDA tensors
    (used in place). The arrays are kept referenced until the request is
    released."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 8 << 30, max_inflight: int = 16):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.cg_server_create(device, hbm_budget_bytes, max_inflight, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.cg_server_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, pts, a, b) -> int:
        torch = _torch()
        if isinstance(pts, torch.Tensor):
            n, d = pts.shape
            sc = CgScene(_dev(pts, torch.int32, "pts").value, n, d,
                         _dev(a, torch.int32, "a").value, _dev(b, torch.int64, "b").value,
                         a.shape[0])
            on_host = 0
            keep = (pts, a, b)
        else:
            keep = tuple(np.ascontiguousarray(x, dtype=t) for x, t in
                         ((pts, np.int32), (a, np.int32), (b, np.int64)))
            p_, a_, b_ = keep
            n, d = p_.shape
            sc = CgScene(p_.ctypes.data if n else 0, n, d, a_.ctypes.data, b_.ctypes.data,
                         a_.shape[0])
            on_host = 1
        t = ctypes.c_int64(0)
        _check(self._lib.cg_server_submit(self._h, ctypes.byref(sc), on_host, ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int(0)
        _check(self._lib.cg_server_poll(self._h, ticket, ctypes.byref(st)))
        return st.value

    def wait(self, ticket: int, timeout_s: float = -1.0) -> bool:
        """True when the request finished, False when the timeout ran out."""
        rc = self._lib.cg_server_wait(self._h, ticket, float(timeout_s))
        if rc == ERR_TIMEOUT:
            return False
        _check(rc)
        return True

    def result(self, ticket: int) -> dict:
        r = CgServerResult()
        _check(self._lib.cg_server_result_get(self._h, ticket, ctypes.byref(r)))
        msg = self._lib.cg_last_error().decode() if r.status else ""
        return {"status": r.status, "error": msg, "n_cells": r.n_cells, "n_edges": r.n_edges,
                "words": r.words, "submit_us": r.submit_us, "admit_us": r.admit_us,
                "done_us": r.done_us, "retries": r.retries}

    def fetch(self, ticket: int):
        """(cells uint64 [U, W], edges uint32 [E, 2]) of a finished request, as
        numpy arrays on the host."""
        r = self.result(ticket)
        if r["status"]:
            raise CellGraphError(r["status"], r["error"])
        cells = np.empty((r["n_cells"], r["words"]), dtype=np.uint64)
        edges = np.empty((r["n_edges"], 2), dtype=np.uint32)
        _check(self._lib.cg_server_copy(self._h, ticket, cells.ctypes.data, cells.size,
                                        edges.ctypes.data, edges.shape[0]))
        return cells, edges

    def release(self, ticket: int):
        _check(self._lib.cg_server_release(self._h, ticket))
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        st = CgServerStats()
        _check(self._lib.cg_server_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in CgServerStats._fields_}

    def use_tuning(self, ctx: "Context"):
        _check(self._lib.cg_server_use_tuning(self._h, ctx._h))

    def inject_alloc_failures(self, count: int):
        _check(self._lib.cg_server_inject_alloc_failures(self._h, count))
