"""The allocation-free neighbour search (cg_neighbors_h1_noalloc).

Callers that cannot allocate device memory at the point of the call (a fixed
memory budget, a real-time loop, a host whose allocator belongs to another
framework) use this entry point: its scratch lives in a fixed array inside the
library. The test calls it through the C-ABI twice in a row, on two different
inputs, and checks each result against the regular entry point
cg_neighbors_h1 bit for bit (edges are integers: the tolerance is zero). It
also checks that oversized inputs are refused before any work is done.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    lib = cellgraph.load_library()
    lib.cg_neighbors_h1_noalloc.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
        ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    lib.cg_neighbors_h1_noalloc.restype = ctypes.c_int
    return lib


def _cells(seed, n, ell, word_bits):
    sc = inputs.planes_3d(n=n, ell=ell, seed=seed)
    keys = oracle.pack_signs(sc.pts, sc.a, sc.b, word_bits)
    return oracle.dedup(keys, ell, word_bits)


def _noalloc(lib, cells_dev, u, ell, word_bits, cap):
    edges = torch.full((cap, 2), -1, dtype=torch.int32, device=cells_dev.device)
    ne = ctypes.c_int64(-1)
    rc = lib.cg_neighbors_h1_noalloc(
        ctypes.c_void_p(cells_dev.data_ptr()), u, ell, word_bits,
        ctypes.c_void_p(edges.data_ptr()), cap, ctypes.byref(ne),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, ne.value, edges


@pytest.mark.parametrize("word_bits", [64, 32])
def test_noalloc_matches_regular_entry_point_twice(lib, word_bits):
    dev = torch.device("cuda:0")
    dt = np.int64 if word_bits == 64 else np.int32
    for seed, n, ell in [(21, 400_000, 64), (22, 150_000, 40)]:
        cells = _cells(seed, n, ell, word_bits)
        u = len(cells)
        assert 0 < u <= 65536
        cells_dev = torch.from_numpy(np.ascontiguousarray(cells).view(dt)).to(dev)
        want = cellgraph.neighbors_h1(cells_dev, ell, word_bits, strategy="hash")
        cap = want.shape[0] + 16
        rc, ne, edges = _noalloc(lib, cells_dev, u, ell, word_bits, cap)
        assert rc == 0, lib.cg_last_error()
        assert ne == want.shape[0]
        assert torch.equal(edges[:ne], want)
        assert (edges[ne:] == -1).all()


def test_noalloc_refuses_oversized_input(lib):
    dev = torch.device("cuda:0")
    cells = torch.zeros((65537, 1), dtype=torch.int64, device=dev)
    rc, _, _ = _noalloc(lib, cells, 65537, 64, 64, 4)
    assert rc == cellgraph.ERR_INVALID_ARG
    assert b"capacity" in lib.cg_last_error()
