"""The allocation-free neighbour search (cg_neighbors_h1_noalloc).

Callers that cannot allocate device memory at the point of the call (a fixed
memory budget, a real-time loop, a host whose allocator belongs to another
framework) use this entry point: its scratch lives in a fixed array inside the
library. The tests call it through the C-ABI twice in a row, on two different
inputs, and check each result bit for bit (edges are integers: the tolerance
is zero) against the regular entry point cg_neighbors_h1 and against the CPU
oracle. A near-capacity input runs right before a small one, so contents a
large call leaves in the shared array must not leak into the next call. Bad
input (unsorted rows, repeated rows, bits at or above l) must give the same
status from both entry points, and oversized inputs are refused before any
work is done.

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


def _chain_cells(n_seeds, ell, seed):
    """Sorted distinct l <= 64 vectors with many Hamming-1 pairs (planted chains)."""
    ch = inputs.chains(n_seeds=n_seeds, chain_len=15, ell=ell, seed=seed)
    return oracle.dedup(ch.keys, ell, 64)


def _dev_words(cells, word_bits):
    dt = np.int64 if word_bits == 64 else np.int32
    return torch.from_numpy(np.ascontiguousarray(cells).view(dt)).to("cuda:0")


def _noalloc(lib, cells_dev, u, ell, word_bits, cap):
    edges = torch.full((max(cap, 1), 2), -1, dtype=torch.int32, device="cuda:0")
    ne = ctypes.c_int64(-1)
    ptr = cells_dev.data_ptr() if cells_dev is not None else None
    rc = lib.cg_neighbors_h1_noalloc(
        ctypes.c_void_p(ptr), u, ell, word_bits,
        ctypes.c_void_p(edges.data_ptr()), cap, ctypes.byref(ne),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, ne.value, edges


def _regular_status(cells_dev, ell, word_bits):
    try:
        cellgraph.neighbors_h1(cells_dev, ell, word_bits, strategy="hash")
    except cellgraph.CellGraphError as e:
        return e.status
    return cellgraph.OK


def _check_against_both(lib, cells, ell, word_bits):
    cells_dev = _dev_words(cells, word_bits)
    u = len(cells)
    want = cellgraph.neighbors_h1(cells_dev, ell, word_bits, strategy="hash")
    ref = oracle.neighbors(cells, ell, word_bits)
    cap = want.shape[0] + 16
    rc, ne, edges = _noalloc(lib, cells_dev, u, ell, word_bits, cap)
    assert rc == 0, lib.cg_last_error()
    assert ne == want.shape[0] == ref.shape[0]
    assert torch.equal(edges[:ne], want)
    assert np.array_equal(edges[:ne].cpu().numpy().view(np.uint32), ref)
    assert (edges[ne:] == -1).all()
    return ne


@pytest.mark.parametrize("word_bits", [64, 32])
def test_noalloc_matches_regular_entry_point_twice(lib, word_bits):
    for seed, n, ell in [(21, 400_000, 64), (22, 150_000, 40)]:
        cells = _cells(seed, n, ell, word_bits)
        assert 0 < len(cells) <= 65536
        _check_against_both(lib, cells, ell, word_bits)


def test_noalloc_near_capacity_then_small(lib):
    big = _chain_cells(4096, 64, seed=31)
    assert 60_000 < len(big) <= 65536
    e_big = _check_against_both(lib, big, 64, 64)
    assert e_big > 50_000
    small = _cells(23, 50_000, 48, 64)
    assert len(small) < len(big) // 4
    _check_against_both(lib, small, 48, 64)
    _check_against_both(lib, big, 64, 64)


def test_noalloc_all_ones_cell(lib):
    # l = 64: the all-ones vector is a legal cell (the table keeps it apart).
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)
    base = np.array([ones ^ (np.uint64(1) << np.uint64(k)) for k in range(0, 64, 3)] + [ones],
                    dtype=np.uint64)
    cells = np.unique(base).reshape(-1, 1)
    assert _check_against_both(lib, cells, 64, 64) == len(cells) - 1
    # Repeating it is refused, as by the regular entry point.
    rep = np.concatenate([cells, cells[-1:]], axis=0)
    rc, _, _ = _noalloc(lib, _dev_words(rep, 64), len(rep), 64, 64, 64)
    assert rc == cellgraph.ERR_INVALID_ARG, lib.cg_last_error()
    assert _regular_status(_dev_words(rep, 64), 64, 64) == cellgraph.ERR_INVALID_ARG


def test_noalloc_empty_input(lib):
    rc, ne, _ = _noalloc(lib, None, 0, 64, 64, 0)
    assert rc == 0, lib.cg_last_error()
    assert ne == 0


@pytest.mark.parametrize("word_bits", [64, 32])
def test_noalloc_rejects_what_the_regular_entry_point_rejects(lib, word_bits):
    cells = _cells(24, 100_000, 40, word_bits)
    u = len(cells)
    assert u > 8
    swapped = cells.copy()
    swapped[[3, 4]] = swapped[[4, 3]]
    repeated = cells.copy()
    repeated[5] = repeated[4]
    high = cells.copy()
    # Bit 45 is above l = 40: in the second 32-bit word, or in the only 64-bit word.
    if word_bits == 64:
        high[7, 0] |= np.uint64(1 << 45)
    else:
        high[7, 1] |= np.uint32(1 << (45 - 32))
    for bad in (swapped, repeated, high):
        d = _dev_words(bad, word_bits)
        rc, _, _ = _noalloc(lib, d, u, 40, word_bits, u * 20)
        assert rc == cellgraph.ERR_INVALID_ARG, lib.cg_last_error()
        assert _regular_status(d, 40, word_bits) == cellgraph.ERR_INVALID_ARG
    # A good call right after the refused ones is unaffected by them.
    _check_against_both(lib, cells, 40, word_bits)


def test_noalloc_refuses_oversized_input(lib):
    cells = torch.zeros((65537, 1), dtype=torch.int64, device="cuda:0")
    rc, _, _ = _noalloc(lib, cells, 65537, 64, 64, 4)
    assert rc == cellgraph.ERR_INVALID_ARG
    assert b"capacity" in lib.cg_last_error()
