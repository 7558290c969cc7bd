"""Bounded device-side waits run out cleanly.

Every wait of the library on another block's progress (the edge kernels'
decoupled look-back, also in the one-pass edge output of PIVOT and HALVES;
the BFS grid barrier; the tensor-core sign kernel's wait for its MMA) gives
up after a fixed number of polls, sets an error bit and returns. These tests lower the limit to 0 polls with cg_set_wait_limit, so
that each wait gives up before it looks (a wait that nothing will end), check
that the public call returns CG_ERR_TIMEOUT and that the GPU context stays
usable, then restore the limit and check the same call against the oracle.
No kernel is made to fault or hang: the waits end by their own bound.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    yield torch.device("cuda:0")


def _timeout(fn):
    with pytest.raises(cellgraph.CellGraphError) as ei:
        fn()
        torch.cuda.synchronize()
    assert ei.value.status == cellgraph.ERR_TIMEOUT, str(ei.value)
    torch.cuda.synchronize()  # the context still answers


def _cells_dev(cells, dev):
    return torch.from_numpy(np.ascontiguousarray(cells).view(np.int64)).to(dev)


@pytest.mark.parametrize("ell,strategy", [(64, "hash"), (64, "sorted"), (64, "pivot"),
                                          (64, "halves")])
def test_lookback_wait_runs_out(dev, ell, strategy):
    sc = inputs.planes_3d(n=300_000, ell=ell, seed=61)
    cells = oracle.dedup(oracle.pack_signs(sc.pts, sc.a, sc.b, 64), ell, 64)
    # more than one chunk (32 cells for HASH and SORTED, 4,096 for the edge
    # pass of PIVOT and HALVES), so later chunks look back
    assert len(cells) > 4096
    cd = _cells_dev(cells, dev)
    cellgraph.set_wait_limit(0)
    try:
        _timeout(lambda: cellgraph.neighbors_h1(cd, ell, 64, strategy=strategy))
    finally:
        cellgraph.set_wait_limit(-1)
    got = cellgraph.neighbors_h1(cd, ell, 64, strategy=strategy)
    want = oracle.neighbors(cells, ell, 64)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("strategy", ["hash", "sorted"])
def test_wide_build_lookback_wait_runs_out(dev, strategy):
    # l = 100 rows of two words: the single-pass build's edge kernel for wide
    # rows (neighbors_emit_wide) finds its output offset by look-back.
    ell = 100
    sc = inputs.planes_3d(n=300_000, ell=ell, seed=64)
    args = tuple(torch.from_numpy(x).to(dev) for x in (sc.pts, sc.a, sc.b))
    ctx = cellgraph.Context(0)
    try:
        bucket = next(i for i, lim in enumerate(cellgraph.TUNE_LIMITS) if ell <= lim)
        ctx.tune_set(bucket, strategy)
        cellgraph.set_wait_limit(0)
        try:
            _timeout(lambda: ctx.build(*args, 64))
        finally:
            cellgraph.set_wait_limit(-1)
        cells, edges = ctx.build(*args, 64)
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
        assert len(want_c) > 64 * 32
        assert np.array_equal(cells.cpu().numpy().view(np.uint64).reshape(want_c.shape), want_c)
        assert np.array_equal(edges.cpu().numpy().view(np.uint32), want_e)
    finally:
        ctx.close()


def test_bfs_grid_barrier_runs_out(dev, monkeypatch):
    monkeypatch.delenv("CG_BFS_LEVELS", raising=False)  # the cooperative form
    ell = 12
    q = np.arange(1 << ell, dtype=np.uint64).reshape(-1, 1)
    edges = oracle.neighbors(q, ell, 64)  # the hypercube Q_12
    ed = torch.from_numpy(edges.view(np.int32)).to(dev)
    n = 1 << ell
    cellgraph.set_wait_limit(0)
    try:
        _timeout(lambda: cellgraph.bfs(ed, n, 0))
    finally:
        cellgraph.set_wait_limit(-1)
    dist, _, reached, depth = cellgraph.bfs(ed, n, 0)
    assert np.array_equal(dist.cpu().numpy(), oracle.bfs(edges, n, 0))
    assert reached == n and depth == ell


def test_tensor_core_mma_wait_runs_out(dev, monkeypatch):
    monkeypatch.setenv("CG_SIGN_KERNEL", "tc")
    # Four real planes and 60 constraints 0 . p >= 0 (always 1): at most 15
    # cells, one chunk of the edge kernel, so no look-back wait is needed and
    # the timeout can only come from the sign kernel's wait for its MMA.
    sc = inputs.planes_3d(n=250_001, ell=64, seed=62)
    sc.a[4:] = 0
    sc.b[4:] = 0
    args = tuple(torch.from_numpy(x).to(dev) for x in (sc.pts, sc.a, sc.b))
    ctx = cellgraph.Context(0)
    try:
        cellgraph.set_wait_limit(0)
        try:
            _timeout(lambda: ctx.build(*args, 64))
        finally:
            cellgraph.set_wait_limit(-1)
        cells, edges = ctx.build(*args, 64)
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
        assert 2 <= len(want_c) <= 15
        assert np.array_equal(cells.cpu().numpy().view(np.uint64), want_c)
        assert np.array_equal(edges.cpu().numpy().view(np.uint32), want_e)
    finally:
        ctx.close()


def test_wait_limit_restored_after_each_test(dev):
    # Whatever ran before, the default limits apply: an ordinary call works.
    sc = inputs.planes_3d(n=50_000, ell=40, seed=63)
    cells = oracle.dedup(oracle.pack_signs(sc.pts, sc.a, sc.b, 64), 40, 64)
    got = cellgraph.neighbors_h1(_cells_dev(cells, dev), 40, 64)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), oracle.neighbors(cells, 40, 64))
