"""Breadth-first search on the cell graph (cg_bfs) against the oracle.

Distances are unique and compared element by element with the oracle's queue
BFS; parents are one valid BFS tree among several, so they are checked for
validity instead: every reached cell other than the source has a parent that
is its neighbour and one level closer. The edge lists are the oracle's (never
the CUDA path's), uploaded to the device.
"""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=["single", "levels"])
def dev(request):
    """Every test runs on both search forms: one cooperative launch for all
    levels, and one launch per level (CG_BFS_LEVELS=1)."""
    if request.param == "levels":
        os.environ["CG_BFS_LEVELS"] = "1"
    else:
        os.environ.pop("CG_BFS_LEVELS", None)
    yield from _device()
    os.environ.pop("CG_BFS_LEVELS", None)


def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    yield torch.device("cuda:0")


def _edges_dev(edges, dev):
    return torch.from_numpy(np.ascontiguousarray(edges, np.uint32).view(np.int32)).to(dev)


def _check(dev, edges, n, source):
    want = oracle.bfs(edges, n, source)
    dist, par, reached, depth = cellgraph.bfs(_edges_dev(edges, dev), n, source)
    got = dist.cpu().numpy()
    assert np.array_equal(got, want)
    assert reached == int((want >= 0).sum())
    assert depth == int(want.max())
    p = par.cpu().numpy()
    es = {(int(i), int(j)) for i, j in np.asarray(edges, np.int64).reshape(-1, 2)}
    for v in np.flatnonzero(want > 0)[:20000]:
        u = int(p[v])
        assert want[u] == want[v] - 1
        assert (min(u, int(v)), max(u, int(v))) in es
    assert p[source] == -1
    assert (p[want < 0] == -1).all()
    return got, p


@pytest.mark.gpu
@pytest.mark.parametrize("source", [0, 1234, 4095])
def test_bfs_hypercube(dev, source):
    ell = 12
    cells = np.arange(1 << ell, dtype=np.uint64).reshape(-1, 1)
    edges = oracle.neighbors(cells, ell, 64)
    got, _ = _check(dev, edges, 1 << ell, source)
    assert got.tolist() == [bin(v ^ source).count("1") for v in range(1 << ell)]


@pytest.mark.gpu
def test_bfs_arrangement_graph_and_path(dev):
    sc = inputs.planes_3d(n=300_000, ell=64, seed=8)
    cells, edges = oracle.build(sc.pts, sc.a, sc.b, 64)
    n = cells.shape[0]
    for source in (0, n // 2, n - 1):
        got, par = _check(dev, edges, n, source)
    # a path from the last source to the farthest cell, edge by edge
    far = int(np.argmax(got))
    path = cellgraph.path_to(par, n - 1, far)
    assert len(path) == got[far] + 1 and path[0] == n - 1 and path[-1] == far
    es = {(int(i), int(j)) for i, j in edges.astype(np.int64)}
    assert all((min(a, b), max(a, b)) in es for a, b in zip(path, path[1:]))


@pytest.mark.gpu
def test_bfs_many_components(dev):
    ch = inputs.chains(n_seeds=3000, ell=1024, seed=10)
    cells = oracle.dedup(ch.keys, 1024, 64)
    edges = oracle.neighbors(cells, 1024, 64)
    got, par = _check(dev, edges, cells.shape[0], 17)
    assert (got < 0).sum() > cells.shape[0] // 2  # most chains are unreachable
    assert cellgraph.path_to(par, 17, int(np.flatnonzero(got < 0)[0])) == []


@pytest.mark.gpu
def test_bfs_degenerate_graphs(dev):
    # one cell, no edges
    dist, par, reached, depth = cellgraph.bfs(torch.zeros((0, 2), dtype=torch.int32, device=dev),
                                              1, 0)
    assert dist.tolist() == [0] and par.tolist() == [-1] and (reached, depth) == (1, 0)
    # a long path (many levels, more than one group of eight), in shuffled order
    n = 1000
    edges = np.array([[i, i + 1] for i in range(n - 1)], np.uint32)
    edges = edges[np.random.default_rng(0).permutation(n - 1)]
    got, _ = _check(dev, edges, n, 0)
    assert got.tolist() == list(range(n))
    # endpoints >= n_cells are reported, not followed
    bad = _edges_dev(np.array([[0, 1], [1, 7]], np.uint32), dev)
    with pytest.raises(cellgraph.CellGraphError):
        cellgraph.bfs(bad, 5, 0)
    with pytest.raises(cellgraph.CellGraphError):
        cellgraph.bfs(_edges_dev(np.array([[0, 1]], np.uint32), dev), 2, 2)  # source >= n


@functools.lru_cache(maxsize=1)
def _benchmark_graph():
    sc = inputs.planes_3d()
    return oracle.build(sc.pts, sc.a, sc.b, 64)


@pytest.mark.gpu
def test_bfs_on_the_benchmark_graph(dev):
    """The 2^24-point planes_3d scene's graph (8,365 cells), every source
    distance checked, from two sources."""
    cells, edges = _benchmark_graph()
    for source in (0, cells.shape[0] - 1):
        _check(dev, edges, cells.shape[0], source)
