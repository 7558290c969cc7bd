"""Full-size outputs against the oracle, bit for bit, through stored digests.

The oracle needs minutes of CPU time for the long-vector workload and for the
1,024 batched scenes, so ``tests/golden/make_full_size_digests.py`` (which
calls only ``oracle/``) ran it once and stored SHA-256 digests of its complete
outputs: the cells as little-endian words [U][W], the edges as uint32 pairs
[E][2] in canonical order. These tests hash the complete GPU outputs the same
way and compare: every cell and every edge of every scene, not a sample.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1503_06029_gb300 import cellgraph, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIGESTS = os.path.join(os.path.dirname(__file__), "golden", "full_size_digests.json")


@pytest.fixture(scope="module")
def golden():
    with open(DIGESTS) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch.device("cuda:0")


def sha(t) -> str:
    return hashlib.sha256(np.ascontiguousarray(t.cpu().numpy()).tobytes()).hexdigest()


def check(entry, cells, edges):
    assert cells.shape[0] == entry["n_cells"]
    assert edges.shape[0] == entry["n_edges"]
    assert sha(cells) == entry["cells_sha256"]
    assert sha(edges) == entry["edges_sha256"]


def test_planes_3d_full_size_digest(dev, golden):
    sc = inputs.planes_3d()
    ctx = cellgraph.Context(0)
    try:
        args = tuple(torch.from_numpy(x).to(dev) for x in (sc.pts, sc.a, sc.b))
        cells, edges = ctx.build(*args, 64)
        check(golden["planes_3d"], cells, edges)
    finally:
        ctx.close()


def test_spheres_full_size_digest(dev, golden):
    """Quadric constraints at full size: l = 64 spheres over 2^24 points,
    through cg_pack_signs_quadric, cg_dedup_cells and cg_neighbors_h1."""
    sc = inputs.spheres_3d()
    args = [torch.from_numpy(x).to(dev) for x in (sc.pts, sc.q, sc.a, sc.b)]
    cells, edges = cellgraph.build_quadric(*args, 64)
    check(golden["spheres_3d"], cells, edges)


@pytest.mark.parametrize("strategy", ["hash", "pivot", "halves", "tree"])
def test_chains_full_size_digest(dev, golden, strategy):
    """l = 1024, N = 5,242,880 vectors: all 4,190,741 cells and all 3,932,003
    edges, for every lookup strategy that handles this size."""
    ch = inputs.chains()
    keys = torch.from_numpy(ch.keys.view(np.int64)).to(dev)
    del ch
    cells = cellgraph.dedup_cells(keys, 1024, 64)
    del keys
    edges = cellgraph.neighbors_h1(cells, 1024, 64, strategy=strategy)
    check(golden["chains"], cells, edges)


@pytest.mark.parametrize("tuning", ["default", "pivot_halves"])
def test_batch_1024_scenes_full_size_digest(dev, golden, tuning):
    """The 1,024 batched scenes (146.5 M points, 10.8 M cells, 17.3 M edges):
    every scene's cells and edges from one cg_build_batch call, run eagerly,
    captured into a CUDA graph and replayed; under the default lookups and
    under PIVOT (3 pivots) for 64 < l <= 128 with HALVES above."""
    spec = inputs.scene_batch_spec()
    scenes = []
    for s in range(len(spec.n)):
        sc = inputs.batch_scene(spec, s)
        scenes.append(tuple(torch.from_numpy(x).to(dev) for x in (sc.pts, sc.a, sc.b)))
    entries = golden["batch_scenes"]
    assert len(entries) == len(scenes)
    ctx = cellgraph.Context(0)
    if tuning == "pivot_halves":
        ctx.tune_set(cellgraph.TUNE_LIMITS.index(128), "pivot", 3)
        ctx.tune_set(cellgraph.TUNE_LIMITS.index(256), "halves")
    try:
        for rep in range(3):  # eager, captured, replayed
            got = ctx.build_batch(scenes)
            bad = [i for i, (c, e) in enumerate(got)
                   if c.shape[0] != entries[i]["n_cells"] or e.shape[0] != entries[i]["n_edges"]
                   or sha(c) != entries[i]["cells_sha256"] or sha(e) != entries[i]["edges_sha256"]]
            assert not bad, f"pass {rep}: scenes {bad[:10]} differ from the oracle"
    finally:
        ctx.close()
