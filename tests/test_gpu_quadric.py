"""Quadric constraints (curved boundaries, §2.1) on the GPU against the oracle.

cg_pack_signs_quadric must give the oracle's sign vectors bit for bit: the
kernel decides almost every bit in fp32 with a proven error bound and settles
the rest in exact integer arithmetic, so any disagreement is a bug. Cases:
every point dimension, word widths 32 and 64, l across word and chunk
boundaries (and above 512, where the constraint rows are staged in groups),
ragged point counts, spheres, general quadrics, int32 extremes, points exactly
on the surfaces; then whole builds (pack, dedup, neighbours) of sphere scenes.
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
    return torch.device("cuda:0")


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def keys_np(t, word_bits):
    return t.cpu().numpy().view(np.uint64 if word_bits == 64 else np.uint32)


def _check_keys(sc, dev, word_bits):
    got = cellgraph.pack_signs_quadric(T(sc.pts, dev), T(sc.q, dev), T(sc.a, dev), T(sc.b, dev),
                                       word_bits)
    want = oracle.pack_signs_quadric(sc.pts, sc.q, sc.a, sc.b, word_bits)
    assert np.array_equal(keys_np(got, word_bits).reshape(want.shape), want)
    return want


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("ell,word_bits", [(5, 32), (33, 64), (64, 64), (100, 32), (200, 64)])
def test_quadrics_match_oracle(dev, d, ell, word_bits):
    sc = inputs.quadrics_3d(n=30_001, ell=ell, seed=90 + d, d=d, coord=1 << 18)
    want = _check_keys(sc, dev, word_bits)
    assert len(np.unique(want, axis=0)) >= min(8, ell)  # the surfaces cut the sampled region


@pytest.mark.parametrize("d", [2, 3])
def test_spheres_match_oracle(dev, d):
    sc = inputs.spheres_3d(n=200_003, ell=64, seed=91, d=d)
    want = _check_keys(sc, dev, 64)
    assert len(np.unique(want, axis=0)) > 100


def test_many_constraints_in_groups(dev):
    # l = 1300 > 512: the rows are staged in three groups per tile.
    sc = inputs.quadrics_3d(n=5_003, ell=1300, seed=92, coord=1 << 16)
    _check_keys(sc, dev, 64)
    _check_keys(sc, dev, 32)


def test_quadric_extremes_and_ties(dev):
    rng = np.random.default_rng(93)
    ell, d = 70, 3
    c = rng.integers(-(1 << 30) + 1, 1 << 30, size=(ell, d), dtype=np.int64)
    r = rng.integers(0, 1 << 31, size=ell, dtype=np.int64)
    q = np.zeros((ell, 6), np.int32)
    q[:, [0, 3, 5]] = 1
    a = (-2 * c).astype(np.int32)
    b = np.array([int(rr) ** 2 - sum(int(x) ** 2 for x in cc) for cc, rr in zip(c, r)], np.int64)
    lim = (1 << 31) - 1
    pts = rng.integers(-lim - 1, lim, size=(5000, d), dtype=np.int64, endpoint=True)
    # points exactly on spheres (ties satisfy the constraint) and at the centres
    for i in range(40):
        pts[i] = c[i] + [int(r[i]), 0, 0] if i % 2 else c[i] - [0, 0, int(r[i])]
    pts[40:50] = c[:10]
    pts = np.clip(pts, -lim - 1, lim).astype(np.int32)
    sc = inputs.QuadricScene(pts=pts, q=q, a=a, b=b)
    _check_keys(sc, dev, 64)
    # mixed general quadrics at the coefficient limits
    q2 = rng.integers(-lim - 1, lim, size=(ell, 6), dtype=np.int64, endpoint=True).astype(np.int32)
    a2 = rng.integers(-lim - 1, lim, size=(ell, 3), dtype=np.int64, endpoint=True).astype(np.int32)
    b2 = rng.integers(-(1 << 62), 1 << 62, size=ell, dtype=np.int64)
    _check_keys(inputs.QuadricScene(pts=pts, q=q2, a=a2, b=b2), dev, 64)


def test_quadric_empty_and_bad_arguments(dev):
    lib = cellgraph.load_library()
    z = torch.zeros(4, dtype=torch.int32, device=dev)
    assert lib.cg_pack_signs_quadric(None, 0, 3, None, None, None, 8, 64, None, None) == 0
    assert lib.cg_pack_signs_quadric(z.data_ptr(), 1, 5, z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), 8, 64, z.data_ptr(), None) == \
        cellgraph.ERR_INVALID_ARG


@pytest.mark.parametrize("strategy", ["auto", "halves"])
def test_sphere_build_matches_oracle(dev, strategy):
    sc = inputs.spheres_3d(n=1 << 20, ell=64)
    cells, edges = cellgraph.build_quadric(T(sc.pts, dev), T(sc.q, dev), T(sc.a, dev),
                                           T(sc.b, dev), 64, strategy=strategy)
    want_c, want_e = oracle.build_quadric(sc.pts, sc.q, sc.a, sc.b, 64)
    assert np.array_equal(keys_np(cells, 64).reshape(want_c.shape), want_c)
    assert np.array_equal(edges.cpu().numpy().view(np.uint32), want_e)
    assert len(want_e) > 0


def test_nested_spheres_build_closed_form(dev):
    # Concentric spheres: l + 1 thermometer cells on a path of l edges.
    ell = 40
    radii = (np.arange(1, ell + 1, dtype=np.int64) * 20_000)
    q = np.zeros((ell, 6), np.int32)
    q[:, [0, 3, 5]] = 1
    a = np.zeros((ell, 3), np.int32)
    b = radii * radii
    pts = inputs.spheres_3d(n=300_000, ell=1, seed=94).pts // 2  # |p| up to ~0.9e6
    cells, edges = cellgraph.build_quadric(T(pts, dev), T(q, dev), T(a, dev), T(b, dev), 64)
    got = keys_np(cells, 64).reshape(-1).tolist()
    assert got == [(1 << i) - 1 for i in range(ell + 1)]
    assert edges.cpu().numpy().tolist() == [[i, i + 1] for i in range(ell)]
