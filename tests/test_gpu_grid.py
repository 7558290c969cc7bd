"""The sign step's box grid against the oracle, bit for bit.

With the grid (tuning sign_kernel 2; 0, the default, from 2^18 points in
device memory on; 3 never uses it), most bits of a vector come from the cell
of a grid laid over the points, and only the constraints that cross the cell
are tested per point. The cells are classified a column
at a time from a few tests per (column, constraint), relying on the value
moving monotonically along the column. The cases aim at what that adds:
planes through cell corners with points on and next to them, points outside
the grid (never in the sample that places it), int32 coordinate and int64
offset extremes, constant constraints, every dimension, one and two
32-constraint chunks, and both word widths.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRID_ALWAYS, GRID_NEVER = 2, 3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch.device("cuda:0")


def _ctx(sign_kernel):
    c = cellgraph.Context(0)
    for b in range(cellgraph.TUNE_BUCKETS):
        c.tune_set(b, "hash", 4, sign_kernel)
    return c


@pytest.fixture(scope="module")
def gctx(dev):
    c = _ctx(GRID_ALWAYS)
    yield c
    c.close()


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def check(c, dev, pts, a, b, wb=64):
    cells, edges = c.build(T(pts, dev), T(a, dev), T(b, dev), wb)
    want_c, want_e = oracle.build(pts, a, b, wb)
    got_c = cells.cpu().numpy().view(np.uint64 if wb == 64 else np.uint32)
    assert np.array_equal(got_c.reshape(want_c.shape), want_c)
    assert np.array_equal(edges.cpu().numpy().view(np.uint32).reshape(-1, 2), want_e)
    return len(want_c)


def grid_geometry(pts):
    """The grid the library places over these points (its documented rule):
    per axis, cnt slabs of 2^s integers from lo, covering the range of 1,024
    evenly spaced sample points and 1/256 of it a side; s raised on the axis
    with the most slabs (the last of equal ones) until axis 0 has <= 256, the others <= 2048 together
    and all of them fit 2^total."""
    n, d = pts.shape
    lg = n.bit_length() - 1
    total = max(6, min(20, lg - 4))
    S = 1024
    idx = np.arange(n) if n <= S else (np.arange(S, dtype=np.int64) * (n - 1)) // (S - 1)
    first = [int(pts[idx, k].min()) for k in range(d)]
    ext = [int(pts[idx, k].max()) - first[k] + 1 for k in range(d)]
    want = [min(e + e // 128 + 2, 2**32) for e in ext]
    s, cnt = [0] * d, list(want)
    while True:  # axis 0 <= 256 slabs, the others <= 2048 together, all <= 2^total
        other = sum(cnt[1:])
        if cnt[0] > 256:
            kk = 0
        elif other > 2048 or np.prod([float(c) for c in cnt]) > 2.0 ** total:
            k0 = 1 if other > 2048 else 0
            kk = max((k for k in range(k0, d) if s[k] < 31), key=lambda k: (cnt[k], k))
        else:
            break
        s[kk] += 1
        cnt[kk] = -(-want[kk] // (1 << s[kk]))
    geo = []
    for k in range(d):
        span = cnt[k] << s[k]
        if span > 2**32:
            cnt[k] = 2**32 >> s[k]
            span = cnt[k] << s[k]
        lo = max(first[k] - (span - ext[k]) // 2, -2**31)
        if lo + span > 2**31:
            lo = 2**31 - span
        geo.append((lo, s[k], cnt[k]))
    return geo


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("ell", [17, 32, 64])
def test_grid_ties_and_extremes(gctx, dev, d, ell):
    """Points on and one unit off the constraints, int32 extremes, int64
    offsets at both ends and a constant constraint."""
    rng = np.random.default_rng(1000 + 10 * d + ell)
    n = 30_000
    a = rng.integers(-2**31, 2**31, size=(ell, d), dtype=np.int64).astype(np.int32)
    a[: ell // 3] = rng.integers(-3, 4, size=(ell // 3, d))
    pts = rng.integers(-2**31, 2**31, size=(n, d), dtype=np.int64).astype(np.int32)
    pts[: n // 2] = rng.integers(-50, 51, size=(n // 2, d))
    pts[n // 2: n // 2 + 8] = np.iinfo(np.int32).max
    pts[n // 2 + 8: n // 2 + 16] = np.iinfo(np.int32).min
    anchor = pts[rng.integers(0, n, size=ell)]
    bo = (a.astype(object) * anchor.astype(object)).sum(axis=1) + rng.integers(-1, 2, size=ell)
    b = np.array([max(min(int(v), 2**63 - 1), -2**63) for v in bo], dtype=np.int64)
    b[0] = np.iinfo(np.int64).min
    b[1] = np.iinfo(np.int64).max
    a[2], b[2] = 0, 0
    check(gctx, dev, pts, a, b)


@pytest.mark.parametrize("d", [2, 3])
def test_grid_planes_through_cell_corners(gctx, dev, d):
    """Constraints through (or one unit off) corners of the grid's cells, and
    points on and around those corners: the cells meeting at a corner are
    where a wrong cell classification would show."""
    rng = np.random.default_rng(70 + d)
    n, ell, R = 50_000, 64, 1 << 20
    pts = rng.integers(-R, R + 1, size=(n, d)).astype(np.int32)
    pts[0], pts[-1] = -R, R  # the sample's range, and so the grid, is fixed
    geo = grid_geometry(pts)
    corners = np.array([[lo + (int(rng.integers(1, cnt)) << s) for (lo, s, cnt) in geo]
                        for _ in range(ell)], dtype=np.int64)
    a = rng.integers(-1024, 1025, size=(ell, d)).astype(np.int32)
    a[: ell // 4] = 0
    for i in range(ell // 4):  # axis-parallel planes on a cell face
        a[i, i % d] = 1 if i % 2 else -1
    b = (a.astype(np.int64) * corners).sum(axis=1) + rng.integers(-1, 2, size=ell)
    offs = np.array(np.meshgrid(*[[-1, 0, 1]] * d, indexing="ij")).reshape(d, -1).T
    near = (corners[:, None, :] + offs[None, :, :]).reshape(-1, d)
    pts[1: 1 + len(near)] = np.clip(near, -R, R)
    assert check(gctx, dev, pts, a, b.astype(np.int64)) > 100


def test_grid_points_outside_the_grid(gctx, dev):
    """Points far outside the sampled range (indices the sample never reads)
    test every constraint; the rest use the grid."""
    sc = inputs.planes_3d(n=20_000, ell=64, seed=77)
    pts = sc.pts.copy()
    far = np.array([[2**31 - 1, 0, 0], [-2**31, 5, -5], [1 << 30, 1 << 30, -(1 << 30)],
                    [0, 0, (1 << 24) + 3], [-(1 << 21), 1 << 21, 3]], dtype=np.int32)
    pts[1: 1 + len(far)] = far
    pts[7: 12] = far // 3 + 7
    check(gctx, dev, pts, sc.a, sc.b)


@pytest.mark.parametrize("kind,n,d,ell,wb", [("lines", 20_000, 2, 16, 32),
                                             ("lines", 20_000, 2, 16, 64),
                                             ("planes", 262_147, 3, 64, 64),
                                             ("planes", 100_003, 3, 33, 32),
                                             ("rand", 9_001, 1, 64, 64),
                                             ("rand", 40_000, 4, 48, 32),
                                             ("rand", 5_000, 2, 1, 64)])
def test_grid_scenes(gctx, dev, kind, n, d, ell, wb):
    if kind == "lines":
        sc = inputs.lines_2d(n=n, ell=ell)
    elif kind == "planes":
        sc = inputs.planes_3d(n=n, ell=ell, seed=19)
    else:
        sc = inputs.arrangement(n + ell, n, d, ell, 1000, 10**6, 1000)
    assert check(gctx, dev, sc.pts, sc.a, sc.b, wb) >= 1


def test_grid_degenerate_inputs(gctx, dev):
    """One point; every point the same; constant constraints of both signs."""
    sc = inputs.planes_3d(n=1, ell=64, seed=3)
    check(gctx, dev, sc.pts, sc.a, sc.b)
    sc = inputs.planes_3d(n=5_000, ell=40, seed=4)
    same = np.repeat(sc.pts[:1], 5_000, axis=0)
    check(gctx, dev, same, sc.a, sc.b)
    a = sc.a.copy()
    b = sc.b.copy()
    a[:3] = 0
    b[:3] = [0, 1, -1]  # 0 >= 0 holds, 0 >= 1 fails, 0 >= -1 holds
    check(gctx, dev, sc.pts, a, b)


def test_grid_default_and_never_agree(dev):
    """The default setting (the grid from 2^18 points on) and the grid
    switched off give the oracle's output on a scene of 300,001 points."""
    sc = inputs.planes_3d(n=300_001, ell=64, seed=88)
    for sk in (0, GRID_NEVER):
        c = _ctx(sk)
        try:
            check(c, dev, sc.pts, sc.a, sc.b)
        finally:
            c.close()
