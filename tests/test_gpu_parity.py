"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Everything here is integer and bit-level work, so the bar is bit-exact: packed
vectors, cells (in value order) and edge lists (in lexicographic order) must be
identical, element by element, to the oracle's on the same seeded inputs.

Sizes span several tiles and ragged tails (the sign kernel's tile is 1024
points, the radix tile 2048 items, the scan block 4096 items). The full-size
cases run the workloads at the sizes the benchmark times: the whole 2^24-point
3-D arrangement through the oracle, and the 5,242,880-vector chain workload
through sampled rows plus properties that hold at any size.
"""
import ctypes
import functools

import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs
from tests.helpers import as_u64_rows, popcount64, rows_to_ints

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(dev):
    c = cellgraph.Context(0)
    yield c
    c.close()


def T(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def words_np(t, word_bits):
    return t.cpu().numpy().view(np.uint64 if word_bits == 64 else np.uint32)


def words_dev(x, word_bits, dev):
    dt = np.int64 if word_bits == 64 else np.int32
    return T(np.ascontiguousarray(x).view(dt), dev)


def edges_np(t):
    return t.cpu().numpy().view(np.uint32).reshape(-1, 2)


def random_scene(seed, n, d, ell, coef=1000, off=10**6, coord=1000):
    return inputs.arrangement(seed, n, d, ell, coef, off, coord)


def tie_scene(seed, n, d, ell):
    """Points on and one unit off the constraints (a . p - b in {-1, 0, 1}),
    plus int32/int64 extremes: every bit near the fp32 filter's boundary."""
    rng = np.random.default_rng(seed)
    a = rng.integers(-2**31, 2**31, size=(ell, d), dtype=np.int64).astype(np.int32)
    a[: ell // 4] = rng.integers(-3, 4, size=(ell // 4, d))
    pts = rng.integers(-2**31, 2**31, size=(n, d), dtype=np.int64).astype(np.int32)
    pts[: n // 3] = rng.integers(-5, 6, size=(n // 3, d))
    pts[n // 3: n // 3 + 8] = np.iinfo(np.int32).max
    pts[n // 3 + 8: n // 3 + 16] = np.iinfo(np.int32).min
    # offsets through chosen points, so that ties and near-ties happen
    anchor = pts[rng.integers(0, n, size=ell)]
    b = (a.astype(object) * anchor.astype(object)).sum(axis=1) + rng.integers(-1, 2, size=ell)
    b = np.array([max(min(int(v), 2**63 - 1), -2**63) for v in b], dtype=np.int64)
    b[0] = np.iinfo(np.int64).min
    if ell > 1:
        b[1] = np.iinfo(np.int64).max
    a[2 % ell] = 0  # a constant constraint: 0 >= b
    b[2 % ell] = 0
    return inputs.Scene(pts=pts, a=a, b=b)


# ------------------------------- step 1 ----------------------------------

PACK_CASES = [
    ("lines", 20_000, 2, 16, 32),
    ("lines", 20_000, 2, 16, 64),
    ("planes", 200_003, 3, 64, 64),
    ("planes", 70_001, 3, 65, 64),
    ("planes", 50_000, 3, 100, 32),
    ("planes", 30_011, 3, 256, 64),
    ("rand", 4099, 1, 7, 64),
    ("rand", 4099, 4, 33, 32),
    ("rand", 1, 2, 1, 64),
    ("rand", 1023, 3, 31, 32),
]


@pytest.mark.parametrize("kind,n,d,ell,wb", PACK_CASES)
def test_pack_signs_matches_oracle(dev, kind, n, d, ell, wb):
    if kind == "lines":
        sc = inputs.lines_2d(n=n, ell=ell)
    elif kind == "planes":
        sc = inputs.planes_3d(n=n, ell=ell, seed=7)
    else:
        sc = random_scene(ell * 31 + d, n, d, ell)
    got = words_np(cellgraph.pack_signs(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), wb), wb)
    want = oracle.pack_signs(sc.pts, sc.a, sc.b, wb)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("d,ell", [(1, 40), (2, 64), (3, 97), (4, 130)])
def test_pack_signs_ties_and_extremes(dev, d, ell):
    sc = tie_scene(100 + d, 5000, d, ell)
    got = words_np(cellgraph.pack_signs(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64), 64)
    want = oracle.pack_signs(sc.pts, sc.a, sc.b, 64)
    assert np.array_equal(got, want)


def test_pack_signs_unaligned_points(dev):
    sc = inputs.planes_3d(n=10_001, ell=64, seed=5)
    buf = T(np.concatenate([[0], sc.pts.reshape(-1)]).astype(np.int32), dev)
    pts = buf[1:].view(-1, 3)  # 4-byte offset: not 16-byte aligned
    got = words_np(cellgraph.pack_signs(pts, T(sc.a, dev), T(sc.b, dev), 64), 64)
    assert np.array_equal(got, oracle.pack_signs(sc.pts, sc.a, sc.b, 64))


# ------------------------------- step 2 ----------------------------------

def _dedup_case(kind, wb):
    if kind == "lines":
        sc = inputs.lines_2d()
        return oracle.pack_signs(sc.pts, sc.a, sc.b, wb), 16
    if kind == "planes64":
        sc = inputs.planes_3d(n=300_000, ell=64, seed=8)
        return oracle.pack_signs(sc.pts, sc.a, sc.b, wb), 64
    if kind == "planes200":
        sc = inputs.planes_3d(n=100_000, ell=200, seed=9)
        return oracle.pack_signs(sc.pts, sc.a, sc.b, wb), 200
    if kind == "chains":
        ch = inputs.chains(n_seeds=3000, ell=1024, seed=10)
        keys = ch.keys if wb == 64 else ch.keys.view(np.uint32)
        return keys, 1024
    if kind == "chains130":
        ch = inputs.chains(n_seeds=5000, ell=130, seed=11)
        return ch.keys, 130
    raise ValueError(kind)


@pytest.mark.parametrize("kind,wb", [("lines", 32), ("lines", 64), ("planes64", 64),
                                     ("planes200", 64), ("planes200", 32), ("chains", 64),
                                     ("chains", 32), ("chains130", 64)])
def test_dedup_matches_oracle(dev, kind, wb):
    keys, ell = _dedup_case(kind, wb)
    cells, pc = cellgraph.dedup_cells(words_dev(keys, wb, dev), ell, wb, point_cell=True)
    want, want_pc = oracle.dedup(keys, ell, wb, point_cell=True)
    assert np.array_equal(words_np(cells, wb), want)
    assert np.array_equal(pc.cpu().numpy().view(np.uint32), want_pc)


@pytest.mark.parametrize("ell,runs", [(1024, [2, 3, 17, 29, 30]), (1024, [2, 31]),
                                      (1024, [2, 5, 200]), (4096, [2, 6, 7]),
                                      (4096, [3, 8]), (200, [2, 40, 64]), (200, [65, 300]),
                                      (256, [64, 65, 340, 2048]), (256, [3, 2049]),
                                      (140, [70, 500])])
def test_dedup_runs_sharing_the_top_bits(dev, ell, runs):
    """Rows longer than the cached 128-bit key that share their top 128 bits
    in runs of the given lengths (shuffled, with duplicates): short runs are
    ordered by one warp each, a run longer than a warp's share of shared
    memory sends the whole sort through the full-row comparison pass."""
    rng = np.random.default_rng(ell + len(runs))
    w = (ell + 63) // 64
    rows = []
    for m in runs:
        top = rng.integers(0, 2**63, size=w, dtype=np.int64).astype(np.uint64)
        if ell % 64:
            top[-1] &= np.uint64((1 << (ell % 64)) - 1)
        for _ in range(m):
            r = top.copy()
            r[: w - 2] = rng.integers(0, 2**63, size=w - 2, dtype=np.int64).astype(np.uint64)
            r[w - 3] &= np.uint64(0xFF)  # runs differ only far below the top
            rows.append(r)
    keys = np.stack(rows)
    keys = np.concatenate([keys, keys[rng.choice(len(keys), size=len(keys) // 3)]])
    keys = keys[rng.permutation(len(keys))]
    cells = cellgraph.dedup_cells(words_dev(keys, 64, dev), ell, 64)
    assert np.array_equal(words_np(cells, 64), oracle.dedup(keys, ell, 64))


def test_dedup_all_duplicates_and_empty(dev):
    keys = np.full((5000, 1), 12345, dtype=np.uint64)
    cells = cellgraph.dedup_cells(words_dev(keys, 64, dev), 20, 64)
    assert words_np(cells, 64).tolist() == [[12345]]
    empty = cellgraph.dedup_cells(words_dev(np.zeros((0, 1), np.uint64), 64, dev), 20, 64)
    assert empty.shape[0] == 0


# ------------------------------ steps 3-4 --------------------------------

@pytest.mark.parametrize("strategy", ["hash", "sorted", "pivot", "tree", "halves", "allpairs"])
@pytest.mark.parametrize("kind,wb", [("lines", 32), ("planes64", 64), ("planes200", 64),
                                     ("planes200", 32), ("chains", 64), ("chains130", 64)])
def test_neighbors_match_oracle(dev, kind, wb, strategy):
    keys, ell = _dedup_case(kind, wb)
    cells = oracle.dedup(keys, ell, wb)
    got = cellgraph.neighbors_h1(words_dev(cells, wb, dev), ell, wb, strategy=strategy)
    want = oracle.neighbors(cells, ell, wb)
    assert np.array_equal(edges_np(got), want)
    assert len(want) > 0


@pytest.mark.parametrize("strategy", ["hash", "sorted", "pivot", "tree", "halves", "allpairs"])
def test_neighbors_hypercube(dev, strategy):
    ell = 12
    cells = np.arange(1 << ell, dtype=np.uint64).reshape(-1, 1)
    got = edges_np(cellgraph.neighbors_h1(words_dev(cells, 64, dev), ell, 64, strategy=strategy))
    assert len(got) == ell * (1 << (ell - 1))
    assert np.array_equal(got, oracle.neighbors(cells, ell, 64))


@pytest.mark.parametrize("pivots", ["1", "2", "5", "8"])
def test_neighbors_pivot_counts(dev, pivots, monkeypatch):
    """Any number of pivots gives the same edges (wide and small vectors)."""
    monkeypatch.setenv("CG_PIVOTS", pivots)
    for kind, wb in (("planes64", 64), ("chains130", 64), ("planes200", 32)):
        keys, ell = _dedup_case(kind, wb)
        cells = oracle.dedup(keys, ell, wb)
        got = cellgraph.neighbors_h1(words_dev(cells, wb, dev), ell, wb, strategy="pivot")
        assert np.array_equal(edges_np(got), oracle.neighbors(cells, ell, wb))


def test_neighbors_tree_degenerate_shapes(dev):
    """Tree corner cases: one cell, two cells differing in the lowest bit only
    (a single long shared prefix), l not a multiple of the digit width."""
    for ell, vals in ((5, [3]), (64, [0, 1]), (70, [0, 1, 1 << 69, (1 << 69) | 1]),
                      (13, list(range(0, 1 << 13, 3)))):
        cells = np.array([[v & ((1 << 64) - 1), v >> 64] if ell > 64 else [v] for v in vals],
                         dtype=np.uint64)
        want = oracle.neighbors(cells, ell, 64)
        got = cellgraph.neighbors_h1(words_dev(cells, 64, dev), ell, 64, strategy="tree")
        assert np.array_equal(edges_np(got), want), ell


@pytest.mark.parametrize("ell", [1, 2, 3, 17, 63, 64, 65, 127, 128, 129, 200, 1030])
def test_neighbors_halves_split_positions(dev, ell):
    """HALVES splits the bits at s = l // 2: partners that differ just below
    and just above s, at bit 0 and at bit l - 1, inside one word and across
    word boundaries, plus cells that agree on one part with many others (long
    runs) and random rows."""
    rng = np.random.default_rng(ell)
    w = (ell + 63) // 64
    s = ell // 2

    def row(v):
        return [(v >> (64 * q)) & ((1 << 64) - 1) for q in range(w)]

    vals = set()
    for _ in range(200):
        base = int(rng.integers(0, 2**62)) | (int(rng.integers(0, 2**62)) << 62)
        base |= int(rng.integers(0, 2**62)) << 124
        base &= (1 << ell) - 1
        vals.add(base)
        for k in {0, ell - 1, max(s - 1, 0), min(s, ell - 1), min(s + 1, ell - 1),
                  int(rng.integers(0, ell))}:
            vals.add(base ^ (1 << k))
    hi = int(rng.integers(0, 2**62)) << s & ((1 << ell) - 1)
    for lo in range(min(1 << s, 64)):  # one run of equal high part
        vals.add(hi | lo)
    cells = np.array([row(v) for v in sorted(vals)], dtype=np.uint64)
    want = oracle.neighbors(cells, ell, 64)
    got = cellgraph.neighbors_h1(words_dev(cells, 64, dev), ell, 64, strategy="halves")
    assert np.array_equal(edges_np(got), want)
    if ell > 2:
        assert len(want) > 0


@pytest.mark.parametrize("pivots", ["1", "2", "4", "8"])
def test_neighbors_allpairs_against_the_heuristic_oracle(dev, pivots, monkeypatch):
    """ALLPAIRS is Algorithm 2 on the device: its edges equal those of the
    oracle's literal heuristic (Algorithms 1-2, pivots = the first h cells;
    the device spreads its pivots over the sorted cells instead -- any
    pivots give the same edges) for any pivot count."""
    monkeypatch.setenv("CG_PIVOTS", pivots)
    for kind, wb in (("lines", 32), ("chains130", 64)):
        keys, ell = _dedup_case(kind, wb)
        cells = oracle.dedup(keys, ell, wb)[:3000]
        want, _ = oracle.heuristic(cells, ell, wb, h=int(pivots))
        got = cellgraph.neighbors_h1(words_dev(cells, wb, dev), ell, wb, strategy="allpairs")
        assert np.array_equal(edges_np(got), want), kind
        assert len(want) > 0


def test_neighbors_reject_bits_above_l(dev):
    """Cells whose last word has a bit at or above l are invalid input (the
    wide search reads 64-bit rows in place and checks them)."""
    rng = np.random.default_rng(3)
    vals = sorted({int(v) for v in rng.integers(0, 2**62, size=50)})
    cells = np.array([[v, 0] for v in vals], dtype=np.uint64)
    ok = cellgraph.neighbors_h1(words_dev(cells, 64, dev), 100, 64, strategy="halves")
    assert np.array_equal(edges_np(ok), oracle.neighbors(cells, 100, 64))
    bad = cells.copy()
    bad[-1, 1] = np.uint64(1) << np.uint64(40)  # bit 104 >= l = 100
    for strategy in ("hash", "halves", "tree"):
        with pytest.raises(cellgraph.CellGraphError, match="at or above"):
            cellgraph.neighbors_h1(words_dev(bad, 64, dev), 100, 64, strategy=strategy)


def test_neighbors_pivot_wide_4096(dev):
    """The longest vectors (l = 4096, 64 words): random rows plus one-bit
    variants at every word position."""
    rng = np.random.default_rng(17)
    ell = 4096
    base = rng.integers(0, 2**63, size=(300, 64), dtype=np.int64).astype(np.uint64)
    rows = [base]
    for k in range(0, ell, 37):
        v = base[k % 300].copy()
        v[k // 64] ^= np.uint64(1) << np.uint64(k % 64)
        rows.append(v[None])
    keys = np.concatenate(rows)
    cells = oracle.dedup(keys, ell, 64)
    want = oracle.neighbors(cells, ell, 64)
    assert len(want) > 50
    for strategy in ("hash", "sorted", "pivot", "tree", "halves", "allpairs"):
        got = cellgraph.neighbors_h1(words_dev(cells, 64, dev), ell, 64, strategy=strategy)
        assert np.array_equal(edges_np(got), want), strategy


def test_neighbors_edge_capacity(dev):
    keys, ell = _dedup_case("planes64", 64)
    cells = oracle.dedup(keys, ell, 64)
    want = oracle.neighbors(cells, ell, 64)
    small = cellgraph.neighbors_h1(words_dev(cells, 64, dev), ell, 64, edges_cap=10)
    assert np.array_equal(edges_np(small), want)  # binding retried with the reported E


# ------------------------------ full build -------------------------------

BUILD_CASES = [
    ("lines", 20_000, 16, 32),
    ("lines", 20_000, 16, 64),
    ("planes", 1, 64, 64),
    ("planes", 1000, 8, 64),
    ("planes", 262_147, 64, 64),
    ("planes", 100_000, 33, 32),
    ("planes", 60_000, 100, 64),
    ("planes", 40_000, 256, 64),
    ("planes", 20_000, 1, 64),
]


@pytest.mark.parametrize("kind,n,ell,wb", BUILD_CASES)
def test_build_matches_oracle(ctx, dev, kind, n, ell, wb):
    sc = inputs.lines_2d(n=n, ell=ell) if kind == "lines" else inputs.planes_3d(n=n, ell=ell,
                                                                               seed=12)
    cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), wb)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, wb)
    assert np.array_equal(words_np(cells, wb), want_c)
    assert np.array_equal(edges_np(edges), want_e)


@pytest.mark.parametrize("d,ell,n,wb", [(4, 4096, 3000, 64), (1, 300, 5000, 32),
                                        (2, 2000, 8000, 32), (4, 129, 20_000, 64),
                                        (1, 4096, 2000, 32)])
def test_build_any_dimension_and_length(ctx, dev, d, ell, n, wb):
    """Every point dimension up to 4 with long vectors, up to the longest
    l = 4096 (the multi-pass wide path), in both word widths."""
    sc = random_scene(ell + 7 * d, n, d, ell)
    cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), wb)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, wb)
    assert np.array_equal(words_np(cells, wb), want_c)
    assert np.array_equal(edges_np(edges), want_e)
    assert len(want_c) > 1


def test_build_ties_and_extremes(ctx, dev):
    for d, ell in [(2, 40), (3, 64), (4, 97)]:
        sc = tie_scene(200 + d, 30_000, d, ell)
        cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
        assert np.array_equal(words_np(cells, 64), want_c)
        assert np.array_equal(edges_np(edges), want_e)


def test_build_ties_inside_tensor_range(ctx, dev):
    """Exact ties (a . p = b) and off-by-one values with every magnitude inside
    the range of the exact fp16 split: the tensor-core path must decide them."""
    rng = np.random.default_rng(31)
    ell, n = 64, 200_000
    a = rng.integers(-1024, 1025, size=(ell, 3)).astype(np.int32)
    pts = rng.integers(-(1 << 19), (1 << 19) + 1, size=(n, 3)).astype(np.int32)
    anchors = pts[rng.integers(0, n, size=ell)]
    b = (a.astype(np.int64) * anchors).sum(axis=1) + rng.integers(-1, 2, size=ell)
    pts[: n // 2] = anchors[rng.integers(0, ell, size=n // 2)]  # many points on planes
    cells, edges = ctx.build(T(pts, dev), T(a, dev), T(b.astype(np.int64), dev), 64)
    want_c, want_e = oracle.build(pts, a, b, 64)
    assert np.array_equal(words_np(cells, 64), want_c)
    assert np.array_equal(edges_np(edges), want_e)


def test_build_mixed_tile_ranges(ctx, dev):
    """Some 128-point tiles hold coordinates beyond the exact-split range
    (|p| >= 2^22): those tiles go through the fp32 path, the rest through the
    tensor cores; together they must still match the oracle."""
    sc = inputs.planes_3d(n=300_000, ell=64, seed=41)
    pts = sc.pts.copy()
    rng = np.random.default_rng(5)
    far = rng.choice(len(pts), size=300, replace=False)
    pts[far] = rng.integers(-(1 << 26), 1 << 26, size=(300, 3)).astype(np.int32)
    cells, edges = ctx.build(T(pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
    want_c, want_e = oracle.build(pts, sc.a, sc.b, 64)
    assert np.array_equal(words_np(cells, 64), want_c)
    assert np.array_equal(edges_np(edges), want_e)


@pytest.mark.parametrize("kernel", ["tc", "ffma"])
def test_build_both_sign_kernels(ctx, dev, kernel, monkeypatch):
    monkeypatch.setenv("CG_SIGN_KERNEL", kernel)
    for sc, wb in [(inputs.lines_2d(), 32), (inputs.planes_3d(n=250_001, ell=64, seed=42), 64),
                   (inputs.planes_3d(n=99_999, ell=20, seed=43), 64)]:
        cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), wb)
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, wb)
        assert np.array_equal(words_np(cells, wb), want_c)
        assert np.array_equal(edges_np(edges), want_e)


def test_build_all_ones_vector(ctx, dev):
    # l = 64, constraints 1..63 always hold (0 >= 0); constraint 0 is x >= 0:
    # the cells are ~0 - 1 and ~0 (the all-ones vector, kept off the table).
    a = np.zeros((64, 2), np.int32)
    a[0] = (1, 0)
    b = np.zeros(64, np.int64)
    pts = np.array([[5, 1], [-5, 2], [0, 0], [-1, 9]] * 700, np.int32)
    cells, edges = ctx.build(T(pts, dev), T(a, dev), T(b, dev), 64)
    assert words_np(cells, 64).reshape(-1).tolist() == [2**64 - 2, 2**64 - 1]
    assert edges_np(edges).tolist() == [[0, 1]]
    want_c, want_e = oracle.build(pts, a, b, 64)
    assert np.array_equal(words_np(cells, 64), want_c) and np.array_equal(edges_np(edges), want_e)


def test_build_degenerate_inputs(ctx, dev):
    sc = inputs.planes_3d(n=0, ell=20)
    cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
    assert cells.shape[0] == 0 and edges.shape[0] == 0
    pts = np.tile(np.array([[3, -4, 5]], np.int32), (9000, 1))  # one point, repeated
    sc = inputs.planes_3d(n=1, ell=70)
    cells, edges = ctx.build(T(pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
    want_c, want_e = oracle.build(pts, sc.a, sc.b, 64)
    assert np.array_equal(words_np(cells, 64), want_c) and len(want_c) == 1
    assert edges.shape[0] == 0


@pytest.mark.parametrize("ell", [64, 200])
def test_build_overflowing_first_guess(dev, ell, monkeypatch):
    """A first table guess of 1024 slots (512 vectors) overflows; the build is
    re-run with 4x the capacity until it fits, with the same output."""
    monkeypatch.setenv("CG_FIRST_TABLE_CAP", "1024")
    sc = inputs.planes_3d(n=300_000, ell=ell, seed=12)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    assert len(want_c) > 512
    c2 = cellgraph.Context(0)
    try:
        cells, edges = c2.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
        assert np.array_equal(words_np(cells, 64).reshape(want_c.shape), want_c)
        assert np.array_equal(edges_np(edges), want_e)
        scenes = _batch_scenes(6, 100_000, seed=13) + [sc]
        got = c2.build_batch([(T(x.pts, dev), T(x.a, dev), T(x.b, dev)) for x in scenes])
        for x, (c, e) in zip(scenes, got):
            wc, we = oracle.build(x.pts, x.a, x.b, 64)
            assert np.array_equal(words_np(c, 64).reshape(wc.shape), wc)
            assert np.array_equal(edges_np(e), we)
    finally:
        c2.close()


def test_build_coincident_opposite_planes(ctx, dev):
    # Degenerate arrangement with many coincident, oppositely oriented planes:
    # points on them carry vectors that no open cell has.
    rng = np.random.default_rng(3)
    base = rng.integers(-50, 51, size=(8, 2)).astype(np.int32)
    a = np.concatenate([base, -base, base, -base])
    b = np.zeros(32, np.int64)
    pts = rng.integers(-300, 301, size=(50_000, 2)).astype(np.int32)
    cells, edges = ctx.build(T(pts, dev), T(a, dev), T(b, dev), 64)
    want_c, want_e = oracle.build(pts, a, b, 64)
    assert np.array_equal(words_np(cells, 64), want_c)
    assert np.array_equal(edges_np(edges), want_e)


def test_build_capacity_contract(ctx, dev):
    """Too-small outputs: CG_ERR_CAPACITY, both counts written, nothing written
    past either capacity."""
    sc = inputs.planes_3d(n=50_000, ell=64, seed=4)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    lib = cellgraph.load_library()
    cells = torch.full((10, 1), -7, dtype=torch.int64, device=dev)
    edges = torch.full((20, 2), -7, dtype=torch.int32, device=dev)
    nc, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    pts, a, b = T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev)
    P = ctypes.c_void_p
    rc = lib.cg_build(ctx._h, P(pts.data_ptr()), sc.n, 3, P(a.data_ptr()), P(b.data_ptr()), 64,
                      64, P(cells.data_ptr()), 5, ctypes.byref(nc), P(edges.data_ptr()), 8,
                      ctypes.byref(ne), P(torch.cuda.current_stream().cuda_stream))
    assert rc == cellgraph.ERR_CAPACITY
    assert nc.value == len(want_c) and ne.value == len(want_e)
    assert (cells[5:] == -7).all() and (edges[8:] == -7).all()


@pytest.mark.parametrize("mode", ["direct", "pieces", "copy"])
def test_build_host_pinned_points(ctx, dev, mode, monkeypatch):
    """Points in pinned host memory: read in place by the sign kernel
    (default), copied in pieces overlapping it (CG_HOST_INPUT=pieces) or
    copied first (CG_HOST_INPUT=copy); same output every way, including a
    ragged last piece."""
    if mode != "direct":
        monkeypatch.setenv("CG_HOST_INPUT", mode)
    sc = inputs.planes_3d(n=1_000_003, ell=64, seed=43)
    pts = torch.from_numpy(sc.pts).pin_memory().numpy()
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    for _ in range(3):  # eager, captured, replayed
        cells, edges = ctx.build_host(pts, sc.a, sc.b, 64)
        assert np.array_equal(cells.reshape(want_c.shape), want_c)
        assert np.array_equal(edges, want_e)


def test_build_host_matches_oracle(ctx, dev):
    for sc, wb in [(inputs.lines_2d(), 32), (inputs.planes_3d(n=123_457, ell=64, seed=6), 64)]:
        cells, edges = ctx.build_host(sc.pts, sc.a, sc.b, wb)
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, wb)
        assert np.array_equal(cells, want_c)
        assert np.array_equal(edges, want_e)


def test_build_is_deterministic(ctx, dev):
    sc = inputs.planes_3d(n=500_000, ell=64, seed=13)
    args = (T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
    c1, e1 = ctx.build(*args)
    c2, e2 = ctx.build(*args)
    assert torch.equal(c1, c2) and torch.equal(e1, e2)


# ------------------------------ full sizes -------------------------------

def test_full_size_planes_3d(ctx, dev):
    """The benchmark workload: l = 64 planes, N = 2^24 points, whole oracle."""
    sc = inputs.planes_3d()
    cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    assert np.array_equal(words_np(cells, 64), want_c)
    assert np.array_equal(edges_np(edges), want_e)
    assert len(want_c) <= 43_745  # sum_{k<=3} C(64, k)


def test_full_size_lines_2d(ctx, dev):
    sc = inputs.lines_2d()
    cells, edges = ctx.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 32)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 32)
    assert np.array_equal(words_np(cells, 32), want_c)
    assert np.array_equal(edges_np(edges), want_e)


def test_full_size_chains(dev):
    """l = 1024, N = 5,242,880: cells against the oracle in full; edges against
    the oracle on 3,000 sampled cells, plus properties of the whole list."""
    ch = inputs.chains()
    keys_d = words_dev(ch.keys, 64, dev)
    cells = cellgraph.dedup_cells(keys_d, 1024, 64)
    del keys_d
    edges = cellgraph.neighbors_h1(cells, 1024, 64)
    for strategy in ("pivot", "tree", "halves"):
        other = cellgraph.neighbors_h1(cells, 1024, 64, strategy=strategy)
        assert torch.equal(other, edges), strategy
        del other
    got_c = words_np(cells, 64)
    got_e = edges_np(edges).astype(np.int64)
    want_c = oracle.dedup(ch.keys, 1024, 64)
    assert np.array_equal(got_c, want_c)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(len(want_c), size=3000, replace=False))
    want_rows = oracle.neighbors(want_c, 1024, 64, rows=rows)
    sel = got_e[np.isin(got_e[:, 0], rows)]
    assert np.array_equal(sel.astype(np.uint32), want_rows)
    # properties of the whole list: i < j, sorted, unique, distance exactly 1
    assert (got_e[:, 0] < got_e[:, 1]).all()
    key = got_e[:, 0] * len(got_c) + got_e[:, 1]
    assert (np.diff(key) > 0).all()
    for lo in range(0, len(got_e), 1 << 19):
        blk = got_e[lo: lo + (1 << 19)]
        x = got_c[blk[:, 0]] ^ got_c[blk[:, 1]]
        assert (popcount64(x).sum(axis=1) == 1).all()
    # planted chain edges that survive are present
    order = np.lexsort(tuple(got_c[:, j] for j in range(got_c.shape[1])))
    assert (order == np.arange(len(got_c))).all()
    base_par = ch.base[ch.planted[:, 0]]
    base_chi = ch.base[ch.planted[:, 1]]
    dist = popcount64(base_par ^ base_chi).sum(axis=1)
    keep = dist == 1
    assert keep.mean() > 0.99
    # locate rows through a 64-bit row hash (MurmurHash3 finaliser of every
    # word, XOR-combined), then verify whole rows
    def row_hash(rows):
        h = np.zeros(rows.shape[0], dtype=np.uint64)
        for j in range(rows.shape[1]):
            x = rows[:, j] ^ np.uint64((0x9E3779B97F4A7C15 * (j + 1)) % 2**64)
            x = x ^ (x >> np.uint64(33))
            x = x * np.uint64(0xFF51AFD7ED558CCD)
            x = x ^ (x >> np.uint64(33))
            x = x * np.uint64(0xC4CEB9FE1A85EC53)
            x = x ^ (x >> np.uint64(33))
            h ^= x
        return h

    fc = row_hash(got_c)
    fo = np.argsort(fc, kind="stable")
    fs = fc[fo]

    def find(q):
        idx = fo[np.clip(np.searchsorted(fs, row_hash(q)), 0, len(fs) - 1)]
        assert (got_c[idx] == q).all()
        return idx.astype(np.int64)

    pi, ci = find(base_par[keep]), find(base_chi[keep])
    lo_, hi_ = np.minimum(pi, ci), np.maximum(pi, ci)
    planted = lo_ * len(got_c) + hi_
    assert np.isin(planted, key).all()


# ------------------------------- batches ---------------------------------

def _batch_scenes(n_scenes, n_hi, seed=4):
    spec = inputs.scene_batch_spec(n_scenes=n_scenes, seed=seed, n_hi=n_hi)
    return [inputs.batch_scene(spec, s) for s in range(n_scenes)]


def test_batch_matches_oracle_and_plain(ctx, dev):
    scenes = _batch_scenes(40, 30_000)
    scenes.insert(7, inputs.planes_3d(n=0, ell=24, seed=1))  # an empty scene
    dscenes = [(T(s.pts, dev), T(s.a, dev), T(s.b, dev)) for s in scenes]
    got = ctx.build_batch(dscenes)
    assert len(got) == len(scenes)
    for sc, (pts, a, b), (c, e) in zip(scenes, dscenes, got):
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
        assert np.array_equal(words_np(c, 64).reshape(want_c.shape), want_c)
        assert np.array_equal(edges_np(e), want_e)
        pc, pe = ctx.build(pts, a, b, 64)
        assert torch.equal(pc, c) and torch.equal(pe, e)


def test_batch_mixed_dimensions_and_widths(ctx, dev):
    """Scenes of every dimension and of 1 to 5 words in one batch: those of
    64 < l <= 256 and d <= 3 take the segmented wide path (one chain per
    (d, words) group on its own stream), d = 4 and l > 256 their per-scene
    pipelines, l <= 64 the segmented small path; each equals the oracle."""
    cases = [(1, 70), (1, 200), (2, 65), (2, 129), (2, 256), (3, 96), (3, 160), (3, 250),
             (4, 100), (3, 300), (1, 20), (2, 64), (3, 40), (4, 48), (2, 190), (3, 128)]
    scenes = [inputs.arrangement((7, i), 4_000 + 1_500 * i, d, ell, 1000, 1_000_000, 1000)
              for i, (d, ell) in enumerate(cases)]
    dscenes = [(T(s.pts, dev), T(s.a, dev), T(s.b, dev)) for s in scenes]
    wanted = [oracle.build(sc.pts, sc.a, sc.b, 64) for sc in scenes]
    for _ in range(3):  # eager, then captured, then replayed
        got = ctx.build_batch(dscenes)
        for (want_c, want_e), (c, e) in zip(wanted, got):
            assert np.array_equal(words_np(c, 64).reshape(want_c.shape), want_c)
            assert np.array_equal(edges_np(e), want_e)


def test_batch_repeated_and_resized(ctx, dev):
    """Repeating a batch gives the same bytes; a degenerate scene whose cell
    count exceeds the first table-size guess is resized and rerun inside the
    call."""
    rng = np.random.default_rng(3)
    base = rng.integers(-50, 51, size=(8, 2)).astype(np.int32)
    a = np.concatenate([base, -base, base, -base])
    deg = inputs.Scene(pts=rng.integers(-300, 301, size=(50_000, 2)).astype(np.int32), a=a,
                       b=np.zeros(32, np.int64))
    scenes = _batch_scenes(12, 20_000, seed=9) + [deg]
    dscenes = [(T(s.pts, dev), T(s.a, dev), T(s.b, dev)) for s in scenes]
    first = [(c.clone(), e.clone()) for c, e in ctx.build_batch(dscenes)]
    for _ in range(3):  # eager, then captured into a CUDA graph, then replayed
        again = ctx.build_batch(dscenes)
        for (c1, e1), (c2, e2) in zip(first, again):
            assert torch.equal(c1, c2) and torch.equal(e1, e2)
    second = again
    want_c, want_e = oracle.build(deg.pts, deg.a, deg.b, 64)
    assert np.array_equal(words_np(second[-1][0], 64).reshape(want_c.shape), want_c)
    assert np.array_equal(edges_np(second[-1][1]), want_e)


def test_batch_capacity_contract(ctx, dev):
    scenes = _batch_scenes(6, 5_000, seed=11)
    dscenes = [(T(s.pts, dev), T(s.a, dev), T(s.b, dev)) for s in scenes]
    lib = cellgraph.load_library()
    S = len(scenes)
    arr = (cellgraph.CgScene * S)()
    for i, (p, a, b) in enumerate(dscenes):
        arr[i] = cellgraph.CgScene(p.data_ptr(), p.shape[0], p.shape[1], a.data_ptr(),
                                   b.data_ptr(), a.shape[0])
    cells = torch.full((4,), -7, dtype=torch.int64, device=dev)
    edges = torch.full((4, 2), -7, dtype=torch.int32, device=dev)
    nc, ne = np.zeros(S, np.int64), np.zeros(S, np.int64)
    co, eo = np.zeros(S + 1, np.int64), np.zeros(S + 1, np.int64)
    out = cellgraph.CgBatchOut(cells.data_ptr(), 4, edges.data_ptr(), 4, nc.ctypes.data,
                               ne.ctypes.data, co.ctypes.data, eo.ctypes.data)
    rc = lib.cg_build_batch(ctx._h, ctypes.cast(arr, ctypes.c_void_p), S, ctypes.byref(out),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cellgraph.ERR_CAPACITY
    for i, sc in enumerate(scenes):
        want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
        assert nc[i] == len(want_c) and ne[i] == len(want_e)
    assert co[S] == sum(int(x) * ((s.ell + 63) // 64) for x, s in zip(nc, scenes))
    assert (cells == -7).all() and (edges == -7).all()


# ------------------------------ tuning ------------------------------------

def _tuning_scenes():
    return [inputs.planes_3d(n=60_000, ell=24, seed=31), inputs.planes_3d(n=80_000, ell=64, seed=32),
            inputs.planes_3d(n=50_000, ell=200, seed=33),
            inputs.planes_3d(n=20_000, ell=1500, seed=34),
            random_scene(35, 3000, 4, 4096)]


@functools.lru_cache(maxsize=None)
def _tuning_want(k):
    sc = _tuning_scenes()[k]
    return oracle.build(sc.pts, sc.a, sc.b, 64)


@pytest.mark.parametrize("setting", [("hash", 4, 0), ("sorted", 4, 0), ("pivot", 1, 0),
                                     ("pivot", 3, 0), ("pivot", 4, 1), ("hash", 4, 1),
                                     ("tree", 4, 0), ("halves", 4, 0)])
def test_build_under_every_tuning(dev, setting):
    strategy, pivots, sk = setting
    c2 = cellgraph.Context(0)
    try:
        for b in range(cellgraph.TUNE_BUCKETS):
            c2.tune_set(b, strategy, pivots, sk)
        for k, sc in enumerate(_tuning_scenes()):
            cells, edges = c2.build(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), 64)
            want_c, want_e = _tuning_want(k)
            assert np.array_equal(words_np(cells, 64).reshape(want_c.shape), want_c)
            assert np.array_equal(edges_np(edges), want_e)
    finally:
        c2.close()


def test_autotune_keeps_results(dev, tmp_path):
    scenes = _tuning_scenes() + _batch_scenes(12, 40_000, seed=35)
    dsc = [(T(s.pts, dev), T(s.a, dev), T(s.b, dev)) for s in scenes]
    c2 = cellgraph.Context(0)
    try:
        chosen = c2.autotune(dsc, reps=1)
        buckets = {cellgraph.load_library().cg_tune_bucket(int(s.ell)) for s in scenes}
        assert set(chosen) == buckets
        path = str(tmp_path / "tune.json")
        c2.save_tuning(path, "test-gpu")
        c3 = cellgraph.Context(0)
        assert c3.load_tuning(path, "test-gpu")
        assert c3.tuning() == c2.tuning()
        c3.close()
        got = c2.build_batch(dsc)
        for sc, (c, e) in zip(scenes, got):
            want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
            assert np.array_equal(words_np(c, 64).reshape(want_c.shape), want_c)
            assert np.array_equal(edges_np(e), want_e)
        with cellgraph.Server(0, hbm_budget_bytes=4 << 30, max_inflight=4) as srv:
            srv.use_tuning(c2)
            ts = [srv.submit(s.pts, s.a, s.b) for s in scenes[:4]]
            for sc, t in zip(scenes, ts):
                srv.wait(t, 60.0)
                cells, edges = srv.fetch(t)
                want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
                assert np.array_equal(cells.reshape(want_c.shape), want_c)
                assert np.array_equal(edges, want_e)
    finally:
        c2.close()


# ---------------------------- asynchronous build ---------------------------

def test_build_dev_matches_and_captures(ctx, dev):
    sc = inputs.planes_3d(n=300_000, ell=64, seed=41)
    args = (T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev))
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    cells = torch.full((len(want_c) + 5, 1), -1, dtype=torch.int64, device=dev)
    edges = torch.full((len(want_e) + 5, 2), -1, dtype=torch.int32, device=dev)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    ctx.build_dev(*args, cells, edges, counts)
    torch.cuda.synchronize()
    u, e, st = counts.tolist()
    assert st == 0 and u == len(want_c) and e == len(want_e)
    assert np.array_equal(words_np(cells[:u], 64), want_c)
    assert np.array_equal(edges_np(edges[:e]), want_e)
    # captured by the caller into a CUDA graph and replayed
    cells.fill_(-1)
    edges.fill_(-1)
    counts.zero_()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ctx.build_dev(*args, cells, edges, counts)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert counts.tolist() == [u, e, 0]
    assert np.array_equal(words_np(cells[:u], 64), want_c)
    assert np.array_equal(edges_np(edges[:e]), want_e)


def test_build_dev_capacity_status(ctx, dev):
    sc = inputs.planes_3d(n=50_000, ell=40, seed=42)
    want_c, want_e = oracle.build(sc.pts, sc.a, sc.b, 64)
    cells = torch.full((30, 1), -7, dtype=torch.int64, device=dev)
    edges = torch.full((20, 2), -7, dtype=torch.int32, device=dev)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    # capacities 3 and 2: views of the first rows; nothing may land past them
    ctx.build_dev(T(sc.pts, dev), T(sc.a, dev), T(sc.b, dev), cells[:3], edges[:2], counts)
    torch.cuda.synchronize()
    assert counts.tolist() == [len(want_c), len(want_e), cellgraph.ERR_CAPACITY]
    assert (cells[3:] == -7).all() and (edges[2:] == -7).all()


def test_neighbors_rejects_unsorted_cells(dev):
    cells = np.array([[5], [3], [9]], dtype=np.uint64)
    with pytest.raises(cellgraph.CellGraphError) as ei:
        cellgraph.neighbors_h1(words_dev(cells, 64, dev), 8, 64)
    assert ei.value.status == cellgraph.ERR_INVALID_ARG
    dup = np.array([[1], [2], [2]], dtype=np.uint64)
    with pytest.raises(cellgraph.CellGraphError):
        cellgraph.neighbors_h1(words_dev(dup, 64, dev), 8, 64, strategy="sorted")
    wide = np.array([[0, 2], [5, 1]], dtype=np.uint64)  # row 1 < row 0 (top word)
    with pytest.raises(cellgraph.CellGraphError):
        cellgraph.neighbors_h1(words_dev(wide, 64, dev), 100, 64)


@pytest.mark.parametrize("ell", [100, 1024, 1030])
def test_neighbors_halves_checks_given_rows(dev, ell):
    """HALVES over 64-bit rows given in place checks their order in its key
    pass (2 to 16 words) or before it (more words): rows out of order within a
    warp's 32 rows or across two warps' rows, and a repeated row, are
    CG_ERR_INVALID_ARG; the sorted rows give the oracle's edges."""
    rng = np.random.default_rng(ell)
    w = (ell + 63) // 64
    rows = rng.integers(0, 2**63, size=(70, w), dtype=np.int64).astype(np.uint64)
    if ell % 64:
        rows[:, -1] &= np.uint64((1 << (ell % 64)) - 1)
    rows = np.unique(rows, axis=0)
    order = np.lexsort(rows.T)  # last word most significant
    rows = np.ascontiguousarray(rows[order])
    got = cellgraph.neighbors_h1(words_dev(rows, 64, dev), ell, 64, strategy="halves")
    assert np.array_equal(edges_np(got), oracle.neighbors(rows, ell, 64))
    bad = []
    for i, j in ((5, 6), (31, 32)):
        b = rows.copy()
        b[[i, j]] = b[[j, i]]
        bad.append(b)
    dup = rows.copy()
    dup[32] = dup[31]
    bad.append(dup)
    for b in bad:
        with pytest.raises(cellgraph.CellGraphError) as ei:
            cellgraph.neighbors_h1(words_dev(b, 64, dev), ell, 64, strategy="halves")
        assert ei.value.status == cellgraph.ERR_INVALID_ARG
