"""Pins for the CPU oracle: each test ties it to something other than itself.

* Figure 1 of the paper (§2.1): the three-line scene and its four printed
  vectors; the dense sampling of the same scene (7 cells, the cube Q3 minus
  vertex 000, 9 edges; the paper notes vector 000 has no point).
* Figure 2 of the paper (§3.2): the six printed vectors and their two
  Hamming-1 pairs.
* Exact sign evaluation against Python's arbitrary-precision integers, at the
  int32 / int64 extremes and on exact ties (a . p = b).
* Sort + unique against Python's ``sorted(set(...))`` (§3.2 reduces to it).
* Neighbours against brute force over all pairs (the naive algorithm of §3.1,
  i.e. the heuristic with h = 0), for l across word boundaries.
* Closed forms: the full hypercube Q_l has l * 2^(l-1) edges.
* Invariants: distance exactly 1, i < j, no repeats, degree <= l,
  |E| <= U l / 2 (§2.2); output unchanged by shuffling or duplicating X (§3.2,
  multiset robustness); the arrangement bound sum_{k<=d} C(l,k) on U.
* Planted chains: surviving planted Hamming-1 pairs are edges; every edge lies
  within one chain.
* The heuristic of §3.1 (Algorithms 1-2): against brute force for every pivot
  count (h = 0 is the naive method and must compare every pair), on Figure 2's
  vectors, on the hypercube's closed form, for any segment count w; and the
  pivot test as printed ("> 1") finds no edge at all, which is why the oracle
  reads it as inverted.
* Quadric constraints (curved boundaries, §2.1): with a zero quadratic form
  they equal the half-space oracle; nested concentric spheres give the closed
  form (l + 1 thermometer cells on a path of l edges, ties satisfied); spheres
  written as monomials agree with the distance form in Python integers near
  the int32 limits; renaming coordinates leaves every vector unchanged.
* BFS on G_X (§6): distances on the hypercube are Hamming distances (closed
  form), on Figure 1's dense arrangement (Q3 minus 000) too, on a path graph
  |i - s|, and on random small graphs they equal Floyd-Warshall's.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import inputs
from tests.helpers import (as_u64_rows, brute_force_edges, ints_to_rows, paper_string_to_int,
                           popcount64, rows_to_ints)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig1():
    cons, pts = [], []
    with open(os.path.join(GOLDEN, "fig1_three_lines.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "constraint":
                cons.append([int(x) for x in t[1:]])
            elif t[0] == "point":
                pts.append((t[1], int(t[2]), int(t[3]), t[4]))
    a = np.array([c[:2] for c in cons], dtype=np.int32)
    b = np.array([c[2] for c in cons], dtype=np.int64)
    return a, b, pts


def _read_fig2():
    vecs = []
    with open(os.path.join(GOLDEN, "fig2_six_vectors.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            vecs.append((t[0], t[1]))
    return vecs


@pytest.mark.parametrize("word_bits", [32, 64])
def test_fig1_printed_vectors(word_bits):
    a, b, pts = _read_fig1()
    P = np.array([[x, y] for _, x, y, _ in pts], dtype=np.int32)
    keys = oracle.pack_signs(P, a, b, word_bits)
    got = rows_to_ints(keys, word_bits)
    want = [paper_string_to_int(v) for *_, v in pts]
    assert got == want


@pytest.mark.parametrize("word_bits", [32, 64])
def test_fig1_cells_and_edges(word_bits):
    a, b, pts = _read_fig1()
    P = np.array([[x, y] for _, x, y, _ in pts], dtype=np.int32)
    cells, edges = oracle.build(P, a, b, word_bits)
    names = {paper_string_to_int(v): n for n, _, _, v in pts}
    # value order: C (100 -> 1) < B (110 -> 3) < D (101 -> 5) < A (111 -> 7)
    assert [names[v] for v in rows_to_ints(cells, word_bits)] == ["C", "B", "D", "A"]
    # the 4-cycle C-B-A-D-C; A-C and B-D are at distance 2
    assert edges.tolist() == [[0, 1], [0, 2], [1, 3], [2, 3]]


def test_fig1_dense_sampling_gives_cube_minus_000():
    a, b, _ = _read_fig1()
    g = np.arange(-40, 61, dtype=np.int32)
    P = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    cells, edges = oracle.build(P, a, b, 64)
    vals = rows_to_ints(cells, 64)
    assert vals == [1, 2, 3, 4, 5, 6, 7]  # every pattern but 000 (§2.1)
    assert len(edges) == 9  # Q3 has 12 edges, vertex 000 takes 3


def test_fig2_pairs():
    vecs = _read_fig2()
    vals = sorted(paper_string_to_int(v) for v, _ in vecs)
    cells = ints_to_rows(vals, 6, 64)
    edges = oracle.neighbors(cells, 6, 64)
    named = [(vals[i], vals[j]) for i, j in edges.tolist()]
    p = paper_string_to_int
    assert named == [(p("110100"), p("110110")), (p("110110"), p("110111"))]


def _read_fig2_tree():
    out = {}
    with open(os.path.join(GOLDEN, "fig2_tree_levels.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            out[t[0]] = [int(x) for x in t[1:]]
    return out


def test_fig2_digit_recoding():
    """Figure 2 lists every vector's base-4 recoding (r = 2)."""
    vecs = _read_fig2()
    cells = ints_to_rows([paper_string_to_int(v) for v, _ in vecs], 6, 64)
    got = oracle.tree_digits(cells, 6, 64, r=2, order=0)
    assert ["".join(str(d) for d in row) for row in got.tolist()] == [t for _, t in vecs]


def test_fig2_tree_levels_and_edges():
    """Figure 2's tree has 3, 4 and 6 nodes below the root; its search finds
    the two Hamming-1 pairs of the example."""
    vecs = _read_fig2()
    want = _read_fig2_tree()
    vals = sorted(paper_string_to_int(v) for v, _ in vecs)
    cells = ints_to_rows(vals, 6, 64)
    counts, edges = oracle.tree(cells, 6, 64, r=want["r"][0], order=0)
    assert counts.tolist() == want["levels"]
    assert edges.tolist() == oracle.neighbors(cells, 6, 64).tolist()
    p = paper_string_to_int
    assert [(vals[i], vals[j]) for i, j in edges.tolist()] == [
        (p("110100"), p("110110")), (p("110110"), p("110111"))]


def _prefix_counts(vals, ell, r, order):
    """Distinct prefixes of h digits, h = 0..L, from integer arithmetic: the
    paper's order reads bits from x(0) up, so a prefix is the value modulo
    2^(h r); the value order reads from bit l - 1 down, so it is the value
    shifted right by l - h r."""
    L = (ell + r - 1) // r
    out = []
    for h in range(L + 1):
        nb = min(h * r, ell)
        if order == 0:
            out.append(len({v & ((1 << nb) - 1) for v in vals}))
        else:
            out.append(len({v >> (ell - nb) for v in vals}))
    return out


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("r", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("ell", [1, 7, 16, 64, 65, 130])
def test_tree_levels_and_search_against_lookup(ell, r, order):
    rng = np.random.default_rng(ell * 100 + r * 10 + order)
    n = 300
    vals = set()
    # clustered vectors, so that the tree has long shared prefixes and many
    # Hamming-1 pairs
    base = [int(rng.integers(0, 2**63)) | (int(rng.integers(0, 2**63)) << 63) for _ in range(6)]
    for _ in range(n):
        v = base[int(rng.integers(0, 6))]
        for _ in range(int(rng.integers(0, 4))):
            v ^= 1 << int(rng.integers(0, ell))
        vals.add(v & ((1 << ell) - 1))
    vals = sorted(vals)
    cells = ints_to_rows(vals, ell, 64)
    counts, edges = oracle.tree(cells, ell, 64, r=r, order=order)
    assert counts.tolist() == _prefix_counts(vals, ell, r, order)
    assert counts[-1] == len(vals) and counts[0] == 1
    assert np.array_equal(edges, oracle.neighbors(cells, ell, 64))
    assert len(edges) > 0 or ell == 1


@pytest.mark.parametrize("ell,r", [(6, 2), (8, 3), (9, 8)])
def test_tree_hypercube_levels(ell, r):
    """All 2^l vectors: every prefix occurs, 2^(min(h r, l)) nodes on level h,
    and the search finds the l 2^(l-1) cube edges."""
    cells = np.arange(1 << ell, dtype=np.uint64).reshape(-1, 1)
    counts, edges = oracle.tree(cells, ell, 64, r=r, order=0)
    L = (ell + r - 1) // r
    assert counts.tolist() == [1 << min(h * r, ell) for h in range(L + 1)]
    assert len(edges) == ell * (1 << (ell - 1))


def _python_signs(pts, a, b):
    out = []
    for p in pts.tolist():
        v = 0
        for i, (ai, bi) in enumerate(zip(a.tolist(), b.tolist())):
            if sum(x * y for x, y in zip(ai, p)) >= bi:
                v |= 1 << i
        out.append(v)
    return out


@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("ell,d", [(1, 1), (7, 2), (32, 3), (33, 4), (64, 3), (65, 2), (130, 3)])
def test_pack_matches_bigint(ell, d, word_bits):
    rng = np.random.default_rng(ell * 10 + d)
    n = 60
    i32 = np.iinfo(np.int32)
    i64 = np.iinfo(np.int64)
    pts = rng.integers(-50, 51, size=(n, d)).astype(np.int32)
    pts[:5] = i32.max
    pts[5:10] = i32.min
    a = rng.integers(-50, 51, size=(ell, d)).astype(np.int32)
    a[0] = i32.min
    b = rng.integers(-3000, 3001, size=ell).astype(np.int64)
    b[-1] = i64.min if ell > 1 else b[-1]
    if ell > 2:
        b[1] = i64.max
    keys = oracle.pack_signs(pts, a, b, word_bits)
    assert rows_to_ints(keys, word_bits) == _python_signs(pts, a, b)


def test_ties_count_as_satisfied():
    # a . p == b exactly: the constraint a . p >= b holds, so the bit is 1
    # and one unit below the offset it fails, so the bit is 0
    a = np.array([[3, -7], [0, 0], [-2, 4]], dtype=np.int32)
    pts = np.array([[7, 3], [0, 0], [5, 2], [7, 2]], dtype=np.int32)
    b = np.array([0, 0, -2], dtype=np.int64)
    keys = oracle.pack_signs(pts, a, b, 64)
    # (7,3): 0>=0, 0>=0, -2>=-2 | (0,0): ties everywhere | (5,2): 1, 0, -2>=-2
    # (7,2): 7>=0, 0>=0, -6<-2
    assert rows_to_ints(keys, 64) == [0b111, 0b111, 0b111, 0b011]


@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("ell", [1, 3, 31, 32, 33, 64, 65, 130])
def test_dedup_is_sorted_set(ell, word_bits):
    rng = np.random.default_rng(ell)
    pool = [int(rng.integers(0, 1 << min(ell, 62))) << max(0, ell - 62) for _ in range(37)]
    pool = [v & ((1 << ell) - 1) for v in pool]
    vals = [pool[int(i)] for i in rng.integers(0, len(pool), size=500)]
    keys = ints_to_rows(vals, ell, word_bits)
    cells, pc = oracle.dedup(keys, ell, word_bits, point_cell=True)
    want = sorted(set(vals))
    assert rows_to_ints(cells, word_bits) == want
    assert [want[i] for i in pc.tolist()] == vals


def _clustered(rng, n, ell, n_seeds, flips):
    seeds = [int.from_bytes(rng.bytes((ell + 7) // 8), "little") & ((1 << ell) - 1)
             for _ in range(n_seeds)]
    vals = []
    for _ in range(n):
        v = seeds[int(rng.integers(0, n_seeds))]
        for _ in range(int(rng.integers(0, flips + 1))):
            v ^= 1 << int(rng.integers(0, ell))
        vals.append(v)
    return vals


@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("ell", [1, 2, 5, 31, 32, 33, 63, 64, 65, 70, 130])
def test_neighbors_match_brute_force(ell, word_bits):
    rng = np.random.default_rng(1000 + ell)
    vals = sorted(set(_clustered(rng, 700, ell, 12, 3)))
    cells = ints_to_rows(vals, ell, word_bits)
    got = oracle.neighbors(cells, ell, word_bits)
    want = brute_force_edges(as_u64_rows(cells, ell, word_bits))
    assert got.tolist() == want.tolist()
    assert len(got) > 0


@pytest.mark.parametrize("ell", range(1, 11))
def test_hypercube_closed_form(ell):
    cells = ints_to_rows(list(range(1 << ell)), ell, 64)
    edges = oracle.neighbors(cells, ell, 64)
    assert len(edges) == ell * (1 << (ell - 1))
    deg = np.bincount(edges.reshape(-1), minlength=1 << ell)
    assert (deg == ell).all()


def _check_invariants(cells_u64, edges, ell):
    u = cells_u64.shape[0]
    e = edges.astype(np.int64)
    if len(e):
        assert (e[:, 0] < e[:, 1]).all()
        assert e.max() < u
        x = cells_u64[e[:, 0]] ^ cells_u64[e[:, 1]]
        assert (popcount64(x).sum(axis=1) == 1).all()
        assert len({tuple(r) for r in e.tolist()}) == len(e)
        order = np.lexsort((e[:, 1], e[:, 0]))
        assert (order == np.arange(len(e))).all()
        assert np.bincount(e.reshape(-1), minlength=u).max() <= ell
    assert len(e) <= u * ell / 2


@pytest.mark.parametrize("word_bits", [32, 64])
def test_multiset_and_shuffle_invariance(word_bits):
    sc = inputs.planes_3d(n=3000, ell=40, seed=11)
    keys = oracle.pack_signs(sc.pts, sc.a, sc.b, word_bits)
    cells = oracle.dedup(keys, 40, word_bits)
    edges = oracle.neighbors(cells, 40, word_bits)
    rng = np.random.default_rng(5)
    mixed = np.concatenate([keys, keys[rng.integers(0, len(keys), 4000)]])
    mixed = mixed[rng.permutation(len(mixed))]
    cells2 = oracle.dedup(mixed, 40, word_bits)
    edges2 = oracle.neighbors(cells2, 40, word_bits)
    assert np.array_equal(cells, cells2) and np.array_equal(edges, edges2)
    _check_invariants(as_u64_rows(cells, 40, word_bits), edges, 40)


def test_arrangement_bounds_lines_and_planes():
    for sc, word_bits in [(inputs.lines_2d(n=20_000), 32), (inputs.planes_3d(n=200_000), 64)]:
        cells, edges = oracle.build(sc.pts, sc.a, sc.b, word_bits)
        bound = sum(math.comb(sc.ell, k) for k in range(sc.d + 1))
        assert 1 < len(cells) <= bound
        _check_invariants(as_u64_rows(cells, sc.ell, word_bits), edges, sc.ell)
        assert len(edges) > len(cells) // 2  # a sampled arrangement is well connected


def test_rows_subset_matches_full():
    sc = inputs.planes_3d(n=5000, ell=64, seed=3)
    cells, edges = oracle.build(sc.pts, sc.a, sc.b, 64)
    rows = np.array([0, 5, 17, len(cells) - 1], dtype=np.int64)
    sub = oracle.neighbors(cells, 64, 64, rows=rows)
    want = edges[np.isin(edges[:, 0], rows)]
    assert sub.tolist() == want.tolist()


def test_planted_chains():
    ch = inputs.chains(n_seeds=300, chain_len=15, ell=130, seed=9)
    cells = oracle.dedup(ch.keys, ch.ell, 64)
    edges = oracle.neighbors(cells, ch.ell, 64)
    vals = rows_to_ints(cells, 64)
    index = {v: i for i, v in enumerate(vals)}
    base_vals = rows_to_ints(ch.base, 64)
    eset = {tuple(e) for e in edges.tolist()}
    planted_kept = 0
    for p, c in ch.planted.tolist():
        x, y = base_vals[p], base_vals[c]
        if x == y:
            continue
        i, j = sorted((index[x], index[y]))
        assert (i, j) in eset
        planted_kept += 1
    assert planted_kept > 0.95 * len(ch.planted)
    chain_of = {}
    for r, v in enumerate(base_vals):
        chain_of.setdefault(v, set()).add(r // 16)
    for i, j in edges.tolist():
        assert chain_of[vals[i]] & chain_of[vals[j]]
    assert len(vals) == len(set(base_vals))


# ------------------------- heuristic (§3.1, Algorithms 1-2) ------------------

@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("ell", [1, 5, 33, 64, 70, 130])
@pytest.mark.parametrize("h", [0, 1, 3, 5])
def test_heuristic_matches_brute_force(ell, word_bits, h):
    rng = np.random.default_rng(2000 + ell + h)
    vals = sorted(set(_clustered(rng, 300, ell, 8, 3)))
    cells = ints_to_rows(vals, ell, word_bits)
    got, tested = oracle.heuristic(cells, ell, word_bits, h=h)
    want = brute_force_edges(as_u64_rows(cells, ell, word_bits))
    assert got.tolist() == want.tolist()
    u = len(vals)
    if h == 0:
        assert tested == u * (u - 1) // 2  # no pivots: every pair is compared
    else:
        assert len(want) <= tested <= u * (u - 1) // 2


def test_heuristic_pruning_only_shrinks_with_more_pivots():
    rng = np.random.default_rng(77)
    vals = sorted(set(_clustered(rng, 500, 96, 20, 4)))
    cells = ints_to_rows(vals, 96, 64)
    counts = [oracle.heuristic(cells, 96, 64, h=h)[1] for h in range(0, 7)]
    # the pivots for h + 1 include those for h, and the test is a conjunction
    assert all(a >= b for a, b in zip(counts, counts[1:])), counts
    assert counts[-1] < counts[0] // 4, counts  # and it does prune


@pytest.mark.parametrize("w", [1, 2, 7, 32, 64, 200])
def test_heuristic_any_segment_count(w):
    rng = np.random.default_rng(5)
    ell = 70  # not a multiple of most w: the last segment is shorter
    vals = sorted(set(_clustered(rng, 300, ell, 6, 2)))
    cells = ints_to_rows(vals, ell, 64)
    got, _ = oracle.heuristic(cells, ell, 64, h=2, w=w)
    assert got.tolist() == brute_force_edges(as_u64_rows(cells, ell, 64)).tolist()


@pytest.mark.parametrize("h", [0, 1, 2, 3])
def test_heuristic_fig2_pairs(h):
    vecs = _read_fig2()
    vals = sorted(paper_string_to_int(v) for v, _ in vecs)
    got, _ = oracle.heuristic(ints_to_rows(vals, 6, 64), 6, 64, h=h)
    p = paper_string_to_int
    assert [(vals[i], vals[j]) for i, j in got.tolist()] == [(p("110100"), p("110110")),
                                                             (p("110110"), p("110111"))]


@pytest.mark.parametrize("h", [1, 2, 4])
def test_heuristic_hypercube_closed_form(h):
    ell = 8
    got, _ = oracle.heuristic(ints_to_rows(list(range(1 << ell)), ell, 64), ell, 64, h=h)
    assert len(got) == ell * (1 << (ell - 1))


def test_heuristic_test_as_printed_finds_nothing():
    """Every true edge has |dist(x_i, x_p) - dist(x_j, x_p)| = 1 for every
    pivot, so Algorithm 2's test as printed ("> 1 for all d") rejects all of
    them; with h = 0 the test is vacuous and both forms are the naive method."""
    rng = np.random.default_rng(9)
    vals = sorted(set(_clustered(rng, 300, 40, 6, 3)))
    cells = ints_to_rows(vals, 40, 64)
    want = brute_force_edges(as_u64_rows(cells, 40, 64))
    assert len(want) > 0
    for h in (1, 3):
        got, _ = oracle.heuristic(cells, 40, 64, h=h, as_printed=True)
        assert len(got) == 0
    got, _ = oracle.heuristic(cells, 40, 64, h=0, as_printed=True)
    assert got.tolist() == want.tolist()


# ------------------------------ BFS on G_X (§6) -------------------------------

@pytest.mark.parametrize("ell,source", [(1, 0), (4, 5), (9, 0), (9, 300)])
def test_bfs_hypercube_distances_are_hamming(ell, source):
    cells = ints_to_rows(list(range(1 << ell)), ell, 64)
    edges = oracle.neighbors(cells, ell, 64)
    dist = oracle.bfs(edges, 1 << ell, source)
    assert dist.tolist() == [bin(v ^ source).count("1") for v in range(1 << ell)]


def test_bfs_fig1_dense_arrangement():
    # Q3 without 000 (§2.1, Figure 1): every remaining pair is still joined by
    # a path of Hamming length avoiding 000
    vals = list(range(1, 8))
    cells = ints_to_rows(vals, 3, 64)
    edges = oracle.neighbors(cells, 3, 64)
    for s in range(7):
        dist = oracle.bfs(edges, 7, s)
        assert dist.tolist() == [bin(vals[s] ^ v).count("1") for v in vals]


def test_bfs_path_and_unreachable():
    n = 50
    edges = np.array([[i, i + 1] for i in range(n - 1) if i != 30], np.uint32)
    dist = oracle.bfs(edges, n, 10)
    assert dist.tolist() == [abs(i - 10) if i <= 30 else -1 for i in range(n)]


@pytest.mark.parametrize("seed", range(5))
def test_bfs_against_floyd_warshall(seed):
    rng = np.random.default_rng(seed)
    n = 40
    pairs = {tuple(sorted(map(int, rng.choice(n, 2, replace=False)))) for _ in range(45)}
    edges = np.array(sorted(pairs), np.uint32)
    inf = 10**9
    d = np.full((n, n), inf, np.int64)
    np.fill_diagonal(d, 0)
    for i, j in pairs:
        d[i, j] = d[j, i] = 1
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    for s in (0, 7, 39):
        want = [int(x) if x < inf else -1 for x in d[s]]
        assert oracle.bfs(edges, n, s).tolist() == want


# --------------------- quadric constraints (curved boundaries) ---------------------

def _monomials(d):
    return [(j, k) for j in range(d) for k in range(j, d)]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("ell,word_bits", [(7, 32), (40, 64), (130, 64), (33, 32)])
def test_quadric_with_zero_form_is_the_linear_oracle(d, ell, word_bits):
    # q = 0 reduces the quadric test to the half-space test, a separate function.
    sc = inputs.arrangement(70 + d, 3000, d, ell, 1 << 20, 1 << 40, (1 << 31) - 1)
    q = np.zeros((ell, d * (d + 1) // 2), np.int32)
    got = oracle.pack_signs_quadric(sc.pts, q, sc.a, sc.b, word_bits)
    assert np.array_equal(got, oracle.pack_signs(sc.pts, sc.a, sc.b, word_bits))


def _sphere_quadric(c, r):
    d = c.shape[1]
    q = np.zeros((c.shape[0], d * (d + 1) // 2), np.int32)
    for t, (j, k) in enumerate(_monomials(d)):
        if j == k:
            q[:, t] = 1
    a = (-2 * c).astype(np.int32)
    b = np.array([int(rr) ** 2 - sum(int(x) ** 2 for x in cc) for cc, rr in zip(c, r)],
                 dtype=np.int64)
    return q, a, b


def test_quadric_nested_spheres_closed_form():
    # Concentric spheres of radii r_0 < ... < r_{l-1}: a point at distance rho
    # from the centre has bit i = [rho >= r_i], so the cells are the l + 1
    # "thermometer" vectors 0, 1, 11, ..., 1...1, and consecutive ones differ in
    # one bit: the cell graph is a path with l edges. Points are placed between
    # consecutive radii and exactly on them (a tie counts as satisfied).
    ell, d = 50, 3
    centre = np.array([[123456, -654321, 99999]], np.int64)
    radii = np.cumsum(np.arange(1, ell + 1) * 1000).astype(np.int64)
    q, a, b = _sphere_quadric(np.repeat(centre, ell, axis=0), radii)
    rho = np.concatenate([[0], radii - 1, radii, radii + 7])
    pts = []
    for i, r in enumerate(rho):
        axis = i % d
        p = centre[0].copy()
        p[axis] += r if i % 2 else -r
        pts.append(p)
    pts = np.array(pts, np.int32)
    keys = oracle.pack_signs_quadric(pts, q, a, b, 64)
    cells = oracle.dedup(keys, ell, 64)
    edges = oracle.neighbors(cells, ell, 64)
    want = [(1 << i) - 1 for i in range(ell + 1)]
    assert rows_to_ints(cells, 64) == want
    assert edges.tolist() == [[i, i + 1] for i in range(ell)]
    # each point's vector counts the radii it reaches
    for p, k in zip(rho, rows_to_ints(keys, 64)):
        assert k == (1 << int((radii <= p).sum())) - 1


def test_quadric_spheres_match_distance_form_at_extremes():
    # Spheres written as monomials (|p|^2 - 2 c.p >= r^2 - |c|^2) against the
    # distance form sum_k (p_k - c_k)^2 >= r^2 in Python integers, with
    # coordinates near the int32 limits (products near 2^62).
    rng = np.random.default_rng(75)
    ell, d = 70, 3
    c = rng.integers(-(1 << 30) + 1, 1 << 30, size=(ell, d), dtype=np.int64)
    r = rng.integers(0, 1 << 31, size=ell, dtype=np.int64)
    q, a, b = _sphere_quadric(c, r)
    lim = (1 << 31) - 1
    pts = rng.integers(-lim, lim, size=(400, d), dtype=np.int64, endpoint=True)
    pts[:8] = [[lim, lim, lim], [-lim - 1, -lim - 1, -lim - 1], [0, 0, 0], [lim, -lim - 1, 0],
               c[0], c[1] + [int(r[1]), 0, 0], c[2] + [0, int(r[2]) - 1, 0], c[3]]
    pts = pts.astype(np.int32)
    keys = oracle.pack_signs_quadric(pts, q, a, b, 64)
    got = rows_to_ints(keys, 64)
    for p, k in zip(pts.tolist(), got):
        want = 0
        for i in range(ell):
            dist2 = sum((int(p[t]) - int(c[i][t])) ** 2 for t in range(d))
            if dist2 >= int(r[i]) ** 2:
                want |= 1 << i
        assert k == want


@pytest.mark.parametrize("d", [2, 3, 4])
def test_quadric_invariant_under_coordinate_permutation(d):
    # Renaming the coordinates (points, linear terms and the monomial indices
    # together) describes the same sets: a mixed-up monomial index fails this.
    sc = inputs.quadrics_3d(n=2000, ell=45, seed=80 + d, d=d, coord=1 << 16)
    perm = np.random.default_rng(d).permutation(d)
    mono = _monomials(d)
    where = {jk: t for t, jk in enumerate(mono)}
    q2 = np.zeros_like(sc.q)
    for t, (j, k) in enumerate(mono):
        pj, pk = sorted((int(np.flatnonzero(perm == j)[0]), int(np.flatnonzero(perm == k)[0])))
        q2[:, where[(pj, pk)]] = sc.q[:, t]
    # new coordinate i is old coordinate perm[i]
    a2 = sc.a[:, perm]
    pts2 = sc.pts[:, perm]
    k1 = oracle.pack_signs_quadric(sc.pts, sc.q, sc.a, sc.b, 64)
    k2 = oracle.pack_signs_quadric(pts2, q2, a2, sc.b, 64)
    assert np.array_equal(k1, k2)
    assert len(set(rows_to_ints(k1, 64))) > 20
