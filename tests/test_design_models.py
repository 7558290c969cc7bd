"""Host-side models of two device protocols, checked on the CPU.

These restate, in a few lines of Python, the argument a kernel relies on, and
check it against the oracle or a plain search, so that a change to the
argument fails here before it can reach a GPU:

* HALVES (two-part multi-index hashing): splitting the bits at s = l // 2,
  the pairs at distance 1 that differ below s are found inside runs of equal
  high part of the sorted cells, the others inside runs of equal low-part key
  of a stable sort, and each group checking its own case exactly finds every
  edge once -- even when the low-part key collides (here a deliberately weak
  key is used as well as the exact one).
* Box grid of the sign step: with the grid's box kept inside the int32 range,
  a point's slab (p - lo) >> s computed modulo 2^32 is below 2^bits exactly
  when lo <= p < lo + 2^(bits + s), so one unsigned subtraction and one
  compare place any int32 point, inside the grid or not; the box covers the
  sample's range it was placed on.
* Box grid classification: with fp32 arithmetic emulated exactly (rows
  scaled so the FMA chain's error bound is below 1, the threshold 2 + R with
  R >= s sum |a_k| h_k rounded upwards, the rounded cell centre), every cell
  the column walk proves "bit 1" has a . p >= b at every integer point of its
  box and every cell it proves "bit 0" has a . p < b there.
* BFS frontier counters: level d reads count[d % 3], appends to
  count[(d + 1) % 3] and clears count[(d + 2) % 3] even when its own frontier
  is empty; with the host looking only after every 16th level, no stale count
  is ever read.
"""
import collections
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import ints_to_rows


def _halves_edges(vals, ell, low_key):
    """The HALVES search over sorted distinct ints (model of the kernels)."""
    s = ell // 2
    lo_mask = (1 << s) - 1
    u = len(vals)
    found = []
    # group A: runs of equal high part, contiguous in value order
    for i in range(u):
        j = i + 1
        while j < u and (vals[j] >> s) == (vals[i] >> s):
            d = (vals[i] ^ vals[j]) & lo_mask
            if d and d & (d - 1) == 0:  # one differing bit, below s
                found.append((i, j))
            j += 1
    # group B: runs of equal low-part key after a stable sort of (key, cell)
    order = sorted(range(u), key=lambda i: low_key(vals[i] & lo_mask))
    for a in range(u):
        b = a + 1
        ka = low_key(vals[order[a]] & lo_mask)
        while b < u and low_key(vals[order[b]] & lo_mask) == ka:
            i, j = order[a], order[b]
            x = vals[i] ^ vals[j]
            if x & lo_mask == 0 and x and x & (x - 1) == 0:  # low parts equal, one bit above
                found.append((min(i, j), max(i, j)))
            b += 1
    return found


@pytest.mark.parametrize("ell", [1, 2, 7, 20, 64, 97])
@pytest.mark.parametrize("weak", [False, True])
def test_halves_model_finds_every_edge_once(ell, weak):
    rng = np.random.default_rng(ell * 2 + weak)
    vals = set()
    for _ in range(150):
        v = int(rng.integers(0, 2**62)) & ((1 << ell) - 1)
        vals.add(v)
        for _ in range(3):
            v ^= 1 << int(rng.integers(0, ell))
            vals.add(v)
    vals = sorted(vals)
    low_key = (lambda x: x % 3) if weak else (lambda x: x)  # weak: many collisions
    found = _halves_edges(vals, ell, low_key)
    assert len(found) == len(set(found))  # never twice
    want = oracle.neighbors(ints_to_rows(vals, ell, 64), ell, 64)
    assert sorted(found) == [tuple(e) for e in want.tolist()]


def _levels(adj, source):
    dist = {source: 0}
    q = collections.deque([source])
    sizes = collections.Counter({0: 1})
    while q:
        u = q.popleft()
        for v in adj[u]:
            if v not in dist:
                dist[v] = dist[u] + 1
                sizes[dist[v]] += 1
                q.append(v)
    return [sizes[d] for d in range(max(sizes) + 1)]


@pytest.mark.parametrize("seed", range(6))
def test_bfs_counter_rotation_model(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 300))
    adj = collections.defaultdict(list)
    for _ in range(int(rng.integers(0, 2 * n))):
        i, j = (int(x) for x in rng.integers(0, n, 2))
        if i != j:
            adj[i].append(j)
            adj[j].append(i)
    want = _levels(adj, 0)
    # the device protocol, levels enqueued in groups of 16
    count = [1, 0, 0]
    frontier, dist, seen = [0], {0: 0}, []
    d, group = 0, 16
    while True:
        for level in range(d, d + group):
            cnt = count[level % 3]
            count[(level + 2) % 3] = 0  # cleared even when this level is empty
            if cnt == 0:
                continue
            assert cnt == len(frontier)  # never a stale count
            seen.append(cnt)
            nxt = []
            for u in frontier:
                for v in adj[u]:
                    if v not in dist:
                        dist[v] = level + 1
                        nxt.append(v)
                        count[(level + 1) % 3] += 1
            frontier = nxt
        d += group
        if count[d % 3] == 0:  # the host's look after the group
            break
    assert seen == want


def _grid_axis(lo_s, hi_s, s, cnt):
    """The grid's placement on one axis: cnt slabs of 2^s integers around the
    sample range [lo_s, hi_s], kept inside the int32 range (model of the
    set-up kernel's last step)."""
    ext = hi_s - lo_s + 1
    span = cnt << s
    if span > 2**32:
        cnt = 2**32 >> s
        span = cnt << s
    lo = max(lo_s - (span - ext) // 2, -2**31)
    if lo + span > 2**31:
        lo = 2**31 - span
    return lo, cnt, span


@pytest.mark.parametrize("seed", range(8))
def test_grid_slab_test_model(seed):
    rng = np.random.default_rng(seed)
    I32 = (-2**31, 2**31 - 1)
    ranges = [(0, 0), I32, (I32[0], I32[0]), (I32[1], I32[1]), (-5, 5), (I32[1] - 3, I32[1]),
              (I32[0], I32[0] + 1000)]
    for _ in range(30):
        x, y = sorted(int(v) for v in rng.integers(I32[0], I32[1] + 1, 2, dtype=np.int64))
        ranges.append((x, y))
        c = int(rng.integers(-2**20, 2**20))
        ranges.append((c, c + int(rng.integers(0, 2**12))))
    for lo_s, hi_s in ranges:
        ext = hi_s - lo_s + 1
        want = min(ext + ext // 128 + 2, 2**32)
        for s in (0, 1, 5, 16, 30, 31):
            cnt0 = -(-want // (1 << s))  # slabs covering want
            for cnt in {cnt0, max(1, cnt0 // 3)}:
                if cnt > 2**20:
                    continue
                lo, cnt, span = _grid_axis(lo_s, hi_s, s, cnt)
                assert -2**31 <= lo and lo + span <= 2**31  # inside the int32 range
                if cnt == cnt0:
                    assert lo <= lo_s and hi_s < lo + span  # covers the sample
                probes = {lo - 1, lo, lo + span - 1, lo + span, lo_s, hi_s, *I32, 0}
                probes |= {int(v) for v in rng.integers(I32[0], I32[1] + 1, 48, dtype=np.int64)}
                for p in probes:
                    if not I32[0] <= p <= I32[1]:
                        continue
                    g = ((p - lo) % 2**32) >> s  # uint32 subtraction, then the shift
                    assert (g < cnt) == (lo <= p < lo + span)
                    if g < cnt:  # and the slab's integers hold p
                        assert lo + (g << s) <= p <= lo + ((g + 1) << s) - 1


# ---- fp32 emulated exactly on rationals (round to nearest even, round up) ----

def _rn32(x):
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    sign, x = (-1 if x < 0 else 1), abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1  # now 2^e <= x < 2^(e + 1)
    ulp = Fraction(2) ** (e - 23)
    q = x / ulp
    n = math.floor(q)
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * n * ulp


def _ru32(x):
    """Round towards +infinity (the inputs here are never negative)."""
    x = Fraction(x)
    assert x >= 0
    if x == 0:
        return Fraction(0)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    return math.ceil(x / ulp) * ulp


def _fma(a, b, c):
    return _rn32(a * b + c)


def _row(a, b, M, d):
    """The sign step's scaled row for a box with |p_k| <= M_k: (f, c, scale)."""
    T = Fraction(0)
    for k in range(d):
        T = _ru32(_ru32(abs(a[k])) * _ru32(M[k]) + T)
    T = _ru32(T + _ru32(abs(b)))
    if T == 0:
        return [Fraction(0)] * d, Fraction(4), Fraction(0)
    E = _ru32(T * Fraction(d + 4, 2 ** 24))
    e = E.numerator.bit_length() - E.denominator.bit_length()
    if Fraction(2) ** e > E:
        e -= 1
    e += 1  # E = m 2^e, 1/2 <= m < 1
    sc = Fraction(2) ** -e
    return [_rn32(a[k]) * sc for k in range(d)], -_rn32(b) * sc, sc


def _column_runs(cen0, s0, f0, c1, q):
    """Model of the set-up kernel's walk along one column: (one_lo, one_hi,
    cr_lo, cr_hi); every other cell is proven bit 0."""
    G0 = len(cen0)

    def test(g):
        v = _fma(f0, cen0[g], c1)
        return 1 if v >= q else (2 if v <= -q else 0)

    if f0 == 0:
        t = test(0)
        return (0, G0, 0, 0) if t == 1 else ((0, 0, 0, G0) if t == 0 else (0, 0, 0, 0))
    w0 = 2.0 ** s0  # the slab width (exact; the rounded centres may coincide)
    g_one = (float(q - c1) / float(f0) - float(cen0[0])) / w0
    g_zero = (float(-q - c1) / float(f0) - float(cen0[0])) / w0
    clamp = lambda g, lo, hi: int(min(max(g, lo), hi))
    if f0 > 0:
        a = clamp(math.ceil(g_one), 0, G0)
        while a < G0 and test(a) != 1:
            a += 1
        while 0 < a < G0 and test(a - 1) == 1:
            a -= 1
        z = clamp(math.floor(g_zero), -1, G0 - 1)
        while z >= 0 and test(z) != 2:
            z -= 1
        while 0 <= z < G0 - 1 and test(z + 1) == 2:
            z += 1
        return a, G0, z + 1, max(a, z + 1)
    a = clamp(math.floor(g_one), -1, G0 - 1)
    while a >= 0 and test(a) != 1:
        a -= 1
    while 0 <= a < G0 - 1 and test(a + 1) == 1:
        a += 1
    z = clamp(math.ceil(g_zero), 0, G0)
    while z < G0 and test(z) != 2:
        z += 1
    while 0 < z < G0 and test(z - 1) == 2:
        z -= 1
    return 0, a + 1, a + 1, max(z, a + 1)


@pytest.mark.parametrize("seed", range(6))
def test_grid_classification_model_is_sound(seed):
    rng = np.random.default_rng(100 + seed)
    d = 2 + seed % 2
    checked = 0
    for _case in range(4):
        s = [int(rng.integers(0, 21)) for _ in range(d)]
        cnt = [int(rng.integers(2, 25 if k == 0 else 5)) for k in range(d)]
        lo = []
        for k in range(d):
            span = cnt[k] << s[k]
            lo.append(int(rng.integers(-2**31, 2**31 - span + 1)))
        M = [max(abs(lo[k]), abs(lo[k] + (cnt[k] << s[k]) - 1)) for k in range(d)]
        hh = [Fraction(1, 2) * _ru32((1 << s[k]) - 1) for k in range(d)]

        def centre(k, g):
            return Fraction(1, 2) * _rn32(2 * (lo[k] + (g << s[k])) + (1 << s[k]) - 1)

        for _plane in range(12):
            kind = int(rng.integers(0, 3))
            if kind == 0:
                a = [int(x) for x in rng.integers(-3, 4, d)]
            elif kind == 1:
                a = [int(x) for x in rng.integers(-1024, 1025, d)]
            else:
                a = [int(x) for x in rng.integers(-2**31, 2**31, d, dtype=np.int64)]
            # through (or one unit off) a cell corner, or anywhere
            corner = [lo[k] + (int(rng.integers(0, cnt[k] + 1)) << s[k]) for k in range(d)]
            b = sum(a[k] * corner[k] for k in range(d)) + int(rng.integers(-2, 3))
            if int(rng.integers(0, 4)) == 0:
                b = int(rng.integers(-2**62, 2**62))
            f, c, sc = _row(a, b, M, d)
            R = Fraction(0)
            if sc != 0:
                for k in range(d):
                    R = _ru32(_ru32(abs(a[k])) * hh[k] + R)
                R = _ru32(R * sc)
            q = _ru32(2 + R)
            cen0 = [centre(0, g) for g in range(cnt[0])]
            for col in range(int(np.prod(cnt[1:]))):
                gk, rest = [0] * d, col
                for k in range(1, d):
                    gk[k], rest = rest % cnt[k], rest // cnt[k]
                c1 = c
                for k in range(1, d):
                    c1 = _fma(f[k], centre(k, gk[k]), c1)
                one_lo, one_hi, cr_lo, cr_hi = _column_runs(cen0, s[0], f[0], c1, q)
                for g0 in range(cnt[0]):
                    gk[0] = g0
                    box = [(lo[k] + (gk[k] << s[k]), lo[k] + ((gk[k] + 1) << s[k]) - 1)
                           for k in range(d)]
                    vmin = sum(min(a[k] * box[k][0], a[k] * box[k][1]) for k in range(d)) - b
                    vmax = sum(max(a[k] * box[k][0], a[k] * box[k][1]) for k in range(d)) - b
                    if one_lo <= g0 < one_hi:
                        assert vmin >= 0, (a, b, box)
                    elif not cr_lo <= g0 < cr_hi:
                        assert vmax < 0, (a, b, box)
                    checked += 1
    assert checked > 500
