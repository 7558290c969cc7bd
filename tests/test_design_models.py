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
* BFS frontier counters: level d reads count[d % 3], appends to
  count[(d + 1) % 3] and clears count[(d + 2) % 3] even when its own frontier
  is empty; with the host looking only after every 16th level, no stale count
  is ever read.
"""
import collections

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
