"""Seeded synthetic inputs for the cell-graph hot path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no sign evaluation, no sorting, no neighbour search), so
both the CUDA path and the CPU oracle can take their inputs from it.

The paper's own inputs (a sample generator over SO(3) scenes, §2.1 and §5) are
not available; these workloads stand in for them with the shapes the paper
describes: n in the millions, l in the hundreds (§2.2), heavy duplication of
sample vectors (§2.2, multiset input).

Workloads (sizes are the defaults; every function takes smaller sizes for tests):

* ``lines_2d``      l=16 lines in the plane, N=20,000 integer points.
* ``planes_3d``     l=64 planes in 3-space, N=2**24 integer points.
* ``chains``        l=1024-bit vectors: 2**18 random seeds, each followed by a
                    chain of 15 single-bit-flip descendants, shuffled, then 25%
                    of the entries duplicated and shuffled again.
* ``scene_batch``   1,024 independent 3-D scenes, l log-uniform in [8, 256]
                    (rounded up to a multiple of 8) and N log-uniform in
                    [1e3, 1e6].
* ``poisson_arrivals`` exponential inter-arrival gaps for a request stream.
* ``spheres_3d``    l=64 spheres in 3-space (curved boundaries; bit i: outside
                    or on sphere i), N=2**24 integer points.
* ``quadrics_3d``   l general quadric surfaces with small integer monomial
                    coefficients, each passing through a random anchor point.

Layouts: points ``int32[N][d]`` row-major, constraint normals ``int32[l][d]``,
offsets ``int64[l]``; packed vectors ``uint64[N][ceil(l/64)]`` with bit i of a
vector in word i//64, bit i%64 (bits >= l are zero).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Scene:
    """One constraint arrangement plus its sampled points.

    Constraint i is satisfied by point p iff a[i] . p >= b[i] (§2.1).
    """

    pts: np.ndarray  # int32 [N, d]
    a: np.ndarray  # int32 [l, d]
    b: np.ndarray  # int64 [l]

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def d(self) -> int:
        return int(self.pts.shape[1])

    @property
    def ell(self) -> int:
        return int(self.a.shape[0])


def _uniform_int(rng: np.random.Generator, lo: int, hi: int, size, dtype) -> np.ndarray:
    """Uniform integers on the closed range [lo, hi]."""
    return rng.integers(lo, hi, size=size, dtype=dtype, endpoint=True)


def arrangement(seed, n: int, d: int, ell: int, coef: int, offset: int, coord: int) -> Scene:
    """Random integer arrangement: a ~ U{-coef..coef}^d, b ~ U{-offset..offset},
    points ~ U{-coord..coord}^d, all independent and seeded."""
    rng = np.random.default_rng(seed)
    a = _uniform_int(rng, -coef, coef, (ell, d), np.int32)
    b = _uniform_int(rng, -offset, offset, (ell,), np.int64)
    pts = _uniform_int(rng, -coord, coord, (n, d), np.int32)
    return Scene(pts=pts, a=a, b=b)


def lines_2d(n: int = 20_000, ell: int = 16, seed: int = 1) -> Scene:
    """l lines in the plane; a in [-1000,1000]^2, b in [-1e6,1e6], points on the
    integer grid [-1000,1000]^2. Each vector fits one 32-bit word."""
    return arrangement(seed, n, 2, ell, 1000, 1_000_000, 1000)


def planes_3d(n: int = 1 << 24, ell: int = 64, seed: int = 2) -> Scene:
    """l planes in 3-space; a in [-1024,1024]^3, b in [-2^30,2^30], points on the
    integer grid [-2^20,2^20]^3. With l=64 each vector fits one 64-bit word."""
    return arrangement(seed, n, 3, ell, 1024, 1 << 30, 1 << 20)


@dataclass
class Chains:
    keys: np.ndarray  # uint64 [N, W]: the shuffled multiset handed to the method
    base: np.ndarray  # uint64 [S*(L+1), W]: seeds and descendants in generation order
    planted: np.ndarray  # int64 [P, 2]: (parent, child) rows of ``base``
    ell: int


def chains(n_seeds: int = 1 << 18, chain_len: int = 15, ell: int = 1024,
           dup_frac: float = 0.25, seed: int = 3) -> Chains:
    """Bernoulli(1/2) seed vectors, each followed by a linear chain of
    ``chain_len`` descendants (child k+1 = child k with one uniformly random bit
    flipped). The base set is shuffled, a uniformly chosen ``dup_frac`` of its
    entries is appended again, and the result is shuffled once more.

    With the defaults N = 2^22 + 2^20 = 5,242,880 vectors of 16 words."""
    rng = np.random.default_rng(seed)
    w = (ell + 63) // 64
    cur = rng.integers(0, np.iinfo(np.uint64).max, size=(n_seeds, w), dtype=np.uint64,
                       endpoint=True)
    if ell % 64:
        cur[:, -1] &= np.uint64((1 << (ell % 64)) - 1)
    members = [cur.copy()]
    rows = np.arange(n_seeds)
    for _ in range(chain_len):
        k = rng.integers(0, ell, size=n_seeds)
        cur = cur.copy()
        cur[rows, k // 64] ^= np.left_shift(np.uint64(1), (k % 64).astype(np.uint64))
        members.append(cur)
    base = np.stack(members, axis=1).reshape(n_seeds * (chain_len + 1), w)
    step = np.arange(chain_len)
    parent = (np.arange(n_seeds)[:, None] * (chain_len + 1) + step[None, :]).reshape(-1)
    planted = np.stack([parent, parent + 1], axis=1).astype(np.int64)
    shuffled = base[rng.permutation(base.shape[0])]
    dup = rng.choice(shuffled.shape[0], size=int(round(dup_frac * shuffled.shape[0])),
                     replace=False)
    keys = np.concatenate([shuffled, shuffled[dup]], axis=0)
    keys = np.ascontiguousarray(keys[rng.permutation(keys.shape[0])])
    return Chains(keys=keys, base=base, planted=planted, ell=ell)


@dataclass
class BatchSpec:
    ell: np.ndarray  # int32 [S]
    n: np.ndarray  # int64 [S]
    seeds: list  # per-scene seed material


def scene_batch_spec(n_scenes: int = 1024, seed: int = 4, ell_lo: int = 8, ell_hi: int = 256,
                     n_lo: float = 1e3, n_hi: float = 1e6) -> BatchSpec:
    """Sizes of a batch of independent 3-D scenes: l = 8*ceil(exp(U(ln lo, ln hi))/8),
    N = round(exp(U(ln n_lo, ln n_hi))). Scene s is seeded from (seed, s)."""
    rng = np.random.default_rng(seed)
    ell = 8 * np.ceil(np.exp(rng.uniform(math.log(ell_lo), math.log(ell_hi), n_scenes)) / 8)
    n = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_scenes)))
    return BatchSpec(ell=ell.astype(np.int32), n=n.astype(np.int64),
                     seeds=[(seed, s) for s in range(n_scenes)])


def batch_scene(spec: BatchSpec, s: int) -> Scene:
    """Scene s of a batch, drawn like ``planes_3d`` with its own l and N."""
    return arrangement(list(spec.seeds[s]), int(spec.n[s]), 3, int(spec.ell[s]),
                       1024, 1 << 30, 1 << 20)


def poisson_arrivals(n_requests: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream: exponential gaps with
    mean 1/rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))



@dataclass
class QuadricScene:
    """Points plus l quadric constraints: constraint i is satisfied by p iff
    sum_{j<=k} q[i, jk] p_j p_k + a[i] . p >= b[i] (§2.1 with curved
    boundaries). ``q`` holds the coefficient of the monomial p_j p_k for
    j <= k, in the order (0,0), (0,1), ..., (0,d-1), (1,1), ..., (d-1,d-1)."""

    pts: np.ndarray  # int32 [N, d]
    q: np.ndarray  # int32 [l, d(d+1)/2]
    a: np.ndarray  # int32 [l, d]
    b: np.ndarray  # int64 [l]

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def ell(self) -> int:
        return int(self.a.shape[0])


def _diagonal_monomials(d: int) -> list:
    """Positions of p_j^2 in the monomial order of QuadricScene.q."""
    pos, t = [], 0
    for j in range(d):
        pos.append(t)
        t += d - j
    return pos


def spheres_3d(n: int = 1 << 24, ell: int = 64, seed: int = 13, d: int = 3) -> QuadricScene:
    """l spheres: centres ~ U{-2^20..2^20}^d, radii ~ U{2^19..2^21}; bit i is 1
    when the point lies on or outside sphere i, i.e. |p - c_i|^2 >= r_i^2,
    written as the quadric |p|^2 - 2 c_i . p >= r_i^2 - |c_i|^2. Points ~
    U{-2^20..2^20}^d."""
    rng = np.random.default_rng(seed)
    c = _uniform_int(rng, -(1 << 20), 1 << 20, (ell, d), np.int64)
    r = _uniform_int(rng, 1 << 19, 1 << 21, (ell,), np.int64)
    q = np.zeros((ell, d * (d + 1) // 2), np.int32)
    q[:, _diagonal_monomials(d)] = 1
    a = (-2 * c).astype(np.int32)
    b = (r * r - (c * c).sum(axis=1)).astype(np.int64)
    pts = _uniform_int(rng, -(1 << 20), 1 << 20, (n, d), np.int32)
    return QuadricScene(pts=pts, q=q, a=a, b=b)


def quadrics_3d(n: int = 1 << 20, ell: int = 64, seed: int = 14, d: int = 3,
                qcoef: int = 16, coord: int = 1 << 20) -> QuadricScene:
    """l general quadrics (ellipsoids, hyperboloids, paraboloids, saddles):
    monomial coefficients ~ U{-qcoef..qcoef}, a ~ U{-2^20..2^20}^d, and b
    chosen so that surface i passes through an anchor point z_i ~
    U{-coord..coord}^d (b_i = q_i(z_i) + a_i . z_i). Points ~ U{-coord..coord}^d."""
    rng = np.random.default_rng(seed)
    m = d * (d + 1) // 2
    q = _uniform_int(rng, -qcoef, qcoef, (ell, m), np.int32)
    a = _uniform_int(rng, -(1 << 20), 1 << 20, (ell, d), np.int32)
    z = _uniform_int(rng, -coord, coord, (ell, d), np.int64)
    mono = np.stack([z[:, j] * z[:, k] for j in range(d) for k in range(j, d)], axis=1)
    b = ((q.astype(np.int64) * mono).sum(axis=1) + (a.astype(np.int64) * z).sum(axis=1))
    pts = _uniform_int(rng, -coord, coord, (n, d), np.int32)
    return QuadricScene(pts=pts, q=q, a=a, b=b.astype(np.int64))
