"""Test-side helpers written independently of both the oracle and the CUDA
library: packed rows <-> Python integers, brute-force Hamming-1 pairs."""
from __future__ import annotations

import numpy as np


def row_to_int(row, word_bits: int) -> int:
    v = 0
    for j, w in enumerate(np.asarray(row).tolist()):
        v |= int(w) << (word_bits * j)
    return v


def rows_to_ints(keys, word_bits: int) -> list:
    return [row_to_int(r, word_bits) for r in np.asarray(keys)]


def int_to_row(v: int, ell: int, word_bits: int) -> np.ndarray:
    w = (ell + word_bits - 1) // word_bits
    dt = np.uint64 if word_bits == 64 else np.uint32
    mask = (1 << word_bits) - 1
    return np.array([(v >> (word_bits * j)) & mask for j in range(w)], dtype=dt)


def ints_to_rows(vals, ell: int, word_bits: int) -> np.ndarray:
    w = (ell + word_bits - 1) // word_bits
    dt = np.uint64 if word_bits == 64 else np.uint32
    if len(vals) == 0:
        return np.zeros((0, w), dtype=dt)
    return np.stack([int_to_row(v, ell, word_bits) for v in vals])


def paper_string_to_int(s: str) -> int:
    """The paper writes a vector as x(0) x(1) ... from left to right."""
    return sum(1 << i for i, ch in enumerate(s) if ch == "1")


def popcount64(x: np.ndarray) -> np.ndarray:
    """SWAR popcount of uint64 values (Hacker's Delight, section 5-1)."""
    x = x.astype(np.uint64)
    x = x - ((x >> np.uint64(1)) & np.uint64(0x5555555555555555))
    x = (x & np.uint64(0x3333333333333333)) + ((x >> np.uint64(2)) & np.uint64(0x3333333333333333))
    x = (x + (x >> np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    return ((x * np.uint64(0x0101010101010101)) >> np.uint64(56)).astype(np.int64)


def brute_force_edges(cells_u64: np.ndarray) -> np.ndarray:
    """All pairs (i, j), i < j, with Hamming distance exactly 1, compared
    word by word; cells given as uint64 rows. O(U^2 W)."""
    c = np.asarray(cells_u64, dtype=np.uint64)
    u = c.shape[0]
    out = []
    for i in range(u):
        if i + 1 >= u:
            break
        x = c[i + 1:] ^ c[i]
        dist = popcount64(x).sum(axis=1)
        js = np.nonzero(dist == 1)[0] + i + 1
        out.extend((i, int(j)) for j in js)
    return np.array(out, dtype=np.uint32).reshape(-1, 2)


def as_u64_rows(keys, ell: int, word_bits: int) -> np.ndarray:
    """Re-express packed rows with 64-bit words (same value)."""
    if word_bits == 64:
        return np.asarray(keys, dtype=np.uint64)
    return ints_to_rows(rows_to_ints(keys, 32), ell, 64)
