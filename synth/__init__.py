"""Seeded synthetic operands for the interval Schoenhage-Strassen multiplier.

This module holds no arithmetic of the multiplication method. It only draws
the base-256 digit vectors (little-endian, digit 0 least significant, as in
the paper's digit convention of Section 2) and the batch size mixes that the
tests, the oracle and the benchmark share.

Random bits come from the counter-based splitmix64 generator (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
word k of stream s is mix(s + (k + 1) * 0x9E3779B97F4A7C15) with the
published finaliser constants.  The paper's timing study uses uniformly
random n-digit base-256 inputs (Section 3); "uniform" here means i.i.d. bytes
in [0, 255] with the most significant digit redrawn in [1, 255] so the
operand has exactly n significant digits.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: seed base for the named workloads; workload w uses SEED_BASE + w
SEED_BASE = 0x55AA0000


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Words offset .. offset+count-1 of the splitmix64 stream for `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _substream(seed: int, tag: int) -> int:
    """A derived seed, so independent draws never share words."""
    return int(splitmix64(seed ^ (tag * 0xD1B54A32D192ED03 & 0xFFFFFFFFFFFFFFFF), 1)[0])


def uniform_digits(seed: int, n: int, top_nonzero: bool = True) -> np.ndarray:
    """n i.i.d. uniform bytes; the top digit is redrawn in [1, 255]."""
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    words = splitmix64(seed, (n + 7) // 8)
    d = words.view(np.uint8)[:n].copy()
    if top_nonzero:
        d[n - 1] = np.uint8(1 + int(splitmix64(seed, 1, offset=(n + 7) // 8)[0] % 255))
    return d


def all_ff_digits(n: int) -> np.ndarray:
    """The all-0xFF operand 256^n - 1: every coefficient at its maximum."""
    return np.full(n, 0xFF, dtype=np.uint8)


def operand_pair(seed: int, na: int, nb: int, dist: str = "uniform"):
    """Operands (a, b) of na and nb digits drawn from `dist`.

    dist: "uniform" (top digit nonzero), "ff" (all 0xFF), "zero" (all zero
    digits), "raw" (uniform bytes, top digit unconstrained).
    """
    if dist == "uniform":
        return (uniform_digits(_substream(seed, 1), na),
                uniform_digits(_substream(seed, 2), nb))
    if dist == "raw":
        return (uniform_digits(_substream(seed, 1), na, top_nonzero=False),
                uniform_digits(_substream(seed, 2), nb, top_nonzero=False))
    if dist == "ff":
        return all_ff_digits(na), all_ff_digits(nb)
    if dist == "zero":
        return np.zeros(na, np.uint8), np.zeros(nb, np.uint8)
    raise ValueError(f"unknown distribution {dist!r}")


def uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """count integers uniform in [lo, hi] (inclusive), by 64-bit modulo."""
    w = splitmix64(seed, count)
    return (lo + (w % np.uint64(hi - lo + 1))).astype(np.int64)


def unit_uniform(seed: int, count: int) -> np.ndarray:
    """count doubles uniform in [0, 1) from the top 53 bits of each word."""
    w = splitmix64(seed, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def ladder_batch(seed: int, count: int = 4096, lo: int = 512, hi: int = 32768,
                 ff_fraction: float = 0.10):
    """Size mix of the precision-ladder workload: square products with
    n ~ U{lo..hi}; a seeded Bernoulli(ff_fraction) marks all-0xFF products.
    Returns (na, nb, dist) arrays."""
    n = uniform_int(_substream(seed, 3), count, lo, hi)
    ff = unit_uniform(_substream(seed, 4), count) < ff_fraction
    return n.copy(), n.copy(), np.where(ff, "ff", "uniform")


def uneven_batch(seed: int, count: int = 20000, lo: int = 64, hi: int = 131072):
    """Size mix of the batched uneven workload: na and nb independent and
    log-uniform in [lo, hi], n = floor(lo * (hi/lo)^U)."""
    ua = unit_uniform(_substream(seed, 5), count)
    ub = unit_uniform(_substream(seed, 6), count)
    r = hi / lo
    na = np.minimum(hi, np.floor(lo * r ** ua)).astype(np.int64)
    nb = np.minimum(hi, np.floor(lo * r ** ub)).astype(np.int64)
    return na, nb, np.array(["uniform"] * count)


def batch_operands(seed: int, na, nb, dists):
    """Concatenated digit pools and offsets for a batch of products.

    Returns (a_pool, b_pool, a_off, b_off, z_off) where product p reads
    a_pool[a_off[p] : a_off[p] + na[p]] and writes na[p] + nb[p] digits at
    z_off[p]."""
    na = np.asarray(na, np.int64)
    nb = np.asarray(nb, np.int64)
    a_off = np.concatenate([[0], np.cumsum(na)[:-1]]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(nb)[:-1]]).astype(np.int64)
    z_off = np.concatenate([[0], np.cumsum(na + nb)[:-1]]).astype(np.int64)
    a_pool = np.empty(int(na.sum()), np.uint8)
    b_pool = np.empty(int(nb.sum()), np.uint8)
    for p in range(len(na)):
        a, b = operand_pair(_substream(seed, 1000 + p), int(na[p]), int(nb[p]), str(dists[p]))
        a_pool[a_off[p]:a_off[p] + na[p]] = a
        b_pool[b_off[p]:b_off[p] + nb[p]] = b
    return a_pool, b_pool, a_off, b_off, z_off
