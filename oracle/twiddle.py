"""Rigorous enclosures of the roots of unity omega_N^j = e^{2 pi i j / N} (Section 2.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's transform uses omega = e^{2 pi i / n} (the DFT definition of
Section 2.2) and forms the powers omega^i inside the FFT; it gives a
recurrence for the principal roots (omega_{2n} = (1 + omega_n) / |1 + omega_n|)
but not how the powers are enclosed.  This oracle encloses every power
directly: cos(2 pi j / N) and sin(2 pi j / N) are computed in fixed point
with PREC fractional bits by exact integer arithmetic (Machin's formula for
pi, Taylor series for sin and cos on [0, pi/4]), each with a proved bound
on its error in units of 2^-PREC, and the resulting rational enclosure is
rounded outward to binary64 (or binary32).  Exact values (0, +-1) give
point intervals.  Symmetries of the circle map j to the first octant
without error whenever N is a multiple of 8 (powers of two >= 8 and the
lengths 3 2^k, k >= 3): the quarter turn N/4 and the octant N/8 are then
whole steps.

Pins (tests/test_oracle_twiddle.py): pi against its published decimal
expansion, cos^2 + sin^2 = 1 on the exact rational bounds, containment of
the values from the C library's cos/sin, widths of at most one ulp.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np

PREC = 200                 # fractional bits of the fixed-point computation
_ONE = 1 << PREC


def _arctan_inv(x: int) -> tuple[int, int]:
    """arctan(1/x) in fixed point, and a bound on its error (in units)."""
    total, k, err = 0, 0, 0
    xp = x                 # x^(2k+1)
    while True:
        term = _ONE // (xp * (2 * k + 1))    # truncated: error < 1 unit
        if term == 0:
            break
        total += term if k % 2 == 0 else -term
        err += 1
        k += 1
        xp *= x * x
    return total, err + 1  # + the alternating tail, below one unit


@lru_cache(maxsize=1)
def pi_fixed() -> tuple[int, int]:
    """pi = 16 arctan(1/5) - 4 arctan(1/239) (Machin), in fixed point."""
    a, ea = _arctan_inv(5)
    b, eb = _arctan_inv(239)
    return 16 * a - 4 * b, 16 * ea + 4 * eb


def _sin_cos_fixed(theta: int, etheta: int):
    """sin and cos of theta (fixed point, 0 <= theta <= pi/4 + tiny) with error bounds.

    Taylor series with truncating integer division; every truncation costs
    below one unit, the tail is below its first omitted term, and the input
    error etheta moves sin and cos by at most etheta (both are 1-Lipschitz).
    """
    s, c = 0, 0
    es = ec = 0
    term = theta           # theta^(2k+1)/(2k+1)!  (for sin)
    k = 0
    while term != 0:
        s += term if k % 2 == 0 else -term
        es += 1
        term = term * theta // _ONE * theta // _ONE // ((2 * k + 2) * (2 * k + 3))
        es += 2
        k += 1
    term = _ONE            # theta^(2k)/(2k)!  (for cos)
    k = 0
    while term != 0:
        c += term if k % 2 == 0 else -term
        ec += 1
        term = term * theta // _ONE * theta // _ONE // ((2 * k + 1) * (2 * k + 2))
        ec += 2
        k += 1
    # the per-term truncation errors propagate through later terms with
    # factor theta^2/((2k+1)(2k+2)) < 1, so the counts above dominate them
    return (s, es + etheta + 2), (c, ec + etheta + 2)


def _octant_value(jj: int, N: int):
    """(sin, err), (cos, err) of 2 pi jj / N for 0 <= jj <= N/8."""
    pi, epi = pi_fixed()
    theta = 2 * pi * jj // N
    etheta = (2 * epi * jj) // N + 1
    return _sin_cos_fixed(theta, etheta)


def _to_double_down(num: Fraction, f32: bool = False) -> float:
    x = float(num)
    if f32:
        x = float(np.float32(x))
        while Fraction(x) > num:
            x = float(np.nextafter(np.float32(x), np.float32(-np.inf)))
    else:
        while Fraction(x) > num:
            x = float(np.nextafter(x, -np.inf))
    return x


def _to_double_up(num: Fraction, f32: bool = False) -> float:
    x = float(num)
    if f32:
        x = float(np.float32(x))
        while Fraction(x) < num:
            x = float(np.nextafter(np.float32(x), np.float32(np.inf)))
    else:
        while Fraction(x) < num:
            x = float(np.nextafter(x, np.inf))
    return x


def _enclose(v: int, e: int, f32: bool):
    lo = Fraction(v - e, _ONE)
    hi = Fraction(v + e, _ONE)
    return _to_double_down(lo, f32), _to_double_up(hi, f32)


@lru_cache(maxsize=64)
def octant_table(N: int, f32: bool = False):
    """Enclosures of cos and sin of 2 pi j / N for j = 0 .. N/8 (N >= 8).

    Returns four float64 arrays (cos_lo, cos_hi, sin_lo, sin_hi)."""
    if N < 8 or N % 8:
        raise ValueError("N must be a multiple of 8")
    m = N // 8
    out = np.zeros((4, m + 1))
    for jj in range(m + 1):
        if jj == 0:
            out[:, jj] = (1.0, 1.0, 0.0, 0.0)
            continue
        (s, es), (c, ec) = _octant_value(jj, N)
        out[0, jj], out[1, jj] = _enclose(c, ec, f32)
        out[2, jj], out[3, jj] = _enclose(s, es, f32)
    return out[0], out[1], out[2], out[3]


def enclosures(N: int, f32: bool = False):
    """Enclosures of cos(2 pi j/N) and sin(2 pi j/N) for all j in [0, N).

    Every j is mapped to the first octant by exact symmetries:
    j in octant 0: (c, s) = (C(jj), S(jj)); reflections about pi/4 swap
    C and S; adding a quarter turn maps (c, s) -> (-s, c).
    Returns (cos_lo, cos_hi, sin_lo, sin_hi) float64 arrays of length N.
    """
    if N in (1, 2, 4):
        c = {1: [1.0], 2: [1.0, -1.0], 4: [1.0, 0.0, -1.0, 0.0]}[N]
        s = {1: [0.0], 2: [0.0, 0.0], 4: [0.0, 1.0, 0.0, -1.0]}[N]
        c, s = np.array(c), np.array(s)
        return c, c.copy(), s, s.copy()
    clo, chi, slo, shi = octant_table(N, f32)
    q = N // 4
    j = np.arange(N)
    quad, r = j // q, j % q                  # angle = quad * pi/2 + r * 2pi/N
    refl = r > N // 8                        # second half of the quadrant
    jj = np.where(refl, q - r, r)
    # (c, s) of the in-quadrant angle
    c_lo = np.where(refl, slo[jj], clo[jj])
    c_hi = np.where(refl, shi[jj], chi[jj])
    s_lo = np.where(refl, clo[jj], slo[jj])
    s_hi = np.where(refl, chi[jj], shi[jj])
    # rotate by quad quarter turns: (c, s) -> (-s, c)
    C_lo, C_hi, S_lo, S_hi = c_lo.copy(), c_hi.copy(), s_lo.copy(), s_hi.copy()
    m1 = quad == 1
    C_lo[m1], C_hi[m1], S_lo[m1], S_hi[m1] = -s_hi[m1], -s_lo[m1], c_lo[m1], c_hi[m1]
    m2 = quad == 2
    C_lo[m2], C_hi[m2], S_lo[m2], S_hi[m2] = -c_hi[m2], -c_lo[m2], -s_hi[m2], -s_lo[m2]
    m3 = quad == 3
    C_lo[m3], C_hi[m3], S_lo[m3], S_hi[m3] = s_lo[m3], s_hi[m3], -c_hi[m3], -c_lo[m3]
    # quarter-turn symmetries produce -0.0 from +0.0; normalise to +0.0
    return C_lo + 0.0, C_hi + 0.0, S_lo + 0.0, S_hi + 0.0


def exact_fraction(N: int, j: int):
    """(cos, sin) of 2 pi j / N as exact rational midpoints with their error
    radius, for tests: returns ((c, ec), (s, es)) as Fractions."""
    q = N // 4
    quad, r = (j % N) // q, (j % N) % q
    refl = r > N // 8
    jj = q - r if refl else r
    (s, es), (c, ec) = _octant_value(jj, N) if jj else ((0, 0), (_ONE, 0))
    if refl:
        s, es, c, ec = c, ec, s, es
    for _ in range(quad):
        c, s = -s, c
        ec, es = es, ec
    return (Fraction(c, _ONE), Fraction(ec, _ONE)), (Fraction(s, _ONE), Fraction(es, _ONE))
