"""Pins of the paper-order interval SS oracle (oracle/interval_ss.py).

The interval FFT is pinned to the DFT definition of Section 2.2 (direct sums
with exact rational twiddles), the convolution to the exact coefficients of
Section 2.1, and the product digits to the exact product.  A wrong sign,
index or dropped term moves a value outside its enclosure.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import interval as iv
from oracle import interval_ss as S
from oracle import twiddle as tw


@pytest.mark.parametrize("n,sign", [(1, 1), (2, 1), (4, -1), (8, 1), (16, -1), (32, 1)])
def test_fft_contains_dft_definition(n, sign):
    rng = np.random.default_rng(n)
    xr = rng.integers(0, 256, n).astype(float)
    xi = rng.integers(0, 256, n).astype(float)
    X = S.fft(iv.ic_point(xr, xi), sign)
    for k in range(n):
        re, im, rad = Fr(0), Fr(0), Fr(0)
        for j in range(n):
            (c, ec), (s, es) = tw.exact_fraction(max(n, 1), (j * k) % n) if n >= 4 else \
                ((Fr([1, -1][(j * k) % n] if n == 2 else 1), Fr(0)), (Fr(0), Fr(0)))
            s = s * sign
            a, b = Fr(float(xr[j])), Fr(float(xi[j]))
            re += a * c - b * s
            im += a * s + b * c
            rad += (abs(a) + abs(b)) * (ec + es)
        assert Fr(float(X[0][k])) <= re - rad and re + rad <= Fr(float(X[1][k]))
        assert Fr(float(X[2][k])) <= im - rad and im + rad <= Fr(float(X[3][k]))


def test_inverse_recovers_input():
    x = np.arange(16, dtype=float)
    X = S.fft(iv.ic_point(x), +1)
    y = iv.ic_scale_pow2(S.fft(X, -1), 4)
    assert np.all((y[0] <= x) & (x <= y[1]))
    assert np.all((y[2] <= 0) & (0 <= y[3]))


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 2), (2, 1), (3, 3), (5, 11), (16, 16), (17, 1), (64, 63),
                                   (100, 1000), (1024, 1024), (2000, 96)])
def test_multiply_exact_and_contains(na, nb):
    a, b = synth.operand_pair(na * 31 + nb, na, nb)
    r = S.multiply(a, b)
    assert r["status"] == S.STATUS_OK
    assert np.array_equal(r["digits"], E.product(a, b))
    c = E.conv(a, b).astype(float)
    lo, hi, ilo, ihi = r["intervals"]
    assert np.all((lo <= c) & (c <= hi))
    assert np.all((ilo <= 0) & (0 <= ihi))


def test_exhaustive_small_lengths():
    for na in range(1, 20):
        for nb in range(1, 20, 3):
            a, b = synth.operand_pair(na * 100 + nb, na, nb, "raw")
            r = S.multiply(a, b)
            assert r["status"] == S.STATUS_OK
            assert np.array_equal(r["digits"], E.product(a, b))


def test_all_ff_and_zero():
    a = np.full(300, 0xFF, np.uint8)
    r = S.multiply(a, a)
    assert r["status"] == S.STATUS_OK and np.array_equal(r["digits"], E.product(a, a))
    z = np.zeros(40, np.uint8)
    r = S.multiply(z, a)
    assert r["status"] == S.STATUS_OK and not r["digits"].any() and r["max_width"] == 0.0


def test_fft_length_rule():
    # k = ceil(log2(2n - 1)) for equal lengths (Section 2.3)
    for n in range(1, 200):
        m = S.fft_length(n, n)
        assert m >= 2 * n - 1 and (m == 1 or m // 2 < 2 * n - 1) and m & (m - 1) == 0


def test_f32_small_and_failure_reported():
    a, b = synth.operand_pair(4, 3, 3)
    r = S.multiply(a, b, iv.F32)
    assert r["status"] == S.STATUS_OK and np.array_equal(r["digits"], E.product(a, b))
    # binary32 cannot resolve coefficients near 2^24: reported, never rounded
    a, b = synth.operand_pair(4, 512, 512)
    r = S.multiply(a, b, iv.F32)
    assert r["status"] == S.STATUS_ISOLATION_FAILED
    assert not r["digits"].any()
    c = E.conv(a, b).astype(float)
    lo, hi, _, _ = r["intervals"]
    assert np.all((lo <= c) & (c <= hi))
