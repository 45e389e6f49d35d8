"""Pins of the exact oracle (oracle/exact.py) to facts outside itself.

Python's built-in integers give an independent exact product; closed forms
for all-0xFF operands, the DC and alternating-sum invariants of a
convolution, shifts by powers of the base and residues modulo primes catch a
dropped term, a wrong index or a transposed operand in any routine.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E

PRIMES = [2**31 - 1, 2**61 - 1, 1_000_000_007, 0xFFFFFFFF00000001]


def _pyprod(a, b):
    return E.from_int(E.to_int(a) * E.to_int(b), len(a) + len(b))


def test_exhaustive_one_by_one():
    # Section 2.1 with n = m = 1: z = x0*y0 as two digits
    for x in range(256):
        xs = np.array([x], np.uint8)
        for y in range(0, 256, 1):
            z = E.long_mul(xs, np.array([y], np.uint8))
            assert int(z[0]) + 256 * int(z[1]) == x * y


def test_one_by_two_sampled():
    ys = [0, 1, 2, 127, 128, 200, 254, 255]
    for x in range(256):
        for y0 in ys:
            for y1 in ys:
                z = E.long_mul(np.array([x], np.uint8), np.array([y0, y1], np.uint8))
                assert E.to_int(z) == x * (y0 + 256 * y1)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    na, nb = rng.integers(1, 9, size=2)
    a, b = synth.operand_pair(seed, int(na), int(nb), "raw")
    expect = _pyprod(a, b)
    assert np.array_equal(E.long_mul(a, b), expect)
    assert np.array_equal(E.product(a, b), expect)
    assert np.array_equal(E.carry(E.conv(a, b), na + nb), expect)


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 300), (300, 1), (17, 1000), (2048, 2048), (3000, 2500), (4096, 4096)])
def test_against_python_int(na, nb):
    a, b = synth.operand_pair(11 + na, na, nb)
    expect = _pyprod(a, b)
    assert np.array_equal(E.long_mul(a, b), expect)
    assert np.array_equal(E.product(a, b), expect)


@pytest.mark.parametrize("na,nb", [(1, 1), (5, 3), (1000, 1), (777, 1234), (1 << 12, 1 << 12), (1 << 15, 1 << 13), (40000, 40000)])
def test_ntt_matches_schoolbook(na, nb):
    a, b = synth.operand_pair(na * 3 + nb, na, nb, "raw")
    assert np.array_equal(E.conv(a, b), E.conv_ntt(a, b))


@pytest.mark.parametrize("na,nb", [(1 << 18, 1 << 18), (1 << 20, 1 << 12)])
def test_ntt_product_against_python_int(na, nb):
    a, b = synth.operand_pair(5, na, nb)
    z = E.carry(E.conv_ntt(a, b), na + nb)
    assert E.to_int(z) == E.to_int(a) * E.to_int(b)


def test_ntt_root_is_primitive():
    p = E.ntt_prime()
    assert p == 2**64 - 2**32 + 1
    for k in (1, 5, 18, 24):
        n = 1 << k
        w = E.ntt_root(n)
        assert pow(w, n, p) == 1
        assert pow(w, n // 2, p) == p - 1


@pytest.mark.parametrize("n", [1, 2, 3, 100, 4096, 75000])
def test_all_ff_closed_form(n):
    # (256^n - 1)^2 = 256^(2n) - 2*256^n + 1: digits 01, 00.., FE, FF..
    a = np.full(n, 0xFF, np.uint8)
    z = E.product(a, a)
    expect = np.zeros(2 * n, np.uint8)
    expect[0] = 0x01
    expect[n] = 0xFE
    expect[n + 1:] = 0xFF
    if n == 1:
        expect = np.array([0x01, 0xFE], np.uint8)
    assert np.array_equal(z, expect)
    c = E.conv(a, a) if n < 50000 else E.conv_ntt(a, a)
    i = np.arange(2 * n - 1)
    closed = 65025 * np.minimum.reduce([i + 1, np.full_like(i, n), 2 * n - 1 - i])
    assert np.array_equal(c, closed.astype(np.uint64))
    assert int(c.max()) == 65025 * n


def test_all_ff_max_coefficient_at_75000():
    # the largest coefficient of the paper-scale worst case, 75,000 * 255^2
    a = np.full(75000, 0xFF, np.uint8)
    assert int(E.conv_ntt(a, a).max()) == 4_876_875_000


@pytest.mark.parametrize("na,nb", [(3, 5), (1000, 999), (4096, 17), (20000, 30000)])
def test_convolution_invariants(na, nb):
    a, b = synth.operand_pair(na + 7 * nb, na, nb, "raw")
    c = E.conv(a, b)
    # DC bin of the convolution theorem at i = 0: sum c = (sum a)(sum b)
    assert int(c.astype(object).sum()) == int(a.astype(object).sum()) * int(b.astype(object).sum())
    # evaluation at -1: sum (-1)^i c_i = a(-1) b(-1)
    sgn = lambda n: np.where(np.arange(n) % 2 == 0, 1, -1).astype(object)
    lhs = int((c.astype(object) * sgn(len(c))).sum())
    rhs = int((a.astype(object) * sgn(na)).sum()) * int((b.astype(object) * sgn(nb)).sum())
    assert lhs == rhs


@pytest.mark.parametrize("k", [0, 1, 7, 300])
def test_shift_by_power_of_base(k):
    y = synth.uniform_digits(99, 500)
    x = np.zeros(k + 1, np.uint8)
    x[k] = 1                      # x = 256^k
    z = E.product(x, y)
    expect = np.zeros(k + 1 + 500, np.uint8)
    expect[k:k + 500] = y
    assert np.array_equal(z, expect)
    assert np.array_equal(E.long_mul(x, y), expect)


def test_zero_operands():
    a = np.zeros(50, np.uint8)
    b = synth.uniform_digits(3, 70)
    assert not E.product(a, b).any()
    assert not E.long_mul(b, a).any()


@pytest.mark.parametrize("na,nb", [(4096, 4096), (75000, 75000), (1 << 20, 1 << 12)])
def test_residues(na, nb):
    a, b = synth.operand_pair(na ^ nb, na, nb)
    z = E.product(a, b)
    c = E.conv_auto(a, b)
    for p in PRIMES:
        ra, rb = E.residue(a, p), E.residue(b, p)
        assert E.residue(z, p) == ra * rb % p
        assert E.residue_coeffs(c, p) == ra * rb % p


def test_residue_against_python():
    a = synth.uniform_digits(1, 1000)
    for p in PRIMES:
        assert E.residue(a, p) == E.to_int(a) % p


def test_carry_against_python():
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2**40, size=500, dtype=np.uint64)
    v = sum(int(ci) << (8 * i) for i, ci in enumerate(c))
    nz = (v.bit_length() + 7) // 8
    z = E.carry(c, nz)
    assert E.to_int(z) == v
    with pytest.raises(ValueError):
        E.carry(c, nz - 1)
