"""Pins of the root-of-unity enclosures (oracle/twiddle.py, Section 2.2)."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import twiddle as tw

# pi to 60 decimals (its published expansion)
PI_60 = Fr("3.141592653589793238462643383279502884197169399375105820974944")


def test_pi_digits():
    v, e = tw.pi_fixed()
    pi = Fr(v, 1 << tw.PREC)
    assert abs(pi - PI_60) <= Fr(e + 1, 1 << tw.PREC) + Fr(1, 10 ** 60)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 1024, 8192, 24, 96, 3072, 40, 640])
def test_exact_points_and_widths(N):
    c_lo, c_hi, s_lo, s_hi = tw.enclosures(N)
    pts = {0: (1, 0)}
    if N >= 2:
        pts[N // 2] = (-1, 0)
    if N >= 4:
        pts.update({N // 4: (0, 1), 3 * N // 4: (0, -1)})
    for j, (c, s) in pts.items():
        assert (c_lo[j], c_hi[j], s_lo[j], s_hi[j]) == (c, c, s, s)
    # at most one ulp wide, or two around a value that is a double itself
    # (+-1/2 at the sixths of a turn when 3 divides N)
    for lo, hi in ((c_lo, c_hi), (s_lo, s_hi)):
        assert np.all(hi >= lo)
        one = hi <= np.nextafter(lo, np.inf)
        mid = np.nextafter(lo, np.inf)
        two = (hi <= np.nextafter(mid, np.inf)) & (np.abs(mid) == 0.5)
        assert np.all(one | two)
        if N % 3:
            assert np.all(one)


@pytest.mark.parametrize("N", [16, 256, 4096, 48, 1536, 80, 1280])
def test_pythagoras_and_libm(N):
    c_lo, c_hi, s_lo, s_hi = tw.enclosures(N)
    for j in range(0, N, max(1, N // 512)):
        # cos^2 + sin^2 = 1 must be possible inside the box
        cl, ch, sl, sh = (Fr(float(x[j])) for x in (c_lo, c_hi, s_lo, s_hi))
        c2 = sorted([cl * cl, ch * ch])
        s2 = sorted([sl * sl, sh * sh])
        cmin = 0 if cl <= 0 <= ch else c2[0]
        smin = 0 if sl <= 0 <= sh else s2[0]
        assert cmin + smin <= 1 <= c2[1] + s2[1]
        # the C library value (its argument is itself rounded: allow 1e-15)
        ang = 2 * math.pi * j / N
        assert np.nextafter(c_lo[j], -np.inf) - 1e-15 <= math.cos(ang) <= np.nextafter(c_hi[j], np.inf) + 1e-15
        assert np.nextafter(s_lo[j], -np.inf) - 1e-15 <= math.sin(ang) <= np.nextafter(s_hi[j], np.inf) + 1e-15


def test_closed_forms():
    # cos(pi/4) = sqrt(2)/2: lo^2 <= 1/2 <= hi^2
    c_lo, c_hi, s_lo, s_hi = tw.enclosures(8)
    assert Fr(float(c_lo[1])) ** 2 <= Fr(1, 2) <= Fr(float(c_hi[1])) ** 2
    assert Fr(float(s_lo[1])) ** 2 <= Fr(1, 2) <= Fr(float(s_hi[1])) ** 2
    # cos(pi/8): (4 c^2 - 2)^2 = 2, increasing in c on [0.9, 1]
    c_lo, c_hi, _, _ = tw.enclosures(16)
    f = lambda c: (4 * c * c - 2) ** 2
    assert f(Fr(float(c_lo[1]))) <= 2 <= f(Fr(float(c_hi[1])))


@pytest.mark.parametrize("N", [64, 2048])
def test_double_angle(N):
    # cos(2t) = 2 cos(t)^2 - 1 between entries j of N and j of N/2
    c_lo, c_hi, _, _ = tw.enclosures(N)
    h_lo, h_hi, _, _ = tw.enclosures(N // 2)
    for j in range(1, N // 8):
        lo = 2 * Fr(float(c_lo[j])) ** 2 - 1
        hi = 2 * Fr(float(c_hi[j])) ** 2 - 1
        assert not (hi < Fr(float(h_lo[j])) or lo > Fr(float(h_hi[j])))


def test_f32_enclosures_contain_f64():
    c64 = tw.enclosures(1024)
    c32 = tw.enclosures(1024, f32=True)
    assert np.all(c32[0] <= c64[0]) and np.all(c64[1] <= c32[1])
    assert np.all(c32[2] <= c64[2]) and np.all(c64[3] <= c32[3])
    assert np.all(c32[0].astype(np.float32).astype(np.float64) == c32[0])


def test_closed_forms_thirds():
    # lengths 3 2^k: sin(pi/6) = 1/2 and cos(pi/6)^2 = 3/4 (N = 24, j = 2);
    # cos(2 pi/3) = -1/2 (N = 24, j = 8); cos(pi/12): (2 c^2 - 1)^2 = 3/4 on [0.9, 1]
    c_lo, c_hi, s_lo, s_hi = tw.enclosures(24)
    assert s_lo[2] <= 0.5 <= s_hi[2]
    assert Fr(float(c_lo[2])) ** 2 <= Fr(3, 4) <= Fr(float(c_hi[2])) ** 2
    assert c_lo[8] <= -0.5 <= c_hi[8]
    assert Fr(float(s_lo[8])) ** 2 <= Fr(3, 4) <= Fr(float(s_hi[8])) ** 2
    f = lambda c: (2 * c * c - 1) ** 2
    assert f(Fr(float(c_lo[1]))) <= Fr(3, 4) <= f(Fr(float(c_hi[1])))


@pytest.mark.parametrize("N", [96, 3072, 160, 2560])
def test_double_angle_thirds(N):
    # cos(2t) = 2 cos(t)^2 - 1 between entries j of N and j of N/2 (both 3 2^k)
    c_lo, c_hi, _, _ = tw.enclosures(N)
    h_lo, h_hi, _, _ = tw.enclosures(N // 2)
    for j in range(1, N // 8):
        lo = 2 * Fr(float(c_lo[j])) ** 2 - 1
        hi = 2 * Fr(float(c_hi[j])) ** 2 - 1
        assert not (hi < Fr(float(h_lo[j])) or lo > Fr(float(h_hi[j])))


def test_rejects_lengths_without_octant_symmetry():
    with pytest.raises(ValueError):
        tw.octant_table(12)


def test_closed_forms_fifths():
    # lengths 5 2^k: cos(2 pi / 5) = (sqrt 5 - 1)/4 is the root of 4c^2 + 2c - 1
    # (increasing for c > -1/4); cos(pi / 5) = (sqrt 5 + 1)/4 that of 4c^2 - 2c - 1
    # (increasing for c > 1/4) (N = 40, j = 8 and j = 4)
    c_lo, c_hi, _, _ = tw.enclosures(40)
    f = lambda c: 4 * c * c + 2 * c - 1
    assert f(Fr(float(c_lo[8]))) <= 0 <= f(Fr(float(c_hi[8])))
    g = lambda c: 4 * c * c - 2 * c - 1
    assert g(Fr(float(c_lo[4]))) <= 0 <= g(Fr(float(c_hi[4])))
