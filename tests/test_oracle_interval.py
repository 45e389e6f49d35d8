"""Pins of the directed-rounding and interval oracle (oracle/interval.py).

Each directed operation is checked against exact rational arithmetic: the
result must be a double on the correct side of the exact value, and its
neighbour in the rounding direction must lie on the other side (so it is
the closest one).  Interval operations are checked to contain the exact
hull of the operation over the box corners (Section 2.5).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import interval as iv


def _vals(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-30, 30, n)
    x[:8] = [0.0, 1.0, -1.0, 0.5, 3.0, 1e-300 * 0 + 2.0 ** -899, 2.0 ** 899, 1.0 + 2.0 ** -52]
    return x


def _check_down(r, exact):
    assert Fr(float(r)) <= exact
    nxt = np.nextafter(float(r), np.inf)
    assert Fr(float(nxt)) > exact


def _check_up(r, exact):
    assert Fr(float(r)) >= exact
    prv = np.nextafter(float(r), -np.inf)
    assert Fr(float(prv)) < exact


@pytest.mark.parametrize("seed", range(4))
def test_f64_directed_ops(seed):
    a, b = _vals(seed, 300), _vals(seed + 100, 300)[::-1]
    # include exact cases and cancellation
    b[10], a[10] = -a[10], a[10]
    b[11] = a[11]
    for fn, op, down in [(iv.add_rd, lambda x, y: x + y, True), (iv.add_ru, lambda x, y: x + y, False),
                         (iv.sub_rd, lambda x, y: x - y, True), (iv.sub_ru, lambda x, y: x - y, False),
                         (iv.mul_rd, lambda x, y: x * y, True), (iv.mul_ru, lambda x, y: x * y, False)]:
        r = fn(a, b)
        for k in range(len(a)):
            ex = op(Fr(float(a[k])), Fr(float(b[k])))
            if fn in (iv.mul_rd, iv.mul_ru) and ex != 0 and abs(ex) < Fr(2) ** -900:
                continue
            (_check_down if down else _check_up)(r[k], ex)


def test_f64_division_and_sqrt():
    rng = np.random.default_rng(3)
    a = rng.uniform(-100, 100, 200)
    b = rng.uniform(0.1, 50, 200) * np.where(rng.random(200) < 0.5, -1, 1)
    lo, hi = iv.div_rd(a, b), iv.div_ru(a, b)
    for k in range(200):
        ex = Fr(float(a[k])) / Fr(float(b[k]))
        _check_down(lo[k], ex)
        _check_up(hi[k], ex)
    x = np.abs(a)
    slo, shi = iv.sqrt_rd(x), iv.sqrt_ru(x)
    for k in range(200):
        X = Fr(float(x[k]))
        assert Fr(float(slo[k])) ** 2 <= X <= Fr(float(shi[k])) ** 2
        assert Fr(float(np.nextafter(slo[k], np.inf))) ** 2 > X or slo[k] == shi[k]
    # exact cases stay points
    assert iv.sqrt_rd(np.array([4.0]))[0] == 2.0 == iv.sqrt_ru(np.array([4.0]))[0]


def test_f32_directed_ops():
    rng = np.random.default_rng(5)
    a = (rng.standard_normal(300) * 10.0 ** rng.integers(-10, 10, 300)).astype(np.float32).astype(np.float64)
    b = (rng.standard_normal(300) * 10.0 ** rng.integers(-10, 10, 300)).astype(np.float32).astype(np.float64)
    b[0] = -a[0]
    f32up = lambda r: float(np.nextafter(np.float32(r), np.float32(np.inf)))
    f32dn = lambda r: float(np.nextafter(np.float32(r), np.float32(-np.inf)))
    for fn, op, down in [(iv.add_rd32, lambda x, y: x + y, True), (iv.add_ru32, lambda x, y: x + y, False),
                         (iv.sub_rd32, lambda x, y: x - y, True), (iv.sub_ru32, lambda x, y: x - y, False),
                         (iv.mul_rd32, lambda x, y: x * y, True), (iv.mul_ru32, lambda x, y: x * y, False)]:
        r = fn(a, b)
        for k in range(300):
            ex = op(Fr(float(a[k])), Fr(float(b[k])))
            assert float(np.float32(r[k])) == r[k]
            if down:
                assert Fr(float(r[k])) <= ex < Fr(f32up(r[k]))
            else:
                assert Fr(f32dn(r[k])) < ex <= Fr(float(r[k]))


def test_real_interval_mul_hull():
    rng = np.random.default_rng(9)
    for _ in range(200):
        a = np.sort(rng.uniform(-5, 5, 2))
        b = np.sort(rng.uniform(-5, 5, 2))
        if rng.random() < 0.3:
            b = np.abs(b) + 0.1
        lo, hi = iv.ir_mul((a[:1], a[1:]), (b[:1], b[1:]))
        corners = [Fr(float(x)) * Fr(float(y)) for x in a for y in b]
        _check_down(lo[0], min(corners))
        _check_up(hi[0], max(corners))


def test_complex_interval_mul_contains_points():
    rng = np.random.default_rng(10)
    for _ in range(100):
        z = [np.sort(rng.uniform(-3, 3, 2)) for _ in range(2)]
        w = [np.sort(rng.uniform(-3, 3, 2)) for _ in range(2)]
        Z = (z[0][:1], z[0][1:], z[1][:1], z[1][1:])
        W = (w[0][:1], w[0][1:], w[1][:1], w[1][1:])
        P = iv.ic_mul(Z, W)
        for t in np.linspace(0, 1, 4):
            zr = Fr(float(z[0][0])) * (1 - Fr(t)) + Fr(float(z[0][1])) * Fr(t)
            zi = Fr(float(z[1][1])) * (1 - Fr(t)) + Fr(float(z[1][0])) * Fr(t)
            wr = Fr(float(w[0][1])) * (1 - Fr(t)) + Fr(float(w[0][0])) * Fr(t)
            wi = Fr(float(w[1][0])) * (1 - Fr(t)) + Fr(float(w[1][1])) * Fr(t)
            re, im = zr * wr - zi * wi, zr * wi + zi * wr
            assert Fr(float(P[0][0])) <= re <= Fr(float(P[1][0]))
            assert Fr(float(P[2][0])) <= im <= Fr(float(P[3][0]))


def test_complex_interval_add_sub_sharp():
    z = (np.array([1.0]), np.array([2.0]), np.array([-1.0]), np.array([0.5]))
    w = (np.array([0.25]), np.array([0.5]), np.array([3.0]), np.array([4.0]))
    s = iv.ic_add(z, w)
    d = iv.ic_sub(z, w)
    assert [x[0] for x in s] == [1.25, 2.5, 2.0, 4.5]
    assert [x[0] for x in d] == [0.5, 1.75, -5.0, -2.5]


def test_scale_pow2_exact():
    z = iv.ic_point(np.array([3.0, -7.5]), np.array([1.0, 0.0]))
    s = iv.ic_scale_pow2(z, 3)
    assert list(s[0]) == [0.375, -0.9375]


@pytest.mark.parametrize("lo,hi,val,code", [
    (0.1, 1.9, 1, iv.ISOLATED), (1.0, 2.0, 0, iv.AMBIGUOUS), (1.2, 1.8, 0, iv.EMPTY),
    (2.0, 2.0, 2, iv.ISOLATED), (-0.5, 0.5, 0, iv.ISOLATED), (41.9999, 42.0, 42, iv.ISOLATED),
    (4876874999.5, 4876875000.25, 4876875000, iv.ISOLATED), (-1.5, 0.9, 0, iv.AMBIGUOUS),
])
def test_isolation_cases(lo, hi, val, code):
    v, c = iv.isolate(np.array([lo]), np.array([hi]), np.array([-1e-9]), np.array([1e-9]))
    assert int(c[0]) == code
    if code == iv.ISOLATED:
        assert int(v[0]) == val


def test_isolation_imaginary_part():
    v, c = iv.isolate(np.array([0.9]), np.array([1.1]), np.array([0.1]), np.array([0.2]))
    assert int(c[0]) == iv.IMAG_EXCLUDES_ZERO
    v, c = iv.isolate(np.array([0.9]), np.array([1.1]), np.array([0.0]), np.array([0.2]))
    assert int(c[0]) == iv.ISOLATED


def test_domain_guard():
    with pytest.raises(FloatingPointError):
        iv.add_rd(np.array([np.inf]), np.array([1.0]))
