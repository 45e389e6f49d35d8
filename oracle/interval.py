"""Directed rounding and interval arithmetic (Section 2.5), vectorised in numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Directed rounding.  numpy computes IEEE binary64 with round-to-nearest.
The exact result of a sum or product of two doubles is recovered with
error-free transformations: Knuth's TwoSum (The Art of Computer Programming
vol. 2, 4.2.2, Theorem B) and Dekker's TwoProduct with Veltkamp splitting
(Dekker 1971).  The correctly rounded downward (upward) result is then the
round-to-nearest result, stepped one ulp down (up) when the exact error term
is negative (positive).  For binary32 operands the exact product fits in a
double and the exact sum is a double plus a TwoSum error, and the result is
rounded to binary32 and stepped the same way.

Interval arithmetic (Section 2.5):
  [a]+[b] = [a_lo + b_lo (down), a_hi + b_hi (up)]
  [a]-[b] = [a_lo - b_hi (down), a_hi - b_lo (up)]
  [a]*[b] = [min of the four endpoint products rounded down,
             max of the four endpoint products rounded up]
  [a]/[b] = [a] * [1/b_hi, 1/b_lo] when 0 is not in [b]
  sqrt[a] = [sqrt(a_lo) down, sqrt(a_hi) up] for a_lo >= 0
Rectangular complex intervals: add and subtract componentwise; multiply by
the formula (z1 w1 - z2 w2) + i (z1 w2 + z2 w1) in real interval operations;
division by a positive power of two scales both bounds exactly.

Isolation (Section 1; Section 2.5): the unique integer in a real interval,
or an error when it holds none or several; the imaginary part of an
output coefficient must contain 0.

Parity pins (tests/test_oracle_interval.py): every directed operation is
checked against exact rational arithmetic (fractions.Fraction) and a brute
force search for the neighbouring doubles; interval products against the
exact hull over a grid of points; isolation against hand-worked cases.

Domain: operands are finite and either 0 or of magnitude in
[2^-900, 2^900]; outside it the error-free transforms could overflow or
underflow and the functions raise.
"""
from __future__ import annotations

import numpy as np

F64, F32 = "f64", "f32"
_SPLIT = 134217729.0  # 2^27 + 1, Veltkamp splitter for binary64
_LIM_LO, _LIM_HI = 2.0 ** -900, 2.0 ** 900


def _check(*xs):
    for x in xs:
        ax = np.abs(x)
        bad = ~np.isfinite(x) | ((ax != 0) & ((ax < _LIM_LO) | (ax > _LIM_HI)))
        if np.any(bad):
            raise FloatingPointError("operand outside the exact-rounding domain")


def two_sum(a, b):
    """s = fl(a + b) and e with s + e == a + b exactly (Knuth)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """p = fl(a * b) and e with p + e == a * b exactly (Dekker)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _down(x, e):
    return np.where(e < 0, np.nextafter(x, -np.inf), x)


def _up(x, e):
    return np.where(e > 0, np.nextafter(x, np.inf), x)


# ---- binary64 ---------------------------------------------------------------

def add_rd(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    s, e = two_sum(a, b)
    return _down(s, e)


def add_ru(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    s, e = two_sum(a, b)
    return _up(s, e)


def sub_rd(a, b):
    return add_rd(a, -np.asarray(b, np.float64))


def sub_ru(a, b):
    return add_ru(a, -np.asarray(b, np.float64))


def mul_rd(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    p, e = two_prod(a, b)
    return _down(p, e)


def mul_ru(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    p, e = two_prod(a, b)
    return _up(p, e)


def div_rd(a, b):
    """a / b rounded down (b != 0): q = fl(a/b); the sign of a - q b decides."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    q = a / b
    p, e = two_prod(q, b)
    r = (a - p) - e          # a - q b, exact: Sterbenz and |r| tiny
    r = r * np.sign(b)       # sign of a/b - q
    return _down(q, r)


def div_ru(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    _check(a, b)
    q = a / b
    p, e = two_prod(q, b)
    r = ((a - p) - e) * np.sign(b)
    return _up(q, r)


def sqrt_rd(a):
    a = np.asarray(a, np.float64)
    s = np.sqrt(a)
    p, e = two_prod(s, s)
    r = (a - p) - e          # a - s^2
    return _down(s, r)


def sqrt_ru(a):
    a = np.asarray(a, np.float64)
    s = np.sqrt(a)
    p, e = two_prod(s, s)
    r = (a - p) - e
    return _up(s, r)


# ---- binary32 (values carried in float64 arrays) -----------------------------

def _round32(s, e, up: bool):
    """Directed rounding of the exact value s + e (doubles) to binary32."""
    f = s.astype(np.float32).astype(np.float64)
    d = f - s                # exact: f is within half a binary32 ulp of s
    if up:
        step = (d < e)       # f below the exact value
        g = np.nextafter(f.astype(np.float32), np.float32(np.inf)).astype(np.float64)
    else:
        step = (d > e)       # f above the exact value
        g = np.nextafter(f.astype(np.float32), np.float32(-np.inf)).astype(np.float64)
    return np.where(step, g, f)


def _as32(a):
    a = np.asarray(a, np.float64)
    if np.any(a.astype(np.float32).astype(np.float64) != a):
        raise ValueError("operand is not a binary32 value")
    return a


def add_rd32(a, b):
    s, e = two_sum(_as32(a), _as32(b))
    return _round32(s, e, up=False)


def add_ru32(a, b):
    s, e = two_sum(_as32(a), _as32(b))
    return _round32(s, e, up=True)


def sub_rd32(a, b):
    return add_rd32(a, -np.asarray(b, np.float64))


def sub_ru32(a, b):
    return add_ru32(a, -np.asarray(b, np.float64))


def mul_rd32(a, b):
    p = _as32(a) * _as32(b)  # exact: 24 x 24 bits fit in 53
    return _round32(p, np.zeros_like(p), up=False)


def mul_ru32(a, b):
    p = _as32(a) * _as32(b)
    return _round32(p, np.zeros_like(p), up=True)


def to32_rd(a):
    a = np.asarray(a, np.float64)
    return _round32(a, np.zeros_like(a), up=False)


def to32_ru(a):
    a = np.asarray(a, np.float64)
    return _round32(a, np.zeros_like(a), up=True)


def ops(prec: str):
    """(add_rd, add_ru, sub_rd, sub_ru, mul_rd, mul_ru) for a precision."""
    if prec == F64:
        return add_rd, add_ru, sub_rd, sub_ru, mul_rd, mul_ru
    if prec == F32:
        return add_rd32, add_ru32, sub_rd32, sub_ru32, mul_rd32, mul_ru32
    raise ValueError(prec)


# ---- real intervals (Section 2.5) ---------------------------------------------

def ir_add(a, b, prec=F64):
    ard, aru, *_ = ops(prec)
    return ard(a[0], b[0]), aru(a[1], b[1])


def ir_sub(a, b, prec=F64):
    _, _, srd, sru, _, _ = ops(prec)
    return srd(a[0], b[1]), sru(a[1], b[0])


def ir_mul(a, b, prec=F64):
    """[min of the 4 endpoint products (down), max of the 4 (up)]."""
    *_, mrd, mru = ops(prec)
    lo = np.minimum(np.minimum(mrd(a[0], b[0]), mrd(a[0], b[1])),
                    np.minimum(mrd(a[1], b[0]), mrd(a[1], b[1])))
    hi = np.maximum(np.maximum(mru(a[0], b[0]), mru(a[0], b[1])),
                    np.maximum(mru(a[1], b[0]), mru(a[1], b[1])))
    return lo, hi


def ir_div(a, b):
    """[a] / [b] = [a] * [1/b_hi, 1/b_lo] for 0 not in [b] (binary64)."""
    if np.any((b[0] <= 0) & (b[1] >= 0)):
        raise ZeroDivisionError("0 in divisor interval")
    one = np.ones_like(np.asarray(b[0], np.float64))
    return ir_mul(a, (div_rd(one, b[1]), div_ru(one, b[0])))


def ir_sqrt(a):
    if np.any(np.asarray(a[0]) < 0):
        raise ValueError("sqrt of an interval with a negative bound")
    return sqrt_rd(a[0]), sqrt_ru(a[1])


# ---- rectangular complex intervals (Section 2.5) ------------------------------
# A complex interval is a tuple (re_lo, re_hi, im_lo, im_hi) of arrays.

def ic_point(re, im=None):
    re = np.asarray(re, np.float64)
    im = np.zeros_like(re) if im is None else np.asarray(im, np.float64)
    return re, re.copy(), im, im.copy()


def ic_add(z, w, prec=F64):
    r = ir_add((z[0], z[1]), (w[0], w[1]), prec)
    i = ir_add((z[2], z[3]), (w[2], w[3]), prec)
    return r[0], r[1], i[0], i[1]


def ic_sub(z, w, prec=F64):
    r = ir_sub((z[0], z[1]), (w[0], w[1]), prec)
    i = ir_sub((z[2], z[3]), (w[2], w[3]), prec)
    return r[0], r[1], i[0], i[1]


def ic_mul(z, w, prec=F64):
    """(z1 w1 - z2 w2) + i (z1 w2 + z2 w1), all in real interval arithmetic."""
    z1, z2 = (z[0], z[1]), (z[2], z[3])
    w1, w2 = (w[0], w[1]), (w[2], w[3])
    re = ir_sub(ir_mul(z1, w1, prec), ir_mul(z2, w2, prec), prec)
    im = ir_add(ir_mul(z1, w2, prec), ir_mul(z2, w1, prec), prec)
    return re[0], re[1], im[0], im[1]


def ic_scale_pow2(z, k: int):
    """Division by 2^k: exact while no bound underflows."""
    s = 2.0 ** (-k)
    out = tuple(np.asarray(c, np.float64) * s for c in z)
    for c_in, c_out in zip(z, out):
        if np.any((np.asarray(c_in) != 0) & (np.abs(c_out) < 2.0 ** -1000)):
            raise FloatingPointError("scaling would underflow")
    return out


# ---- isolation (Section 1, Section 2.5) ---------------------------------------

ISOLATED, AMBIGUOUS, EMPTY, IMAG_EXCLUDES_ZERO = 0, 1, 2, 3


def isolate(re_lo, re_hi, im_lo, im_hi):
    """The unique integer in [re_lo, re_hi], with a per-element code.

    ISOLATED: exactly one integer k with re_lo <= k <= re_hi (closed ends),
    and im_lo <= 0 <= im_hi.  AMBIGUOUS: two or more integers.  EMPTY: none.
    IMAG_EXCLUDES_ZERO: the imaginary part cannot be zero.
    """
    re_lo = np.asarray(re_lo, np.float64)
    re_hi = np.asarray(re_hi, np.float64)
    k_lo = np.ceil(re_lo)
    k_hi = np.floor(re_hi)
    code = np.where(k_lo == k_hi, ISOLATED, np.where(k_lo < k_hi, AMBIGUOUS, EMPTY))
    code = np.where((np.asarray(im_lo) > 0) | (np.asarray(im_hi) < 0), IMAG_EXCLUDES_ZERO, code)
    val = np.where(code == ISOLATED, k_lo, 0.0)
    return val, code
