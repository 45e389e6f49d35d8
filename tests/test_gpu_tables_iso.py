"""Two properties of the transform internals, checked through the debug ABI.

1. The step-ordered twiddle tables hold copies of the octant table's values
   (moved by exact symmetries), so every rung's enclosures are the same bits
   whichever table the transforms read.
2. The double-binary32 disc rung decides a coefficient (Section 1: exactly
   one integer in the enclosure) with binary32 and integer operations.  Its
   decision must be sound against exact rational arithmetic on the set
   [h + l - r, h + l + r]: an accepted integer is the only one the set holds
   (up to the decision's own rounding slack, which can only widen the set),
   a set holding two integers is never accepted, and NaN, infinite parts and
   negative values are rejected.  The binary64 decision of the same set is
   held to the same rules.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan, dev  # noqa: E402

OK = abi.SSMUL_OK
RUNGS = [abi.SSMUL_PREC_FP32, abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64,
         abi.SSMUL_PREC_DISC32X2, abi.SSMUL_PREC_NAIVE64]


@pytest.mark.parametrize("na,nb", [(300, 200), (3000, 2500), (40000, 30000)])
def test_step_tables_give_octant_bits(na, nb):
    a, b = synth.operand_pair(synth.SEED_BASE + 900 + na, na, nb)
    with Plan(na, nb) as p:
        for prec in RUNGS:
            s1, r1, z1, lo1, hi1 = p.mul_intervals(a, b, prec)
            assert abi.ssmul_debug_set_fault(p.h, 3, 1) == OK
            s2, r2, z2, lo2, hi2 = p.mul_intervals(a, b, prec)
            assert abi.ssmul_debug_set_fault(p.h, 0) == OK
            assert s1 == s2, prec
            assert r1.max_width == r2.max_width or (math.isnan(r1.max_width) and math.isnan(r2.max_width))
            assert np.array_equal(lo1.view(np.uint64), lo2.view(np.uint64)), prec
            assert np.array_equal(hi1.view(np.uint64), hi2.view(np.uint64)), prec
            assert np.array_equal(z1, z2)


# ---- isolation ----------------------------------------------------------------

F32 = np.float32
INF = float("inf")
NAN = float("nan")


def _f32(x) -> float:
    return float(F32(x))


def _pair(c: Fr):
    h = _f32(float(c))
    return h, _f32(float(c - Fr(h)))


def _cases(seed: int, R: int = 1):
    """(h, l, r, pad) rows: crafted edges first, then seeded random sets
    (R = 3, 5: mostly around R times an integer, radii times R)."""
    rows = [
        (0.0, 0.0, 0.0, 0), (5.0, 0.0, 0.0, 0), (-5.0, 0.0, 0.0, 0), (-5.0, 0.0, 0.1, 0),
        (0.25, 0.0, 0.25, 0), (0.5, 0.0, 0.5, 0), (7.5, 0.0, 0.5, 0), (7.5, 0.0, 0.49, 0),
        (2.0 ** 30, 0.0, 0.4, 0), (2.0 ** 30, 3.0, 0.4, 0), (2.0 ** 40, -17.0, 0.2, 0),
        (2.0 ** 60, 0.0, 1.0, 0), (2.0 ** 60, 0.0, 2.0 ** 30, 0), (3.0, 0.0, 2.0 ** 25, 0),
        (3.0, 0.0, INF, 0), (NAN, 0.0, 0.1, 0), (3.0, NAN, 0.1, 0), (3.0, 0.0, NAN, 0),
        (INF, 0.0, 0.1, 0), (-INF, 0.0, 0.1, 0), (3.0, INF, 0.1, 0),
        (0.0, 0.0, 0.1, 1), (0.3, 0.0, 0.2, 1), (0.3, 0.0, 0.4, 1), (3.0, 0.0, 0.1, 1),
        (3.0, 0.0, 10.0, 1), (2.0 ** 30, 0.0, 2.0 ** 25, 1), (2.0 ** 30, 0.0, 2.0 ** 31, 1),
        (2.0 ** 60, 0.0, 1.0, 1), (NAN, 0.0, 0.1, 1), (3.0, 0.0, INF, 1), (INF, 0.0, 1.0, 1),
    ]
    rng = np.random.default_rng(seed)
    radii = [0.0, 1e-7, 0.01, 0.3, 0.49, 0.5, 0.51, 1.0, 2.5]
    for _ in range(4000):
        mag = int(rng.choice([0, 4, 10, 20, 30, 40, 45, 50]))
        k = int(rng.integers(0, 2 ** mag + 1)) * (1 if rng.random() < 0.9 else -1)
        k *= R if rng.random() < 0.85 else 1
        off = Fr(int(rng.integers(-7000, 7001)) * R, 10000)
        h, l = _pair(Fr(k) + off)
        r = _f32(R * rng.choice(radii) * (1.0 if rng.random() < 0.7 else rng.random()))
        rows.append((h, l, r, int(rng.random() < 0.1)))
    return rows


def _run(path, rows):
    x = np.array(rows, np.float64)
    dx = dev(x.ravel())
    dv = torch.zeros(len(rows), dtype=torch.int64, device="cuda")
    dc = torch.zeros(len(rows), dtype=torch.int32, device="cuda")
    assert abi.ssmul_debug_isolate(path, dx.data_ptr(), dv.data_ptr(), dc.data_ptr(), len(rows)) == OK
    return dv.cpu().numpy(), dc.cpu().numpy()


def _ceil(q: Fr) -> int:
    return -((-q.numerator) // q.denominator)


def _floor(q: Fr) -> int:
    return q.numerator // q.denominator


def _check(row, value, cls, slack, R=1):
    """R = 3, 5: the set encloses R c, and the decision is on it divided by R"""
    h, l, r, pad = row
    if math.isnan(h) or math.isnan(l) or math.isnan(r) or math.isinf(h) or math.isinf(l):
        assert cls == 2, row
        return
    if math.isinf(r):
        assert cls == (0 if pad else 1), row
        return
    c = Fr(h) + Fr(l)
    lo, hi = (c - Fr(r)) / R, (c + Fr(r)) / R
    d = Fr(slack(c, r))
    wlo, whi = lo - d / R, hi + d / R               # the decision's set lies inside this one
    if pad:
        if lo <= 0 <= hi:
            assert cls == 0, row                    # contains 0: never reported empty
        elif not (wlo <= 0 <= whi):
            assert cls == 2, row                    # excludes 0 beyond the slack
        return
    ints = _floor(hi) - _ceil(lo) + 1
    wints = _floor(whi) - _ceil(wlo) + 1
    if cls == 0:
        assert wints >= 1 and _ceil(wlo) <= value <= _floor(whi), row
        assert value >= 0 and abs(c) < 2 ** 53, row
        assert ints <= 1, row                       # never accepts a set with two integers
    elif cls == 1:
        assert wints >= 2, row                      # not isolated only when the set is wide
    else:
        # empty: no integer, a negative one, or a centre past 2^53
        assert ints == 0 or (ints == 1 and _ceil(lo) < 0) or abs(c) >= 2 ** 52, row
    if ints == 1 and wints == 1 and _ceil(lo) >= 0 and abs(c) < 2 ** 52:
        assert cls == 0 and value == _ceil(lo), row  # clear cases are decided
    if ints >= 2 and abs(c) < 2 ** 52:
        assert cls == 1, row


def _exact_isolated(row, R):
    """the exact set [c - r, c + r] / R holds exactly one integer, >= 0, and
    its centre is below 2^52"""
    h, l, r, pad = row
    if pad or any(math.isnan(v) or math.isinf(v) for v in (h, l, r)):
        return False
    c = Fr(h) + Fr(l)
    lo, hi = (c - Fr(r)) / R, (c + Fr(r)) / R
    return _floor(hi) == _ceil(lo) and _ceil(lo) >= 0 and abs(c) < 2 ** 52


def _slack32(c, r):
    return 2.0 ** -22 * (1.0 + r)


def _slack64(c, r):
    return 2.0 ** -50 * (abs(float(c)) + r + 1.0)


@pytest.mark.parametrize("R", [1, 3, 5])
def test_pair_disc_isolation_is_sound(R):
    """R = 3, 5: the decisions of the transform lengths 3 2^k and 5 2^k,
    on sets around R times an integer (and plain ones, mostly empty)"""
    rows = _cases(1234 + R, R)
    path = {1: 0, 3: 2, 5: 4}[R]
    v32, c32 = _run(path, rows)
    v64, c64 = _run(path + 1, rows)
    for i, row in enumerate(rows):
        _check(row, int(v32[i]), int(c32[i]), _slack32, R)
        _check(row, int(v64[i]), int(c64[i]), _slack64, R)
        if c32[i] == 0 and c64[i] == 0:
            assert v32[i] == v64[i], row
    # both decide nearly every set that holds exactly one integer (one
    # multiple of R): the binary32 path works relative to the integer part,
    # the binary64 bounds of a centre near 2^52 round to the nearest half
    exact = np.array([_exact_isolated(row, R) for row in rows])
    assert np.sum(exact & (c32 == 0)) >= 0.99 * np.sum(exact)
    assert np.sum(exact & (c64 == 0)) >= 0.98 * np.sum(exact)


def test_scaled_floor_ceil_exact():
    """floor and ceil of x 2^-k, the 1/N scaling folded into the isolation's
    integer conversion: exact for every binary64 class (normal, subnormal,
    zero of either sign, huge, inf, NaN)"""
    rng = np.random.default_rng(99)
    n = 6000
    mant = rng.uniform(1.0, 2.0, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    ex = rng.integers(-80, 80, n)
    x = np.ldexp(mant, ex)
    k = rng.integers(0, 64, n).astype(np.int32)
    # integers and half-integers after scaling, ties, and the special classes
    x[:400] = np.ldexp(np.round(x[:400]), k[:400].astype(int))
    x[400:800] = np.ldexp(np.floor(x[400:800]) + 0.5, k[400:800].astype(int))
    special = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, -1e-310, 1.0, -1.0,
               2.0 ** 52, 2.0 ** 53 + 2, -(2.0 ** 61), 2.0 ** 62, 2.0 ** 70, -(2.0 ** 80),
               1.7976931348623157e308, math.inf, -math.inf, math.nan]
    x[800:800 + len(special)] = special
    k[800:800 + len(special)] = [0, 0, 0, 3, 1, 5, 0, 0, 0, 0, 0, 0, 0, 0, 1023, 0, 0, 0]
    x[900:910] = [3.0] * 10
    k[900:910] = [0, 1, 2, 60, 61, 62, 63, 64, 100, 1023]
    dx = dev(x)
    dk = torch.from_numpy(k).cuda()
    out = torch.zeros(2 * n, dtype=torch.int64, device="cuda")
    assert abi.ssmul_debug_floor_ceil(dx.data_ptr(), dk.data_ptr(), out.data_ptr(), n) == OK
    o = out.cpu().numpy().reshape(n, 2)
    cap = 2 ** 62
    for i in range(n):
        if math.isnan(x[i]):
            assert o[i, 0] == o[i, 1] == -(2 ** 63)
            continue
        if math.isinf(x[i]):
            assert o[i, 0] == o[i, 1] == (cap if x[i] > 0 else -cap)
            continue
        q = Fr(float(x[i])) / 2 ** int(k[i])
        fl, ce = _floor(q), _ceil(q)
        want = (max(-cap, min(cap, fl)), max(-cap, min(cap, ce)))
        assert (int(o[i, 0]), int(o[i, 1])) == want, (i, x[i], k[i])
