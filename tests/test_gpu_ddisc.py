"""Discs with double-binary32 centres (SSMUL_PREC_DISC32X2) and the fast
ladder (SSMUL_PREC_LADDER_FAST) against exact rational arithmetic and the
CPU oracle.  A pair-disc operation must contain the exact result for points
spread over its operand discs; products must be bit-exact whenever the
status is SSMUL_OK, and a product that does not isolate must say so."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from oracle import exact as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan, batched, dev  # noqa: E402

OK = abi.SSMUL_OK
UNIT = [(Fr(0), Fr(0)), (Fr(1), Fr(0)), (Fr(-1), Fr(0)), (Fr(0), Fr(1)), (Fr(0), Fr(-1)),
        (Fr(3, 5), Fr(4, 5)), (Fr(-4, 5), Fr(3, 5)), (Fr(5, 13), Fr(-12, 13))]


def _pairs_of(v):
    h = v.astype(np.float32).astype(np.float64)
    lo = (v - h).astype(np.float32).astype(np.float64)
    return h, lo


def _rand(rng, n, tw=False):
    if tw:
        ang = rng.uniform(0, 2 * np.pi, n)
        x, y = np.cos(ang), np.sin(ang)
        r = np.full(n, 2.0 ** -46)
    else:
        x = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 8, n)
        y = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 8, n)
        r = (np.abs(x) + np.abs(y)) * 10.0 ** rng.integers(-13, -4, n)
        x[:3], y[:3], r[:3] = [0, 3, -7], [0, 0, 5], [0, 0, 1]
    xh, xl = _pairs_of(x)
    yh, yl = _pairs_of(y)
    r = r.astype(np.float32).astype(np.float64)
    return np.stack([xh, xl, yh, yl, r], 1)


def _op(op, a, b):
    da, db = dev(a.ravel()), dev(b.ravel())
    out = torch.zeros_like(da)
    assert abi.ssmul_debug_ddisc_op(op, da.data_ptr(), db.data_ptr(), out.data_ptr(), len(a)) == OK
    return out.cpu().numpy().reshape(-1, 5)


def _centre(row):
    return (Fr(float(row[0])) + Fr(float(row[1])), Fr(float(row[2])) + Fr(float(row[3])),
            Fr(float(row[4])))


@pytest.mark.parametrize("op", [0, 1, 2, 3, 7, 8])
def test_pair_disc_ops_contain_exact_results(op):
    """ops 7, 8: products by the real and pure imaginary scalar discs of the
    radix-3 and radix-5 steps (the other centre pair is 0)"""
    rng = np.random.default_rng(70 + op)
    a = _rand(rng, 300)
    b = _rand(rng, 300, tw=(op in (2, 7, 8)))
    if op in (7, 8):
        b[:, [2, 3] if op == 7 else [0, 1]] = 0.0
    out = _op(op, a, b)
    for i in range(0, 300, 3):
        ax, ay, ar = _centre(a[i])
        bx, by, br = _centre(b[i])
        ox, oy, orr = _centre(out[i])
        # results stay normalised pairs
        assert abs(out[i, 1]) <= 2.0 ** -24 * abs(out[i, 0]) and abs(out[i, 3]) <= 2.0 ** -24 * abs(out[i, 2])
        for (p, q) in UNIT[:5]:
            for (s, t) in UNIT[::2]:
                u = (ax + ar * p, ay + ar * q)
                v = (bx + br * s, by + br * t)
                if op == 0:
                    re, im = u[0] + v[0], u[1] + v[1]
                elif op == 1:
                    re, im = u[0] - v[0], u[1] - v[1]
                else:
                    re, im = u[0] * v[0] - u[1] * v[1], u[0] * v[1] + u[1] * v[0]
                assert (re - ox) ** 2 + (im - oy) ** 2 <= orr * orr, (op, i)


def test_pair_disc_scale_contains():
    rng = np.random.default_rng(6)
    a = _rand(rng, 100)
    k = np.zeros((100, 5))
    k[:, 0] = rng.integers(0, 26, 100)
    out = _op(4, a, k)
    for i in range(100):
        s = Fr(1, 2 ** int(k[i, 0]))
        ax, ay, ar = _centre(a[i])
        ox, oy, orr = _centre(out[i])
        for (p, q) in UNIT:
            re, im = (ax + ar * p) * s, (ay + ar * q) * s
            assert (re - ox) ** 2 + (im - oy) ** 2 <= orr * orr


@pytest.mark.parametrize("na,nb", [(1, 1), (2, 3), (31, 33), (1000, 999), (2049, 2048), (9000, 7000),
                                   (30000, 30000)])
def test_pair_disc_products(na, nb):
    a, b = synth.operand_pair(synth.SEED_BASE + 17 * na + nb, na, nb)
    with Plan(na, nb, 0, abi.SSMUL_PREC_DISC32X2) as p:
        s, r, z = p.mul(a, b)
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_BALANCED, 1) == OK
        s2, r2, z2 = p.mul(a, b)
    expect = E.product(a, b)
    for st, rr, zz in ((s, r, z), (s2, r2, z2)):
        assert st in (OK, abi.SSMUL_ISOLATION_FAILED), abi.status_string(st)
        if st == OK:
            assert rr.precision_used == abi.SSMUL_PREC_DISC32X2
            assert np.array_equal(zz, expect)
        else:
            assert not zz.any()
    if na * nb <= 9000 * 7000:
        assert s == OK                                  # well inside the rung's reach


@pytest.mark.parametrize("na,nb", [(300, 200), (4096, 4096), (20000, 20000)])
def test_pair_disc_intervals_contain_exact(na, nb):
    a, b = synth.operand_pair(synth.SEED_BASE + na, na, nb)
    with Plan(na, nb) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, abi.SSMUL_PREC_DISC32X2)
    c = E.conv(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi))
    assert r.n_empty == 0


def test_fast_ladder_escalates_and_stays_exact():
    pairs = [synth.operand_pair(synth.SEED_BASE + 800 + i, na, nb) for i, (na, nb) in
             enumerate([(5, 4), (300, 260), (5000, 6000), (75000, 75000), (200000, 150000)])]
    with Plan(200000, 200000, 8, abi.SSMUL_PREC_LADDER_FAST) as p:
        used = []
        for a, b in pairs:
            s, r, z = p.mul(a, b)
            assert s == OK, abi.status_string(s)
            assert np.array_equal(z, E.product(a, b))
            used.append(r.precision_used)
        assert used[0] == abi.SSMUL_PREC_FP32
        assert used[1] == abi.SSMUL_PREC_DISC32X2
        s, res, digits = batched(p, pairs)
        assert s == OK
        for (a, b), rr, zz, u in zip(pairs, res, digits, used):
            assert rr.status == OK and rr.precision_used == u
            assert np.array_equal(zz, E.product(a, b))


@pytest.mark.parametrize("op", [5, 6])
def test_pair_disc_butterfly_contains(op):
    """The radix-4 butterfly gives its four outputs one radius: every output
    must contain the exact butterfly of any points of the four input discs."""
    rng = np.random.default_rng(80 + op)
    n = 120
    x = np.stack([_rand(rng, 4) for _ in range(n)])          # (n, 4, 5)
    x[n // 2:, :, 4] = 0.0                                     # point inputs too
    dx = dev(x.ravel())
    out = torch.zeros_like(dx)
    assert abi.ssmul_debug_ddisc_op(op, dx.data_ptr(), 0, out.data_ptr(), n) == OK
    o = out.cpu().numpy().reshape(n, 4, 5)
    j = Fr(1) if op == 5 else Fr(-1)                            # SIGN
    for i in range(0, n, 2):
        ins = [_centre(x[i, t]) for t in range(4)]
        outs = [_centre(o[i, t]) for t in range(4)]
        assert len({float(q[2]) for q in outs}) == 1             # one shared radius
        for pick in range(6):
            pts = []
            for t, (cx, cy, cr) in enumerate(ins):
                p, q = UNIT[(pick + 2 * t) % len(UNIT)]
                pts.append((cx + cr * p, cy + cr * q))
            (ax, ay), (bx, by), (cx, cy), (dx_, dy) = pts
            # y_u = sum_t x_t (SIGN i)^{t u}
            ex = [(ax + bx + cx + dx_, ay + by + cy + dy),
                  (ax - j * by - cx + j * dy, ay + j * bx - cy - j * dx_),
                  (ax - bx + cx - dx_, ay - by + cy - dy),
                  (ax + j * by - cx - j * dy, ay - j * bx - cy + j * dx_)]
            for u in range(4):
                ox, oy, orr = outs[u]
                assert (ex[u][0] - ox) ** 2 + (ex[u][1] - oy) ** 2 <= orr * orr, (op, i, u)


def _f32(x):
    return np.float32(x)


def _normalised_low(rng, h, n):
    """low parts of magnitude up to half an ulp of h, each pair normalised
    (RN32(h + l) == h)"""
    ulp = np.spacing(np.abs(h).astype(np.float32)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    edge = rng.random(n) < 0.5                    # the extremes, just inside the tie
    lo[edge] = (np.sign(rng.uniform(-1, 1, edge.sum())) * ulp[edge] * (0.5 - 2.0 ** -20)).astype(np.float32)
    keep = (h.astype(np.float32) + lo).astype(np.float32) == h.astype(np.float32)
    return lo.astype(np.float64), keep


@pytest.mark.parametrize("op", [0, 1])
def test_pair_sum_exact_renormalisation_under_cancellation(op):
    """A pair sum ends with FastTwoSum(s, v), exact only when exp(s) >= exp(v).
    Operands whose high parts cancel (within a factor 2, across binade
    boundaries) with low parts at half an ulp are the case where |v| comes
    closest to |s|: the result must be exactly s + v (s, v as the rule
    computes them, emulated here in binary32), normalised, and contain the
    exact sum."""
    rng = np.random.default_rng(90 + op)
    n = 4000
    xh = rng.uniform(0.5, 4.0, n).astype(np.float32)
    f = np.where(rng.random(n) < 0.5, rng.uniform(0.5, 2.0, n),
                 1.0 + rng.integers(-4, 5, n) * 2.0 ** -23)            # near-total cancellation
    yh = (-(xh.astype(np.float64) * f)).astype(np.float32)
    if op == 1:
        yh = -yh                                                          # x - y cancels
    xh, yh = xh.astype(np.float64), yh.astype(np.float64)
    xl, k1 = _normalised_low(rng, xh, n)
    yl, k2 = _normalised_low(rng, yh, n)
    keep = k1 & k2
    xh, xl, yh, yl = xh[keep], xl[keep], yh[keep], yl[keep]
    m = len(xh)
    z = np.zeros(m)
    a = np.stack([xh, xl, z, z, z], 1)
    b = np.stack([yh, yl, z, z, z], 1)
    out = _op(op, a, b)
    sgn = 1.0 if op == 0 else -1.0
    for i in range(m):
        ah, al = _f32(xh[i]), _f32(xl[i])
        bh, bl = _f32(sgn * yh[i]), _f32(sgn * yl[i])
        s = _f32(ah + bh)
        bb = _f32(s - ah)
        e = _f32(_f32(ah - _f32(s - bb)) + _f32(bh - bb))
        v = _f32(e + _f32(al + bl))
        zh, zl = out[i, 0], out[i, 1]
        assert Fr(float(zh)) + Fr(float(zl)) == Fr(float(s)) + Fr(float(v)), i
        assert _f32(_f32(zh) + _f32(zl)) == _f32(zh)
        exact = Fr(float(xh[i])) + Fr(float(xl[i])) + Fr(sgn) * (Fr(float(yh[i])) + Fr(float(yl[i])))
        assert abs(exact - Fr(float(zh)) - Fr(float(zl))) <= Fr(float(out[i, 4])), i


def test_fast_ladder_escalates_part_of_one_length_group():
    """One transform length, some products escalating and some not: at 2^19
    digits the pair discs fail uniform operands and isolate all-0xFF ones,
    so the binary64 disc rung runs a list holding only the uniform products
    (the list's order is free; each product must come out exact under its
    own rung)."""
    n = 1 << 19
    dists = ["uniform", "ff", "uniform", "ff", "ff", "uniform"]
    pairs = [synth.operand_pair(synth.SEED_BASE + 950 + i, n, n, d) for i, d in enumerate(dists)]
    with Plan(n, n, len(pairs), abi.SSMUL_PREC_LADDER_FAST) as p:
        s, res, digits = batched(p, pairs)
    assert s == OK
    for (a, b), r, z, d in zip(pairs, res, digits, dists):
        assert r.status == OK, abi.status_string(r.status)
        want = abi.SSMUL_PREC_DISC32X2 if d == "ff" else abi.SSMUL_PREC_DISC64
        assert r.precision_used == want, (d, r.precision_used)
        assert np.array_equal(z, E.product(a, b))
