"""Circular containment sets (SSMUL_PREC_DISC64) and the naive comparator
(SSMUL_PREC_NAIVE64) against the CPU oracle.

The disc primitives are checked with exact rational arithmetic: the result
disc must contain the exact result of the operation for points spread over
the operand discs (the containment property of Section 2.5, for the
circular sets of Section 4).
"""
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
# rational points of the closed unit disc
UNIT = [(Fr(0), Fr(0)), (Fr(1), Fr(0)), (Fr(-1), Fr(0)), (Fr(0), Fr(1)), (Fr(0), Fr(-1)),
        (Fr(3, 5), Fr(4, 5)), (Fr(-4, 5), Fr(3, 5)), (Fr(5, 13), Fr(-12, 13)), (Fr(-8, 17), Fr(-15, 17))]


def _rand_discs(rng, n, tw=False):
    if tw:
        ang = rng.uniform(0, 2 * np.pi, n)
        x, y = np.cos(ang), np.sin(ang)
        r = (np.abs(rng.standard_normal(n)) * 4e-16).astype(np.float32).astype(np.float64)
        x[:4], y[:4], r[:4] = [1, 0, -1, 0], [0, 1, 0, -1], 0
    else:
        x = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 7, n)
        y = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 7, n)
        r = (np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-14, -2, n)
             * (np.abs(x) + np.abs(y))).astype(np.float32).astype(np.float64)
        x[:3], y[:3], r[:3] = [0, 5, -3], [0, 0, 7], [0, 0, 1]
    return np.stack([x, y, r], 1)


def _disc_op(op, a, b):
    da, db = dev(a.ravel()), dev(b.ravel())
    out = torch.zeros_like(da)
    assert abi.ssmul_debug_disc_op(op, da.data_ptr(), db.data_ptr(), out.data_ptr(), len(a)) == OK
    return out.cpu().numpy().reshape(-1, 3)


def _contains(o, re, im):
    cx, cy, r = Fr(float(o[0])), Fr(float(o[1])), Fr(float(o[2]))
    return (re - cx) ** 2 + (im - cy) ** 2 <= r * r


@pytest.mark.parametrize("op", [0, 1, 2, 3, 5, 6])
def test_disc_ops_contain_exact_results(op):
    """ops 5, 6: products by the real and pure imaginary scalar discs of the
    radix-3 and radix-5 steps (the other centre component is 0)"""
    rng = np.random.default_rng(40 + op)
    a = _rand_discs(rng, 400)
    b = _rand_discs(rng, 400, tw=(op in (2, 5, 6)))
    if op in (5, 6):
        b[:, 1 if op == 5 else 0] = 0.0
        b[:, 2] = (np.abs(b[:, 0 if op == 5 else 1]) * 2.0 ** -50).astype(np.float32)
    out = _disc_op(op, a, b)
    for i in range(0, 400, 3):
        ax, ay, ar = (Fr(float(v)) for v in a[i])
        bx, by, br = (Fr(float(v)) for v in b[i])
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
                assert _contains(out[i], re, im), (op, i)


def test_disc_scale_contains():
    rng = np.random.default_rng(5)
    a = _rand_discs(rng, 200)
    k = np.full((200, 3), 0.0)
    k[:, 0] = rng.integers(0, 25, 200)
    out = _disc_op(4, a, k)
    for i in range(200):
        s = Fr(1, 2 ** int(k[i, 0]))
        ax, ay, ar = (Fr(float(v)) for v in a[i])
        for (p, q) in UNIT:
            assert _contains(out[i], (ax + ar * p) * s, (ay + ar * q) * s)


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 2), (17, 33), (1000, 1000), (2049, 2048),
                                   (16384, 16384), (65535, 3), (75000, 75000)])
def test_disc_products_bit_exact(na, nb):
    a, b = synth.operand_pair(synth.SEED_BASE + 7 * na + nb, na, nb)
    with Plan(na, nb, 0, abi.SSMUL_PREC_DISC64) as p:
        s, r, z = p.mul(a, b)
    assert s == OK, abi.status_string(s)
    assert r.precision_used == abi.SSMUL_PREC_DISC64
    assert np.array_equal(z, E.product(a, b))


@pytest.mark.parametrize("na,nb,dist", [(7, 9, "uniform"), (4096, 4096, "uniform"),
                                        (30000, 20000, "ff"), (75000, 75000, "uniform")])
def test_disc_intervals_contain_exact_and_are_narrower(na, nb, dist):
    a, b = synth.operand_pair(synth.SEED_BASE + na + nb, na, nb, dist)
    with Plan(na, nb) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, abi.SSMUL_PREC_DISC64)
        s2, r2, z2, lo2, hi2 = p.mul_intervals(a, b, abi.SSMUL_PREC_FP64)
    c = (E.conv(a, b) if na * nb < 1e9 else E.conv_ntt(a, b)).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi))
    assert s == OK and np.array_equal(z, E.product(a, b))
    # no wrapping under rotation: once the transforms are long enough for the
    # wrapping of rectangles to dominate, discs are narrower (for a handful
    # of digits the discs' half-ulp terms on both components can dominate)
    if na * nb >= 4096 * 4096:
        assert r.max_width <= r2.max_width


def test_naive_comparator():
    for na, nb in [(5, 5), (4096, 4096), (75000, 75000)]:
        a, b = synth.operand_pair(synth.SEED_BASE + 11, na, nb)
        with Plan(na, nb, 0, abi.SSMUL_PREC_NAIVE64) as p:
            s, r, z = p.mul(a, b)
        assert s == abi.SSMUL_UNVERIFIED and r.precision_used == abi.SSMUL_PREC_NAIVE64
        assert r.max_width < 0.5            # largest distance to the nearest integer
        assert np.array_equal(z, E.product(a, b))


def test_ladder_disc_rungs():
    with Plan(40000, 40000, 0, abi.SSMUL_PREC_LADDER_DISC) as p:
        for na, nb, prec in [(4, 5, abi.SSMUL_PREC_FP32), (300, 260, abi.SSMUL_PREC_DISC64),
                             (40000, 33333, abi.SSMUL_PREC_DISC64)]:
            a, b = synth.operand_pair(synth.SEED_BASE + na, na, nb)
            s, r, z = p.mul(a, b)
            assert s == OK and r.precision_used == prec
            assert np.array_equal(z, E.product(a, b))


@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_LADDER_DISC])
def test_batched_discs(prec):
    rng = np.random.default_rng(8)
    pairs = []
    for i in range(30):
        na, nb = (int(v) for v in np.exp(rng.uniform(0, np.log(50000), 2)).astype(int) + 1)
        pairs.append(synth.operand_pair(synth.SEED_BASE + 300 + i, na, nb))
    mx = max(max(len(a), len(b)) for a, b in pairs)
    with Plan(mx, mx, len(pairs), prec) as p:
        s, res, digits = batched(p, pairs)
    assert s == OK
    for (a, b), r, z in zip(pairs, res, digits):
        assert r.status == OK and np.array_equal(z, E.product(a, b))
