"""Balanced digits (SSMUL_OPT_BALANCED): the transforms carry a_j - 128 and
b_j - 128, and the isolated coefficients are corrected exactly by window sums
of the digits.  The product must not change: digits bit-exact against the
oracle, and every corrected enclosure must contain the exact coefficient."""
import numpy as np
import pytest

import synth
from oracle import exact as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan, batched  # noqa: E402

OK = abi.SSMUL_OK
PRECS = [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_FP32, abi.SSMUL_PREC_NAIVE64]


def _balanced_plan(na, nb, max_products=0, prec=abi.SSMUL_PREC_FP64):
    p = Plan(na, nb, max_products, prec)
    assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_BALANCED, 1) == OK
    return p


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("na,nb,dist", [(1, 1, "uniform"), (1, 9, "raw"), (5, 3, "ff"), (12, 12, "raw"),
                                        (2048, 2047, "uniform"), (2049, 5000, "uniform"),
                                        (4095, 1, "raw"), (40000, 40000, "ff"), (100000, 3001, "raw")])
def test_balanced_products_bit_exact(prec, na, nb, dist):
    a, b = synth.operand_pair(synth.SEED_BASE + 3 * na + nb, na, nb, dist)
    with _balanced_plan(na, nb, 0, prec) as p:
        s, r, z = p.mul(a, b)
    if prec == abi.SSMUL_PREC_FP32 and max(na, nb) > 12:
        # past binary32's isolation limit the failure is reported, never rounded
        assert s in (OK, abi.SSMUL_ISOLATION_FAILED), abi.status_string(s)
        if s != OK:
            assert not z.any()
            return
    expect = abi.SSMUL_UNVERIFIED if prec == abi.SSMUL_PREC_NAIVE64 else OK
    assert s == expect, abi.status_string(s)
    assert np.array_equal(z, E.product(a, b))


# binary32 rectangles at their measured isolation limits (squares, 8 uniform
# products per size drawn as the bench's limit search draws them): bytes
# 16 (all-0xFF 8), balanced bytes 30 (all-0xFF 16), 4-bit digits centred on
# their means 256 (all-0xFF: every size the 4-bit digits take, 1024)
@pytest.mark.parametrize("balanced,nibbles,n,dist", [
    (0, 0, 16, "uniform"), (0, 0, 8, "ff"), (1, 0, 30, "uniform"), (1, 0, 16, "ff"),
    (0, 1, 256, "uniform"), (0, 1, 1024, "ff"), (1, 1, 256, "uniform")])
def test_fp32_isolation_limits(balanced, nibbles, n, dist):
    with Plan(n, n, 0, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_BALANCED, balanced) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, nibbles) == OK
        for t in range(8 if dist == "uniform" else 1):
            a, b = synth.operand_pair(synth.SEED_BASE + 1000 * n + t, n, n, dist)
            s, r, z = p.mul(a, b)
            assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32, abi.status_string(s)
            assert np.array_equal(z, E.long_mul(a, b))


@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64])
def test_balanced_enclosures_contain_and_shrink(prec):
    na = nb = 75000
    a, b = synth.operand_pair(synth.SEED_BASE + 2, na, nb)
    with Plan(na, nb) as p:
        s0, r0, _, _, _ = p.mul_intervals(a, b, prec)
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_BALANCED, 1) == OK
        s1, r1, z1, lo, hi = p.mul_intervals(a, b, prec)
    c = E.conv_ntt(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi))
    assert s0 == OK and s1 == OK and np.array_equal(z1, E.product(a, b))
    assert r1.max_width < r0.max_width          # measured 1.75x (rectangles) at 75k


def test_balanced_zero_operand_and_batch():
    with _balanced_plan(3000, 3000, 30, abi.SSMUL_PREC_LADDER_DISC) as p:
        z0 = np.zeros(3000, np.uint8)
        a = synth.uniform_digits(5, 2999)
        s, r, z = p.mul(z0, a)
        assert s == OK and not z.any()
        rng = np.random.default_rng(2)
        pairs = []
        for i in range(25):
            na, nb = (int(v) for v in rng.integers(1, 3001, 2))
            pairs.append(synth.operand_pair(synth.SEED_BASE + 500 + i, na, nb,
                                            "ff" if i % 6 == 0 else "raw"))
        s, res, digits = batched(p, pairs)
        assert s == OK
        for (x, y), r, zz in zip(pairs, res, digits):
            assert r.status == OK and np.array_equal(zz, E.product(x, y))
