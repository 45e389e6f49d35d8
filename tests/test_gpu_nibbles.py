"""Binary32 rectangles on 4-bit digits (SSMUL_OPT_FP32_NIBBLES) against the oracle.

The binary32 rung transforms the operands' base-16 digits and turns the
isolated base-16 coefficients into base-256 ones (c'_{2k} + 16 c'_{2k+1})
before the carry; a product with na + nb digits then has na + nb
coefficients, one more than its bytes give.  The transform carries each
operand's 4-bit digits minus their rounded mean, and the isolated
coefficients get the exact correction back.  Every product is compared bit
for bit with oracle.exact.product.
"""
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


def _sparse(seed, n, k):
    """n digits, all zero but k random positions and the top digit: few
    coefficients, exact in binary32 at any length."""
    rng = np.random.default_rng(seed)
    x = np.zeros(n, np.uint8)
    x[rng.integers(0, n, k)] = rng.integers(1, 256, k)
    x[n - 1] = 0xF7
    return x


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 7), (3, 2), (16, 16), (31, 33), (64, 64),
                                   (1, 1000), (1023, 2), (100, 1)])
def test_fp32_nibbles_exact_or_reported(na, nb):
    a, b = synth.operand_pair(synth.SEED_BASE + 40 + na, na, nb)
    with Plan(max(na, 64), max(nb, 64), 0, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 1) == OK
        s, r, z = p.mul(a, b)
    assert r.precision_used == abi.SSMUL_PREC_FP32 and r.n_empty == 0
    if s == OK:
        assert np.array_equal(z, E.product(a, b))
    else:
        assert s == abi.SSMUL_ISOLATION_FAILED and not z.any()


@pytest.mark.parametrize("na,nb", [(1, 1), (5, 4), (1024, 1024), (2047, 1), (1000, 1048)])
def test_fp32_nibbles_top_coefficient(na, nb):
    """Sparse operands isolate at any length, so the extra coefficient
    c'_{2(na+nb)-2} (the product of the top 4-bit digits) decides the top
    digits; lengths where 2 (na + nb) - 1 is just above a power of two."""
    a, b = _sparse(na, na, 3), _sparse(nb + 7, nb, 3)
    with Plan(2048, 2048, 0, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 1) == OK
        s, r, z = p.mul(a, b)
    assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32
    assert np.array_equal(z, E.product(a, b))


def test_ladder_with_nibbles_batched_and_single():
    """The ladder under 4-bit binary32 digits: small products resolve in
    binary32, larger ones escalate to binary64; batched and one at a time."""
    pairs = [synth.operand_pair(synth.SEED_BASE + 60 + i, n, m)
             for i, (n, m) in enumerate([(2, 3), (20, 20), (40, 40), (64, 60), (200, 200),
                                         (700, 900), (1500, 500), (3000, 2000)])]
    pairs.append((_sparse(1, 1024, 4), _sparse(2, 1024, 4)))
    with Plan(3000, 3000, len(pairs), abi.SSMUL_PREC_LADDER) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 1) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_MAX_DIGITS, 2048) == OK
        s, res, digits = batched(p, pairs)
        assert s == OK
        for (a, b), r, z in zip(pairs, res, digits):
            assert r.status == OK and np.array_equal(z, E.product(a, b))
        assert res[0].precision_used == abi.SSMUL_PREC_FP32
        assert res[-1].precision_used == abi.SSMUL_PREC_FP32
        assert res[7].precision_used == abi.SSMUL_PREC_FP64
        for (a, b), rb in zip(pairs, res):
            s1, r1, z1 = p.mul(a, b)
            assert s1 == OK and np.array_equal(z1, E.product(a, b))
            assert r1.precision_used == rb.precision_used


def test_split_parts_in_nibbles():
    """Parts of a split product decided by binary32 on 4-bit digits hand the
    parent one more coefficient each; the parent's carry takes them all."""
    a, b = _sparse(3, 3000, 6), _sparse(4, 2500, 6)
    with Plan(3000, 3000, 0, abi.SSMUL_PREC_LADDER) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 1) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_MAX_DIGITS, 2048) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 1024) == OK
        s, r, z = p.mul(a, b)
    assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32
    assert np.array_equal(z, E.product(a, b))


def _nibbles(x):
    """The base-16 digits of a base-256 digit vector (low half first)."""
    x = np.asarray(x, np.uint8)
    return np.stack([x & 15, x >> 4], axis=1).reshape(-1)


@pytest.mark.parametrize("na,nb,dist", [(1, 1, "uniform"), (5, 7, "uniform"), (100, 90, "ff"),
                                        (231, 231, "uniform"), (256, 256, "uniform"),
                                        (1024, 1024, "ff"), (1024, 1, "uniform"), (40, 41, "raw")])
def test_nibble_intervals_contain_exact(na, nb, dist):
    """Every binary32 set of a 4-bit-digit coefficient contains the exact
    c'_i of the oracle's convolution of the 4-bit digit vectors, and those
    coefficients give the product: sum_i c'_i 16^i = a b."""
    a, b = synth.operand_pair(synth.SEED_BASE + 90 + na, na, nb, dist)
    na4, nb4 = _nibbles(a), _nibbles(b)
    c4 = E.conv(na4, nb4)
    assert sum(int(c) << (4 * i) for i, c in enumerate(c4)) == E.to_int(a) * E.to_int(b)
    with Plan(na, nb, 0, abi.SSMUL_PREC_FP32) as p:
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(na + nb, dtype=torch.uint8, device="cuda")
        lp = 2 * (na + nb) - 1
        div = torch.zeros(2 * lp, dtype=torch.float64, device="cuda")
        s, r = abi.ssmul_debug_mul_intervals(p.h, da.data_ptr(), na, db.data_ptr(), nb,
                                             dz.data_ptr(), abi.SSMUL_DEBUG_PREC_FP32_NIBBLES,
                                             div.data_ptr())
        iv = div.cpu().numpy().reshape(lp, 2)
    assert r.n_empty == 0 and r.fft_log2 == max(2, (lp - 1).bit_length())
    c = c4.astype(np.float64)
    assert np.all((iv[:, 0] <= c) & (c <= iv[:, 1]))
    if s == OK:
        assert np.array_equal(dz.cpu().numpy(), E.product(a, b))


def _interval_check(a, b):
    """The 4-bit-digit sets of one product contain the oracle's c'_i; returns
    the product's status and digits."""
    na, nb = len(a), len(b)
    c4 = E.conv(_nibbles(a), _nibbles(b)).astype(np.float64)
    with Plan(na, nb, 0, abi.SSMUL_PREC_FP32) as p:
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(na + nb, dtype=torch.uint8, device="cuda")
        lp = 2 * (na + nb) - 1
        div = torch.zeros(2 * lp, dtype=torch.float64, device="cuda")
        s, r = abi.ssmul_debug_mul_intervals(p.h, da.data_ptr(), na, db.data_ptr(), nb,
                                             dz.data_ptr(), abi.SSMUL_DEBUG_PREC_FP32_NIBBLES,
                                             div.data_ptr())
        iv = div.cpu().numpy().reshape(lp, 2)
    assert r.n_empty == 0
    assert np.all((iv[:, 0] <= c4) & (c4 <= iv[:, 1]))
    return s, dz.cpu().numpy()


@pytest.mark.parametrize("case", ["uniform_sparse", "ff_zero", "ff_uniform", "zero_zero",
                                  "sparse_ff", "one_digit_ff"])
def test_nibbles_operands_of_different_means(case):
    """Each operand is centred on its own mean (0 for sparse and zero
    operands, 15 for all-0xFF, about 8 for uniform digits): pairs of
    different means isolate, stay exact and keep the sets around c'_i."""
    seed = synth.SEED_BASE + 700
    n = 200
    ops = {
        "uniform": synth.operand_pair(seed, n, 1)[0],
        "sparse": _sparse(seed + 1, n, 5),
        "ff": np.full(n, 0xFF, np.uint8),
        "zero": np.zeros(n, np.uint8),
    }
    if case == "one_digit_ff":
        a, b = np.array([0xFF], np.uint8), np.full(1023, 0xFF, np.uint8)
    else:
        ka, kb = case.split("_")
        a, b = ops[ka], ops[kb]
    s, z = _interval_check(a, b)
    assert s == OK
    assert np.array_equal(z, E.product(a, b))


def test_nibble_export_needs_the_option():
    """The 4-bit export is refused on a plan whose binary32 rung transforms
    bytes (its launches have no room for the 4-bit transform)."""
    a, b = synth.operand_pair(synth.SEED_BASE + 710, 50, 50)
    with Plan(50, 50, 0, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 0) == OK
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(100, dtype=torch.uint8, device="cuda")
        div = torch.zeros(2 * 199, dtype=torch.float64, device="cuda")
        s, _ = abi.ssmul_debug_mul_intervals(p.h, da.data_ptr(), 50, db.data_ptr(), 50,
                                             dz.data_ptr(), abi.SSMUL_DEBUG_PREC_FP32_NIBBLES,
                                             div.data_ptr())
    assert s == abi.SSMUL_INVALID_ARG
