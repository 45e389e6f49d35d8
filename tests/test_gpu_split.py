"""Products cut into parts (SSMUL_OPT_SPLIT_DIGITS): past the isolation limit
of one transform, parts that isolate are combined by exact integer
coefficient sums.  Digits bit-exact against the oracle; a failing part makes
the whole product fail and zero-fill."""
import numpy as np
import pytest

import synth
from oracle import exact as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan  # noqa: E402

OK = abi.SSMUL_OK


def test_split_past_the_rectangle_limit():
    n = 1 << 20                      # fp64 rectangles alone fail here (width ~2.8)
    a, b = synth.operand_pair(synth.SEED_BASE + 21, n, n)
    with Plan(n, n) as p:
        s, r, z = p.mul(a, b)
        assert s == abi.SSMUL_ISOLATION_FAILED and not z.any()
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 1 << 18) == OK
        s, r, z = p.mul(a, b)
    assert s == OK, abi.status_string(s)
    assert r.max_width < 1.0
    assert np.array_equal(z, E.carry(E.conv_ntt(a, b), 2 * n))


@pytest.mark.parametrize("na,nb,m,balanced,prec", [
    (300001, 5000, 65536, 0, abi.SSMUL_PREC_FP64),
    (5000, 300001, 4096, 1, abi.SSMUL_PREC_DISC64),
    (70000, 70001, 20000, 1, abi.SSMUL_PREC_LADDER_DISC),
    (2048, 2049, 1024, 0, abi.SSMUL_PREC_FP64),
])
def test_split_parts_bit_exact(na, nb, m, balanced, prec):
    a, b = synth.operand_pair(synth.SEED_BASE + na + 7 * nb, na, nb)
    with Plan(na, nb, 0, prec) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, m) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_BALANCED, balanced) == OK
        s, r, z = p.mul(a, b)
        assert s == OK, abi.status_string(s)
        assert np.array_equal(z, E.product(a, b))
        zh = np.zeros(na + nb, np.uint8)                         # host-buffer call splits too
        s, r = abi.ssmul_mul_host(p.h, a.ctypes.data, na, b.ctypes.data, nb, zh.ctypes.data)
        assert s == OK and np.array_equal(zh, z)


def test_split_failure_is_reported():
    a, b = synth.operand_pair(synth.SEED_BASE + 5, 3000, 2500)
    with Plan(3000, 3000, 0, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 1024) == OK
        s, r, z = p.mul(a, b)
    assert s == abi.SSMUL_ISOLATION_FAILED and r.n_unisolated > 0
    assert not z.any()


def test_split_option_checks():
    with Plan(100, 100) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 10) == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 0) == OK


@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_LADDER])
def test_batched_split_mixed_with_small_products(prec):
    """A batch mixing products past the rectangles' limit (2^20 digits, cut
    into parts of 2^18) with small and mid-size ones: every product exact,
    through ssmul_mul_batched (twice: the part entries are reused) and
    ssmul_mul_batched_host, and a failing split product zero-fills alone."""
    import ctypes
    from tests.gpu_util import batched
    n = 1 << 20
    pairs = [synth.operand_pair(synth.SEED_BASE + 31, n, n),
             synth.operand_pair(synth.SEED_BASE + 32, 7, 9),
             synth.operand_pair(synth.SEED_BASE + 33, 300000, 1000),     # split along a only
             synth.operand_pair(synth.SEED_BASE + 34, 75000, 75000),
             synth.operand_pair(synth.SEED_BASE + 35, n, 5, "ff"),
             synth.operand_pair(synth.SEED_BASE + 36, 1, 1)]
    expect = [E.carry(E.conv_ntt(a, b), len(a) + len(b)) for a, b in pairs]
    with Plan(n, n, len(pairs), prec) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 1 << 18) == OK
        for _ in range(2):
            s, res, digits = batched(p, pairs)
            assert s == OK
            for r, z, e in zip(res, digits, expect):
                assert r.status == OK, abi.status_string(r.status)
                assert np.array_equal(z, e)
        # host pools in, host digits out
        na = [len(a) for a, _ in pairs]
        nb = [len(b) for _, b in pairs]
        a_pool, b_pool = np.concatenate([a for a, _ in pairs]), np.concatenate([b for _, b in pairs])
        a_off, b_off = np.cumsum([0] + na[:-1]), np.cumsum([0] + nb[:-1])
        nz = [x + y for x, y in zip(na, nb)]
        z_off = np.cumsum([0] + nz[:-1])
        zh = np.zeros(sum(nz), np.uint8)
        rh = (abi.ssmul_result * len(pairs))()
        descs = [(int(a_off[i]), int(b_off[i]), int(z_off[i]), na[i], nb[i]) for i in range(len(pairs))]
        assert abi.ssmul_mul_batched_host(p.h, descs, a_pool.ctypes.data, b_pool.ctypes.data,
                                          zh.ctypes.data, rh) == OK
        for i, e in enumerate(expect):
            assert rh[i].status == OK and np.array_equal(zh[z_off[i]:z_off[i] + nz[i]], e)
    # a split product whose parts cannot isolate fails alone, zero-filled
    bad = [synth.operand_pair(synth.SEED_BASE + 37, 3000, 2500), synth.operand_pair(38, 20, 20)]
    with Plan(3000, 3000, 2, abi.SSMUL_PREC_FP32) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_SPLIT_DIGITS, 1024) == OK
        s, res, digits = batched(p, bad)
        assert s == OK
        assert res[0].status == abi.SSMUL_ISOLATION_FAILED and not digits[0].any()
        assert res[1].status == OK and np.array_equal(digits[1], E.product(*bad[1]))
