"""Seeded random batches across every verified precision rule, against the oracle.

Sizes are log-uniform in 1 .. 20,000 digits and independent for a and b;
operands are uniform, unconstrained ("raw", leading zero digits allowed),
all 0xFF, all zero, or sparse (a few nonzero digits).  Each batch runs
through ssmul_mul_batched, ssmul_mul_batched_host and one ssmul_mul per
product; every product must be SSMUL_OK with digits equal to the oracle's
exact product (Sections 2.1 and 2.4), and the three calls must agree on
every outcome.
"""
import ctypes

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
PRECS = [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_LADDER, abi.SSMUL_PREC_DISC64,
         abi.SSMUL_PREC_LADDER_DISC, abi.SSMUL_PREC_DISC32X2, abi.SSMUL_PREC_LADDER_FAST]
KINDS = ("uniform", "raw", "ff", "zero", "sparse")


def _operand(rng, seed, n, kind):
    if kind == "sparse":
        x = np.zeros(n, np.uint8)
        k = int(rng.integers(1, 5))
        x[rng.integers(0, n, k)] = rng.integers(1, 256, k)
        return x
    return synth.operand_pair(seed, n, 1, kind)[0]


def _random_pairs(seed, count):
    rng = np.random.default_rng(seed)
    pairs = []
    for i in range(count):
        na, nb = (int(v) for v in np.exp(rng.uniform(0.0, np.log(20000.0), 2)).astype(int))
        ka, kb = (KINDS[int(v)] for v in rng.integers(0, len(KINDS), 2))
        pairs.append((_operand(rng, synth.SEED_BASE + 5000 + 2 * i + seed, max(na, 1), ka),
                      _operand(rng, synth.SEED_BASE + 5001 + 2 * i + seed, max(nb, 1), kb)))
    return pairs


@pytest.mark.parametrize("prec", PRECS)
def test_random_batches_all_calls_agree_and_are_exact(prec):
    pairs = _random_pairs(prec + 1, 40)
    expect = [E.product(a, b) for a, b in pairs]
    mx = max(max(len(a), len(b)) for a, b in pairs)
    with Plan(mx, mx, len(pairs), prec) as p:
        s, res, digits = batched(p, pairs)
        assert s == OK
        for i, (r, z, e) in enumerate(zip(res, digits, expect)):
            assert r.status == OK, (i, abi.status_string(r.status))
            assert np.array_equal(z, e), i
        # host pools in, host digits out
        na = [len(a) for a, _ in pairs]
        nb = [len(b) for _, b in pairs]
        a_pool = np.concatenate([a for a, _ in pairs])
        b_pool = np.concatenate([b for _, b in pairs])
        a_off, b_off = np.cumsum([0] + na[:-1]), np.cumsum([0] + nb[:-1])
        nz = [x + y for x, y in zip(na, nb)]
        z_off = np.cumsum([0] + nz[:-1])
        zh = np.zeros(sum(nz), np.uint8)
        rh = (abi.ssmul_result * len(pairs))()
        descs = [(int(a_off[i]), int(b_off[i]), int(z_off[i]), na[i], nb[i]) for i in range(len(pairs))]
        assert abi.ssmul_mul_batched_host(p.h, descs, a_pool.ctypes.data, b_pool.ctypes.data,
                                          zh.ctypes.data, rh) == OK
        for i, e in enumerate(expect):
            assert rh[i].as_dict() == res[i].as_dict(), i
            assert np.array_equal(zh[z_off[i]:z_off[i] + nz[i]], e), i
        # one product per call
        for i, (a, b) in enumerate(pairs[:12]):
            s1, r1, z1 = p.mul(a, b)
            assert s1 == OK and np.array_equal(z1, expect[i]), i
            assert r1.precision_used == res[i].precision_used and r1.max_width == res[i].max_width, i
