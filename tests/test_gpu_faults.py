"""Failure paths, with faults injected on the host (ssmul_debug_set_fault):
a rung that cannot isolate makes the ladder escalate; a failure at the last
rung is reported and the digits zero-filled; a carry tile that never
publishes makes the later tiles' bounded waits expire (SSMUL_TIMEOUT), and
the device stays usable afterwards.  Nothing faults or traps the GPU."""
import time

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


def test_fp32_rung_failure_escalates_to_fp64():
    a, b = synth.operand_pair(synth.SEED_BASE + 1, 4, 3)
    with Plan(100, 100, 0, abi.SSMUL_PREC_LADDER) as p:
        s, r, z = p.mul(a, b)
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32
        assert abi.ssmul_debug_set_fault(p.h, 1, 0) == OK
        s, r, z = p.mul(a, b)
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        assert np.array_equal(z, E.product(a, b))


def test_disc_rung_failure_escalates_to_rectangles():
    a, b = synth.operand_pair(synth.SEED_BASE + 2, 3000, 2000)
    with Plan(3000, 3000, 8, abi.SSMUL_PREC_LADDER_DISC) as p:
        assert abi.ssmul_debug_set_fault(p.h, 1, 2) == OK
        s, r, z = p.mul(a, b)
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        assert np.array_equal(z, E.product(a, b))
        pairs = [synth.operand_pair(synth.SEED_BASE + 10 + i, 3000 - 7 * i, 100 + i) for i in range(8)]
        s, res, digits = batched(p, pairs)
        assert s == OK
        for (x, y), rr, zz in zip(pairs, res, digits):
            assert rr.status == OK and rr.precision_used == abi.SSMUL_PREC_FP64
            assert np.array_equal(zz, E.product(x, y))


def test_last_rung_failure_is_reported_and_zero_filled():
    a, b = synth.operand_pair(synth.SEED_BASE + 3, 5000, 5000)
    with Plan(5000, 5000) as p:
        assert abi.ssmul_debug_set_fault(p.h, 1, 1) == OK
        s, r, z = p.mul(a, b)
        assert s == abi.SSMUL_ISOLATION_FAILED and r.n_unisolated > 0
        assert not z.any()
        assert abi.ssmul_debug_set_fault(p.h, 0) == OK
        s, r, z = p.mul(a, b)
        assert s == OK and np.array_equal(z, E.product(a, b))


def test_carry_lookback_wait_expires_with_status():
    a, b = synth.operand_pair(synth.SEED_BASE + 4, 6000, 6000)      # 12000 digits: 3 tiles
    with Plan(6000, 6000) as p:
        assert abi.ssmul_debug_set_fault(p.h, 2, 1) == OK          # tile 1 never publishes
        t0 = time.perf_counter()
        s, r, z = p.mul(a, b)
        elapsed = time.perf_counter() - t0
        assert s == abi.SSMUL_TIMEOUT
        assert not z.any()
        assert elapsed < 30.0                                       # a bounded wait
        assert abi.ssmul_debug_set_fault(p.h, 0) == OK              # the context still works
        s, r, z = p.mul(a, b)
        assert s == OK and np.array_equal(z, E.product(a, b))


def test_fault_argument_checks():
    with Plan(10, 10) as p:
        assert abi.ssmul_debug_set_fault(p.h, 1, 9) == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_debug_set_fault(p.h, 7, 0) == abi.SSMUL_INVALID_ARG
