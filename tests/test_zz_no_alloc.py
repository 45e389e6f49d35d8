"""The allocation-free entry point ssmul_mul_noalloc against ssmul_mul.

Some callers cannot allocate device memory: their device memory is fully
reserved by another allocator, or they cannot accept the device
synchronisation an allocation may bring.  ssmul_mul_noalloc serves them from
one static device array.  This test calls it through the C ABI twice in a
row (so the second call runs on the array the first one left behind) and
checks digits, status and width against the plan-based ssmul_mul.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402


def _run_plan(a, b):
    plan = abi.ssmul_plan(len(a), len(b), 0, abi.SSMUL_PREC_FP64, 0)
    try:
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.full((len(a) + len(b),), 0x5A, dtype=torch.uint8, device="cuda")
        s, r = abi.ssmul_mul(plan, da.data_ptr(), len(a), db.data_ptr(), len(b), dz.data_ptr())
        return s, r, dz.cpu().numpy()
    finally:
        abi.ssmul_plan_destroy(plan)


def _run_noalloc(a, b):
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dz = torch.full((len(a) + len(b),), 0x5A, dtype=torch.uint8, device="cuda")
    s, r = abi.ssmul_mul_noalloc(da.data_ptr(), len(a), db.data_ptr(), len(b), dz.data_ptr())
    return s, r, dz.cpu().numpy()


def test_noalloc_matches_ssmul_mul_on_two_calls_in_a_row():
    cases = [synth.operand_pair(synth.SEED_BASE + 77, 2048, 2049),   # the largest allowed
             synth.operand_pair(synth.SEED_BASE + 78, 1000, 7)]      # smaller, on the stale array
    for a, b in cases:
        s0, r0, z0 = _run_plan(a, b)
        s1, r1, z1 = _run_noalloc(a, b)
        assert s0 == abi.SSMUL_OK and s1 == abi.SSMUL_OK
        assert np.array_equal(z1, z0)
        assert r1.status == r0.status and r1.fft_log2 == r0.fft_log2
        assert r1.n_unisolated == r0.n_unisolated == 0 and r1.n_empty == r0.n_empty == 0
        assert r1.max_width == r0.max_width


def test_noalloc_rejects_sizes_beyond_its_limit():
    a = torch.zeros(4000, dtype=torch.uint8, device="cuda")
    b = torch.zeros(98, dtype=torch.uint8, device="cuda")
    z = torch.zeros(4098, dtype=torch.uint8, device="cuda")
    s, _ = abi.ssmul_mul_noalloc(a.data_ptr(), 4000, b.data_ptr(), 98, z.data_ptr())
    assert s == abi.SSMUL_TOO_LARGE
