"""The allocation-free entry point ssmul_mul_noalloc against ssmul_mul and the oracle.

Some callers cannot allocate device memory: their device memory is fully
reserved by another allocator, or they cannot accept the device
synchronisation an allocation may bring.  ssmul_mul_noalloc serves them from
one static device array.  This test calls it through the C ABI twice in a
row (so the second call runs on the array the first one left behind) and
checks digits, status and width against the plan-based ssmul_mul and the
digits against the CPU oracle; one more call runs on a stream other than
the default stream.
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


def _run_plan(a, b):
    plan = abi.ssmul_plan(len(a), len(b), 0, abi.SSMUL_PREC_FP64, 0)
    try:
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.full((len(a) + len(b),), 0x5A, dtype=torch.uint8, device="cuda")
        s, r = abi.ssmul_mul(plan, da.data_ptr(), len(a), db.data_ptr(), len(b), dz.data_ptr())
        return s, r, dz.cpu().numpy()
    finally:
        abi.ssmul_plan_destroy(plan)


def _run_noalloc(a, b, stream=None):
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dz = torch.full((len(a) + len(b),), 0x5A, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()           # the operands are on the device before a side stream reads them
    s, r = abi.ssmul_mul_noalloc(da.data_ptr(), len(a), db.data_ptr(), len(b), dz.data_ptr(),
                                 stream.cuda_stream if stream is not None else None)
    return s, r, dz.cpu().numpy()


def test_noalloc_matches_ssmul_mul_on_two_calls_in_a_row():
    cases = [synth.operand_pair(synth.SEED_BASE + 77, 2048, 2049),   # the largest allowed
             synth.operand_pair(synth.SEED_BASE + 78, 1000, 7)]      # smaller, on the stale array
    for a, b in cases:
        s0, r0, z0 = _run_plan(a, b)
        s1, r1, z1 = _run_noalloc(a, b)
        assert s0 == abi.SSMUL_OK and s1 == abi.SSMUL_OK
        assert np.array_equal(z1, z0)
        assert np.array_equal(z1, E.product(a, b))
        assert r1.status == r0.status and r1.fft_log2 == r0.fft_log2
        assert r1.n_unisolated == r0.n_unisolated == 0 and r1.n_empty == r0.n_empty == 0
        assert r1.max_width == r0.max_width


def test_noalloc_on_a_side_stream_and_edge_operands():
    stream = torch.cuda.Stream()
    cases = [synth.operand_pair(synth.SEED_BASE + 79, 3000, 1097),
             (np.full(2048, 0xFF, np.uint8), np.full(2049, 0xFF, np.uint8)),
             (np.zeros(5, np.uint8), synth.operand_pair(synth.SEED_BASE + 80, 5, 9)[1]),
             (np.array([255], np.uint8), np.array([255], np.uint8))]
    for a, b in cases:
        s, r, z = _run_noalloc(a, b, stream)
        assert s == abi.SSMUL_OK, abi.status_string(s)
        assert np.array_equal(z, E.product(a, b))
        s0, r0, z0 = _run_plan(a, b)
        assert r.max_width == r0.max_width and np.array_equal(z, z0)


def test_noalloc_rejects_sizes_beyond_its_limit():
    a = torch.zeros(4000, dtype=torch.uint8, device="cuda")
    b = torch.zeros(98, dtype=torch.uint8, device="cuda")
    z = torch.zeros(4098, dtype=torch.uint8, device="cuda")
    s, _ = abi.ssmul_mul_noalloc(a.data_ptr(), 4000, b.data_ptr(), 98, z.data_ptr())
    assert s == abi.SSMUL_TOO_LARGE
