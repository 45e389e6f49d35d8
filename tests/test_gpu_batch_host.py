"""ssmul_mul_batched_host: host pools in, host digits out, against the CPU oracle.

The call copies the operands to the device, runs the batch in pieces whose
copies overlap the computation, and copies every product's digits
(Section 2.4's carry) and outcome back.  Every product here is compared
bit for bit with oracle.exact.product.
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

SENTINEL = 0xA5


def _mixed_pairs():
    """Uneven sizes over the single-CTA and four-step lengths, the worst
    case (all 0xFF), zero operands, one-digit operands and an unbalanced pair."""
    pairs = []
    seed = synth.SEED_BASE + 900
    for k, (na, nb) in enumerate([(1, 1), (1, 3000), (7, 5), (300, 300), (2048, 2049),
                                  (5000, 4000), (20000, 1), (40000, 35000), (75000, 75000)]):
        pairs.append(synth.operand_pair(seed + k, na, nb))
    pairs.append(synth.operand_pair(seed + 50, 6000, 6000, "ff"))
    pairs.append(synth.operand_pair(seed + 51, 75000, 75000, "ff"))
    pairs.append((np.zeros(4096, np.uint8), synth.operand_pair(seed + 52, 4096, 10)[0]))
    pairs.append((np.zeros(1, np.uint8), np.zeros(1, np.uint8)))
    pairs.append((np.array([255], np.uint8), np.array([255], np.uint8)))
    pairs.append(synth.operand_pair(seed + 53, 1 << 12, 1 << 17))
    return pairs


def _layout(pairs, gap=0, reverse=False):
    """Pools with `gap` unused bytes after every range; reverse: the
    descriptors list the products in the opposite order of their offsets."""
    a_parts, b_parts, descs = [], [], []
    ao = bo = zo = 0
    for a, b in pairs:
        descs.append((ao, bo, zo, len(a), len(b)))
        a_parts += [a, np.full(gap, 0x11, np.uint8)]
        b_parts += [b, np.full(gap, 0x22, np.uint8)]
        ao += len(a) + gap
        bo += len(b) + gap
        zo += len(a) + len(b) + gap
    if reverse:
        descs = descs[::-1]
    return np.concatenate(a_parts), np.concatenate(b_parts), zo, descs


def _run(plan, a_pool, b_pool, nz_total, descs, pinned):
    if pinned:
        ha = torch.from_numpy(a_pool).pin_memory()
        hb = torch.from_numpy(b_pool).pin_memory()
        hz = torch.full((nz_total,), SENTINEL, dtype=torch.uint8).pin_memory()
        pa, pb, pz = ha.data_ptr(), hb.data_ptr(), hz.data_ptr()
        z = hz.numpy()
    else:
        ha, hb = np.ascontiguousarray(a_pool), np.ascontiguousarray(b_pool)
        z = np.full(nz_total, SENTINEL, np.uint8)
        pa, pb, pz = ha.ctypes.data, hb.ctypes.data, z.ctypes.data
    res = (abi.ssmul_result * len(descs))()
    s = abi.ssmul_mul_batched_host(plan, descs, pa, pb, pz, res)
    return s, list(res), z.copy()


def _check(pairs, descs, res, z, reverse, gap):
    order = list(range(len(pairs)))[::-1] if reverse else list(range(len(pairs)))
    covered = np.zeros(len(z), bool)
    for slot, i in enumerate(order):
        a, b = pairs[i]
        zo = descs[slot][2]
        nz = len(a) + len(b)
        assert res[slot].status == abi.SSMUL_OK, (i, abi.status_string(res[slot].status))
        assert np.array_equal(z[zo:zo + nz], E.product(a, b)), i
        covered[zo:zo + nz] = True
    # nothing outside the products' ranges was written
    assert np.all(z[~covered] == SENTINEL)
    if gap:
        assert (~covered).sum() == gap * len(pairs)


@pytest.mark.parametrize("pieces,pinned,gap,reverse", [
    (1, True, 0, False), (2, True, 0, False), (3, False, 0, False), (7, True, 5, True),
    (16, False, 3, False)])
def test_host_batch_matches_oracle(pieces, pinned, gap, reverse):
    pairs = _mixed_pairs()
    a_pool, b_pool, nz_total, descs = _layout(pairs, gap, reverse)
    max_n = max(max(len(a), len(b)) for a, b in pairs)
    plan = abi.ssmul_plan(max_n, max_n, len(pairs), abi.SSMUL_PREC_FP64, 0)
    try:
        assert abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_HOST_PIECES, pieces) == abi.SSMUL_OK
        for _ in range(2):             # the second call reuses the grown device buffers
            s, res, z = _run(plan, a_pool, b_pool, nz_total, descs, pinned)
            assert s == abi.SSMUL_OK, abi.status_string(s)
            _check(pairs, descs, res, z, reverse, gap)
    finally:
        abi.ssmul_plan_destroy(plan)


def test_host_batch_equals_device_batch_under_the_ladder():
    """Same outcomes (status, deciding rung, width) as ssmul_mul_batched on
    device pools, on a plan stream other than the default stream."""
    pairs = _mixed_pairs()
    a_pool, b_pool, nz_total, descs = _layout(pairs)
    max_n = max(max(len(a), len(b)) for a, b in pairs)
    stream = torch.cuda.Stream()
    plan = abi.ssmul_plan(max_n, max_n, len(pairs), abi.SSMUL_PREC_LADDER, stream.cuda_stream)
    try:
        s, res_h, z_h = _run(plan, a_pool, b_pool, nz_total, descs, True)
        assert s == abi.SSMUL_OK
        da, db = torch.from_numpy(a_pool).cuda(), torch.from_numpy(b_pool).cuda()
        dz = torch.zeros(nz_total, dtype=torch.uint8, device="cuda")
        res_d = (abi.ssmul_result * len(pairs))()
        dres = torch.zeros(ctypes.sizeof(res_d), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()       # the pools are on the device before the plan's stream reads them
        with torch.cuda.stream(stream):
            assert abi.ssmul_mul_batched(plan, descs, da.data_ptr(), db.data_ptr(), dz.data_ptr(),
                                         dres.data_ptr()) == abi.SSMUL_OK
        stream.synchronize()
        host = dres.cpu().numpy()      # held: memmove reads its memory
        ctypes.memmove(res_d, host.ctypes.data, ctypes.sizeof(res_d))
        assert np.array_equal(dz.cpu().numpy(), z_h)
        for rh, rd in zip(res_h, res_d):
            assert rh.as_dict() == rd.as_dict()
        _check(pairs, descs, res_h, z_h, False, 0)
    finally:
        abi.ssmul_plan_destroy(plan)


def test_host_batch_zero_fills_a_failed_product():
    """A product the plan cannot isolate (binary32 rectangles at 2000 digits)
    comes back zero-filled with its failure status; the others are exact."""
    pairs = [synth.operand_pair(synth.SEED_BASE + 960, 8, 8),
             synth.operand_pair(synth.SEED_BASE + 961, 2000, 2000)]
    a_pool, b_pool, nz_total, descs = _layout(pairs)
    plan = abi.ssmul_plan(2000, 2000, 2, abi.SSMUL_PREC_FP32, 0)
    try:
        s, res, z = _run(plan, a_pool, b_pool, nz_total, descs, True)
        assert s == abi.SSMUL_OK
        assert res[0].status == abi.SSMUL_OK
        assert np.array_equal(z[:16], E.product(*pairs[0]))
        assert res[1].status == abi.SSMUL_ISOLATION_FAILED
        assert np.all(z[16:] == 0)
    finally:
        abi.ssmul_plan_destroy(plan)


def test_host_batch_argument_errors():
    plan = abi.ssmul_plan(100, 100, 2, abi.SSMUL_PREC_FP64, 0)
    try:
        a = np.ones(100, np.uint8)
        z = np.zeros(200, np.uint8)
        res = (abi.ssmul_result * 3)()
        d = [(0, 0, 0, 100, 100)]
        L = abi.load()
        arr = (abi.ssmul_desc * 1)(abi.ssmul_desc(0, 0, 0, 100, 100))
        assert L.ssmul_mul_batched_host(ctypes.c_void_p(plan), 1, arr, a.ctypes.data, a.ctypes.data,
                                        z.ctypes.data, None) == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_mul_batched_host(plan, d * 3, a.ctypes.data, a.ctypes.data, z.ctypes.data,
                                          res) == abi.SSMUL_TOO_LARGE
        assert abi.ssmul_mul_batched_host(plan, [(0, 0, 0, 101, 100)], a.ctypes.data,
                                          a.ctypes.data, z.ctypes.data, res) == abi.SSMUL_TOO_LARGE
        assert abi.ssmul_mul_batched_host(plan, [(0, 0, 0, 0, 100)], a.ctypes.data, a.ctypes.data,
                                          z.ctypes.data, res) == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_mul_batched_host(plan, [], a.ctypes.data, a.ctypes.data, z.ctypes.data,
                                          res) == abi.SSMUL_OK
        assert abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_HOST_PIECES, 0) == abi.SSMUL_INVALID_ARG
    finally:
        abi.ssmul_plan_destroy(plan)
