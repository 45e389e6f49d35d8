"""Batching (grouped launches, CUDA-graph replay), autotuned geometry and the
ladder's binary32 router, against the CPU oracle."""
import ctypes
import os

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


def _pairs(seed, count, lo, hi):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        na, nb = (int(v) for v in np.exp(rng.uniform(np.log(lo), np.log(hi), 2)).astype(int))
        out.append(synth.operand_pair(synth.SEED_BASE + seed * 1000 + i, na, nb,
                                      "ff" if i % 9 == 0 else "uniform"))
    return out


class StreamPlan(Plan):
    def __init__(self, max_na, max_nb, max_products, prec):
        self.stream = torch.cuda.Stream()
        self.h = abi.ssmul_plan(max_na, max_nb, max_products, prec, self.stream.cuda_stream)


def _run_batch_on(plan, pairs, pools=None):
    na = [len(a) for a, _ in pairs]
    nb = [len(b) for _, b in pairs]
    a_off = np.concatenate([[0], np.cumsum(na)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(nb)[:-1]])
    nz = np.array(na) + np.array(nb)
    z_off = np.concatenate([[0], np.cumsum(nz)[:-1]])
    if pools is None:
        pools = (dev(np.concatenate([a for a, _ in pairs])), dev(np.concatenate([b for _, b in pairs])),
                 torch.zeros(int(nz.sum()), dtype=torch.uint8, device="cuda"),
                 torch.zeros(ctypes.sizeof(abi.ssmul_result) * len(pairs), dtype=torch.uint8,
                             device="cuda"))
    da, db, dz, dres = pools
    descs = [(int(a_off[i]), int(b_off[i]), int(z_off[i]), na[i], nb[i]) for i in range(len(pairs))]
    dz.fill_(0xA5)
    s = abi.ssmul_mul_batched(plan.h, descs, da.data_ptr(), db.data_ptr(), dz.data_ptr(),
                              dres.data_ptr())
    plan.stream.synchronize()
    res = (abi.ssmul_result * len(pairs))()
    host = dres.cpu().numpy()
    ctypes.memmove(res, host.ctypes.data, ctypes.sizeof(res))
    z = dz.cpu().numpy()
    return s, list(res), [z[z_off[i]:z_off[i] + nz[i]] for i in range(len(pairs))], pools


def test_graph_replay_and_recapture():
    pairs = _pairs(1, 60, 8, 30000)
    mx = max(max(len(a), len(b)) for a, b in pairs)
    expect = [E.product(a, b) for a, b in pairs]
    with StreamPlan(mx, mx, 80, abi.SSMUL_PREC_LADDER) as p:
        with torch.cuda.stream(p.stream):
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_GRAPH, 1) == OK
            pools = None
            for rep in range(3):                      # capture, then two replays
                s, res, z, pools = _run_batch_on(p, pairs, pools)
                assert s == OK
                for r, zi, ei in zip(res, z, expect):
                    assert r.status == OK and np.array_equal(zi, ei)
            other = _pairs(2, 70, 3, 5000)            # a different batch: recaptured
            s, res, z, _ = _run_batch_on(p, other)
            assert s == OK
            for (a, b), r, zi in zip(other, res, z):
                assert r.status == OK and np.array_equal(zi, E.product(a, b))


def test_autotuned_geometry_is_exact(tmp_path):
    os.environ["SSMUL_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        n = 40000
        with Plan(n, n) as p:
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_AUTOTUNE, 1) == OK
            for ln in range(13, 18):
                s, (l1, l2, lc) = abi.ssmul_debug_geometry(p.h, ln)
                assert s == OK and l1 + l2 == ln and 1 <= l1 <= 12 and 2 <= l2 <= 11
            for na, nb in [(n, n), (5000, 4000), (20000, 3)]:
                a, b = synth.operand_pair(na + nb, na, nb)
                s, r, z = p.mul(a, b)
                assert s == OK and np.array_equal(z, E.product(a, b))
        lines = open(tmp_path / "tune.txt").read().splitlines()
        assert len(lines) == 15                        # 2^13..2^17, 3 2^11..3 2^15, 5 2^10..5 2^14
        with Plan(n, n) as p:                          # read back from the cache
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_AUTOTUNE, 1) == OK
            assert len(open(tmp_path / "tune.txt").read().splitlines()) == 15
            for j in range(11, 16):
                s, (l1, l2, lc) = abi.ssmul_debug_geometry(p.h, 32 + j)
                assert s == OK and l1 + l2 == j and l1 % 2 == 0
            for j in range(10, 15):
                s, (l1, l2, lc) = abi.ssmul_debug_geometry(p.h, 64 + j)
                assert s == OK and l1 + l2 == j and l1 % 2 == 0 and (5 << l1) <= 4096
    finally:
        del os.environ["SSMUL_TUNE_CACHE"]


def test_forced_short_column_geometries_are_exact(tmp_path):
    """Power-of-two lengths split into the shortest columns the four-step
    kernels take (forced through the tuning cache): N1 = 4 (the forward
    columns' exact first step is their only step; the inverse columns' first
    step, which reads W itself, is their only step), N1 = 8 (the forward
    columns end with a radix-2 step that stores Z), N1 = 16 and 32; batched
    and single products bit-exact against the oracle."""
    name = torch.cuda.get_device_properties(0).name
    cache = tmp_path / "tune.txt"
    forced = {13: (11, 9), 14: (11, 10), 15: (11, 11), 16: (11, 12)}
    cache.write_text("".join(f"{name}\t{ln} {l2} {cta}\n" for ln, (l2, cta) in forced.items()))
    os.environ["SSMUL_TUNE_CACHE"] = str(cache)
    try:
        n = 1 << 15
        pairs = [synth.operand_pair(7000 + i, na, nb) for i, (na, nb) in
                 enumerate([(4000, 4000), (3000, 5190), (8000, 8000), (16000, 16000),
                            (32000, 32000), (30000, 1000)])]
        pairs.append(synth.operand_pair(7100, 16000, 16000, "ff"))
        with Plan(n, n, len(pairs)) as p:
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_LENGTHS, 0) == OK
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_AUTOTUNE, 1) == OK
            for ln, (l2, cta) in forced.items():
                s, (g1, g2, gc) = abi.ssmul_debug_geometry(p.h, ln)
                assert s == OK and (g1, g2, gc) == (ln - l2, l2, cta)
            s, res, digits = batched(p, pairs)
            assert s == OK
            for (a, b), r, z in zip(pairs, res, digits):
                assert r.status == OK and np.array_equal(z, E.product(a, b))
            for a, b in pairs[:4]:
                s1, r1, z1 = p.mul(a, b)
                assert s1 == OK and np.array_equal(z1, E.product(a, b))
    finally:
        del os.environ["SSMUL_TUNE_CACHE"]


def test_fp32_router_option():
    a, b = synth.operand_pair(5, 300, 300)
    small = synth.operand_pair(6, 40, 40)
    with Plan(300, 300, 0, abi.SSMUL_PREC_LADDER) as p:
        s, r, z = p.mul(a, b)                       # 600 digits: above the default 512
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        s, r, z = p.mul(*small)                     # 80 digits: binary32 on 4-bit digits
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32
        assert np.array_equal(z, E.product(*small))
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_MAX_DIGITS, 700) == OK
        s, r, z = p.mul(a, b)                       # tried in binary32 (beyond its limit), escalated
        assert s == OK and np.array_equal(z, E.product(a, b))
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_MAX_DIGITS, 0) == OK
        s, r, z = p.mul(*small)                     # 0: never binary32
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_NIBBLES, 0) == OK
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_FP32_MAX_DIGITS, 100) == OK
        s, r, z = p.mul(*small)                     # bytes: 80 digits do not isolate in binary32
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        assert np.array_equal(z, E.product(*small))
        assert abi.ssmul_plan_set_option(p.h, 99, 1) == abi.SSMUL_INVALID_ARG


def test_batched_chunks_beyond_the_arena():
    # each product of 2^16 digits needs 6 MiB of spectra; a 16 MiB arena
    # runs the batch of 6 in three chunks
    pairs = [synth.operand_pair(900 + i, 1 << 16, (1 << 16) - 3 * i) for i in range(6)]
    os.environ["SSMUL_ARENA_MB"] = "16"
    try:
        with Plan(1 << 16, 1 << 16, 6) as p:
            s, res, digits = batched(p, pairs)
    finally:
        del os.environ["SSMUL_ARENA_MB"]
    assert s == OK
    for (a, b), r, z in zip(pairs, res, digits):
        assert r.status == OK and np.array_equal(z, E.product(a, b))


@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64,
                                  abi.SSMUL_PREC_DISC32X2, abi.SSMUL_PREC_LADDER_FAST])
def test_bench_configuration_75k(prec):
    """The launch configuration bench.py times, at the paper's size: one
    ssmul_mul_batched call over products of two 75,000-digit operands from
    the bench's own generator (uniform bytes, the last product all 0xFF),
    on the plan's stream, twice in a row; every product bit-exact."""
    import bench
    B, n = 16, 75000
    (a_pool, b_pool, a_off, b_off, z_off), dists = bench.make_batch(0, B, n)
    expect = [E.product(a_pool[a_off[i]:a_off[i] + n], b_pool[b_off[i]:b_off[i] + n])
              for i in range(B)]
    with StreamPlan(n, n, B, prec) as p:
        with torch.cuda.stream(p.stream):
            descs = [(int(a_off[i]), int(b_off[i]), int(z_off[i]), n, n) for i in range(B)]
            da, db = dev(a_pool), dev(b_pool)
            dres = torch.zeros(ctypes.sizeof(abi.ssmul_result) * B, dtype=torch.uint8, device="cuda")
            outs = []
            for _ in range(2):
                dz = torch.full((B * 2 * n,), 0xA5, dtype=torch.uint8, device="cuda")
                assert abi.ssmul_mul_batched(p.h, descs, da.data_ptr(), db.data_ptr(), dz.data_ptr(),
                                             dres.data_ptr()) == OK
                p.stream.synchronize()
                res = (abi.ssmul_result * B)()
                host = dres.cpu().numpy()
                ctypes.memmove(res, host.ctypes.data, ctypes.sizeof(res))
                outs.append((list(res), dz.cpu().numpy()))
    for res, z in outs:
        for i in range(B):
            assert res[i].status == OK, (i, abi.status_string(res[i].status))
            assert np.array_equal(z[z_off[i]:z_off[i] + 2 * n], expect[i]), i
            assert 0.0 <= res[i].max_width < 1.0
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_LADDER, abi.SSMUL_PREC_LADDER_FAST])
def test_group_lanes_same_outcomes_eager_and_graph(prec):
    """SSMUL_OPT_LANES spreads the length groups over several streams: the
    outcomes (status, deciding rung, width) and digits equal the one-lane
    run's, eager and graph-replayed, and the digits are the oracle's."""
    pairs = _pairs(3, 90, 3, 40000)
    mx = max(max(len(a), len(b)) for a, b in pairs)
    expect = [E.product(a, b) for a, b in pairs]
    runs = []
    for lanes, graph in [(1, 0), (4, 0), (3, 1), (2, 1)]:
        with StreamPlan(mx, mx, 100, prec) as p:
            with torch.cuda.stream(p.stream):
                assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_LANES, lanes) == OK
                assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_GRAPH, graph) == OK
                pools = None
                for _ in range(2 if graph else 1):       # capture, then a replay
                    s, res, z, pools = _run_batch_on(p, pairs, pools)
                    assert s == OK
                    runs.append(([r.as_dict() for r in res], z))
    for res, z in runs:
        assert res == runs[0][0]
        for r, zi, ei in zip(res, z, expect):
            assert r["status"] == OK and np.array_equal(zi, ei)
    with Plan(10, 10, 1) as p:
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_LANES, 0) == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_LANES, 5) == abi.SSMUL_INVALID_ARG
