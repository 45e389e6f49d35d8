"""Report workloads of the benchmark: the configurations besides the 75k headline.

c1      one product of two 4,096-digit uniform operands (FFT length 8,192),
        binary64 rectangles through ssmul_mul, checked against the oracle's
        long multiplication (schoolbook), whose time on one host core is
        reported beside it.
c3      the size sweep: square products of 2^k uniform digits, k = 10 .. 22,
        and the unbalanced 2^20 x 2^12, under binary64 rectangles, binary64
        discs and double-binary32 discs: status, largest width and time per
        product; the largest square size every rung still isolates.  Also
        the binary32 rectangle limit (squares of 1 .. 64 digits).
c4      the precision ladder: 4,096 square products, n ~ U{512..32768}, 10%
        all-0xFF: the ladder (binary32 first, binary64 on failure) batched,
        binary64 batched, the fast ladder batched, and binary64 one product
        at a time; verified digits/s of each and the fraction resolved in
        binary32, per size.
c5      the uneven batch: 20,000 products with na, nb independent and
        log-uniform in [64, 131072], the ladders in one graph-captured
        batched call against binary64 one product at a time.
split   square products of 2^19 .. 2^22 digits, past the rectangles'
        isolation limit: rectangles on the whole product, the same cut into
        parts of 2^18 digits (Section 1's "different algorithm"), and
        binary64 discs on the whole product.

Every product counted as verified has status SSMUL_OK and digits equal to
the CPU oracle's exact product (bench_verify).  `python bench.py --workload
sweep|ladder|uneven|split` prints one report as a JSON line; the default
`python bench.py` run embeds c1, c3, c4 and c5 in its line.
"""
from __future__ import annotations

import ctypes
import json
import time

import numpy as np

import synth
from bench_verify import OraclePool, batch_jobs, digest


class Ctx:
    """torch, the C ABI and a lazily started oracle pool."""

    def __init__(self, lanes: int = 4):
        import torch
        if not torch.cuda.is_available():
            raise SystemExit("the report workloads need a CUDA device")
        from paper_1006_0405_gb300 import abi
        abi.load()
        self.torch, self.abi, self.lanes = torch, abi, lanes
        self._pool = None

    def pool(self) -> OraclePool:
        if self._pool is None:
            self._pool = OraclePool()
        return self._pool

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool = None


class Batch:
    """Device pools and descriptors of a batch drawn by synth.batch_operands."""

    def __init__(self, torch, abi, seed, na, nb, dists):
        self.seed, self.dists = seed, list(dists)
        self.na = np.asarray(na, np.int64)
        self.nb = np.asarray(nb, np.int64)
        (self.a_pool, self.b_pool, self.a_off, self.b_off, self.z_off) = \
            synth.batch_operands(seed, self.na, self.nb, dists)
        self.nz = self.na + self.nb
        self.count = len(self.na)
        self.torch, self.abi = torch, abi
        self.da = torch.from_numpy(self.a_pool).cuda()
        self.db = torch.from_numpy(self.b_pool).cuda()
        self.dz = torch.zeros(int(self.nz.sum()), dtype=torch.uint8, device="cuda")
        self.res_bytes = ctypes.sizeof(abi.ssmul_result) * self.count
        self.dres = torch.zeros(self.res_bytes, dtype=torch.uint8, device="cuda")
        self.descs = (abi.ssmul_desc * self.count)()
        for i in range(self.count):
            self.descs[i] = abi.ssmul_desc(int(self.a_off[i]), int(self.b_off[i]),
                                           int(self.z_off[i]), int(self.na[i]), int(self.nb[i]))

    def jobs(self):
        return batch_jobs(self.seed, self.na, self.nb, self.dists)

    def run(self, plan):
        s = self.abi.ssmul_mul_batched(plan, self.descs, self.da.data_ptr(), self.db.data_ptr(),
                                       self.dz.data_ptr(), self.dres.data_ptr())
        if s != self.abi.SSMUL_OK:
            raise RuntimeError(self.abi.status_string(s))

    def results(self):
        rr = (self.abi.ssmul_result * self.count)()
        host = self.dres.cpu().numpy()
        ctypes.memmove(rr, host.ctypes.data, self.res_bytes)
        return list(rr)

    def digits(self):
        z = self.dz.cpu().numpy()
        return [z[self.z_off[i]:self.z_off[i] + self.nz[i]] for i in range(self.count)]

    def clear(self):
        self.dz.fill_(0xA5)
        self.dres.zero_()
        self.torch.cuda.synchronize()


def _time_batch(torch, plan, batch, reps, stream):
    """Seconds per batched call: one untimed call (it captures the CUDA graph
    when the plan replays graphs), then `reps` calls timed with events on the
    plan's stream."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        batch.run(plan)
        stream.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            batch.run(plan)
        ev1.record(stream)
        stream.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / reps


def _one_at_a_time(torch, abi, batch, max_n, prec):
    """Every product by its own ssmul_mul call (which waits for it), binary64;
    returns (seconds, results)."""
    plan = abi.ssmul_plan(max_n, max_n, 0, prec, 0)
    torch.cuda.synchronize()
    outs = []
    t0 = time.perf_counter()
    for i in range(batch.count):
        dz = batch.dz[batch.z_off[i]:batch.z_off[i] + batch.nz[i]]
        s, r = abi.ssmul_mul(plan, batch.da.data_ptr() + int(batch.a_off[i]), int(batch.na[i]),
                             batch.db.data_ptr() + int(batch.b_off[i]), int(batch.nb[i]),
                             dz.data_ptr())
        outs.append(r)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    abi.ssmul_plan_destroy(plan)
    return el, outs


def _size_buckets(nz):
    """log2 buckets of the output digits (na + nb) of each product."""
    return np.floor(np.log2(np.maximum(nz, 1))).astype(int)


def _fp32_fraction_by_size(abi, results, nz):
    b = _size_buckets(nz)
    out = {}
    for k in sorted(set(b.tolist())):
        idx = np.nonzero(b == k)[0]
        fp32 = sum(1 for i in idx if results[i].status == abi.SSMUL_OK and
                   results[i].precision_used == abi.SSMUL_PREC_FP32)
        out[f"2^{k}..2^{k + 1}"] = round(fp32 / len(idx), 4)
    return out


def _statuses(abi, results):
    st = {}
    for r in results:
        k = abi.status_string(r.status)
        st[k] = st.get(k, 0) + 1
    return st


def _used(abi, results):
    names = {abi.SSMUL_PREC_FP32: "fp32", abi.SSMUL_PREC_FP64: "fp64",
             abi.SSMUL_PREC_DISC64: "disc64", abi.SSMUL_PREC_DISC32X2: "disc32x2",
             abi.SSMUL_PREC_NAIVE64: "naive64"}
    out = {}
    for r in results:
        if r.status == abi.SSMUL_OK:
            k = names.get(r.precision_used, str(r.precision_used))
            out[k] = out.get(k, 0) + 1
    return out


# ---- C1: one 4,096 x 4,096-digit product ---------------------------------------

def c1(ctx, reps: int = 20) -> dict:
    torch, abi = ctx.torch, ctx.abi
    from oracle import exact as E
    n = 4096
    a, b = synth.operand_pair(synth.SEED_BASE + 1, n, n)
    plan = abi.ssmul_plan(n, n, 0, abi.SSMUL_PREC_FP64, 0)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dz = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
    abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
        times.append(time.perf_counter() - t0)
    abi.ssmul_plan_destroy(plan)
    z = dz.cpu().numpy()
    t0 = time.perf_counter()
    school = E.long_mul(a, b)                   # Section 2.1, single thread
    t_school = time.perf_counter() - t0
    ok = bool(s == abi.SSMUL_OK and np.array_equal(z, school))
    return {"workload": f"{n}x{n} base-256 digits, uniform, binary64 rectangles, one product "
                        f"per ssmul_mul call (which waits for it), FFT length "
                        f"{r.fft_odd << r.fft_log2}",
            "ms_per_product": 1e3 * float(np.median(times)), "multiplies_per_s":
                1.0 / float(np.median(times)) if ok else 0.0,
            "status": abi.status_string(s), "max_width": r.max_width,
            "verified": f"{int(ok)}/1 against schoolbook long multiplication",
            "schoolbook_cpu_ms_one_core": 1e3 * t_school}


# ---- C3: the size sweep ---------------------------------------------------------

C3_SIZES = [(1 << k, 1 << k) for k in range(10, 23)] + [(1 << 20, 1 << 12)]


def _rungs(abi):
    return (("fp64", abi.SSMUL_PREC_FP64), ("disc64", abi.SSMUL_PREC_DISC64),
            ("disc32x2", abi.SSMUL_PREC_DISC32X2))


def c3(ctx, sizes=C3_SIZES, dists=("uniform",), balanced=False, fp32_limit=True) -> dict:
    torch, abi = ctx.torch, ctx.abi
    seed = synth.SEED_BASE + 3
    cases = [(na, nb, dist) for na, nb in sizes for dist in dists]
    rows, got = [], []
    for na, nb, dist in cases:
        a, b = synth.operand_pair(seed, na, nb, dist)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(na + nb, dtype=torch.uint8, device="cuda")
        row = {"na": na, "nb": nb, "dist": dist}
        for name, prec in _rungs(abi):
            plan = abi.ssmul_plan(na, nb, 0, prec, 0)
            if balanced:
                abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_BALANCED, 1)
            abi.ssmul_mul(plan, da.data_ptr(), na, db.data_ptr(), nb, dz.data_ptr())
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                dz.fill_(0xA5)
                s, r = abi.ssmul_mul(plan, da.data_ptr(), na, db.data_ptr(), nb, dz.data_ptr())
            el = (time.perf_counter() - t0) / reps
            abi.ssmul_plan_destroy(plan)
            row[name] = {"status": abi.status_string(s), "max_width": r.max_width,
                         "N": r.fft_odd << r.fft_log2, "ms": 1e3 * el}
            got.append((row, name, s, digest(dz.cpu().numpy())))
        rows.append(row)
    expected = ctx.pool().digests([("pair", seed, na, nb, dist, "ntt") for na, nb, dist in cases])
    exp_of = {id(row): e for row, e in zip(rows, expected)}
    for row, name, s, dg in got:
        row[name]["verified"] = bool(s == abi.SSMUL_OK and dg == exp_of[id(row)])
    largest = {}
    for name, _ in _rungs(abi):
        best = None
        for row in rows:
            if row["na"] != row["nb"] or row["dist"] != "uniform":
                continue
            if not row[name]["verified"]:
                break
            best = row["na"]
        largest[name] = best
    n_ok = sum(1 for row, name, s, _ in got if s == abi.SSMUL_OK)
    n_ver = sum(1 for row, name, s, _ in got if row[name]["verified"])
    out = {"workload": "square products of 2^k uniform digits, k = 10..22, and 2^20 x 2^12; "
                       "one product per ssmul_mul call", "balanced_digits": balanced,
           "rows": rows, "largest_isolated_square_digits": largest,
           "verified": f"{n_ver}/{n_ok} products with status SSMUL_OK are bit-exact"}
    if fp32_limit:
        out["fp32_rectangles"] = fp32_isolation_limit(ctx)
    return out


FP32_LIMIT_SIZES = list(range(1, 65)) + list(range(72, 513, 8)) + list(range(544, 2049, 32))


def fp32_isolation_limit(ctx, dists=("uniform", "ff")) -> dict:
    """Binary32 rectangles on squares n x n for n on FP32_LIMIT_SIZES, in three
    representations (bytes, balanced bytes, 4-bit digits): the largest n
    such that every product of every size up to n isolates and is exact (8
    uniform products per size, seeds SEED_BASE + 1000 n + t; one all-0xFF)."""
    torch, abi = ctx.torch, ctx.abi
    from oracle import exact as E
    out = {}
    for mode, balanced, nibbles in (("bytes", 0, 0), ("balanced_bytes", 1, 0),
                                    ("nibbles", 0, 1)):
        plan = abi.ssmul_plan(2048, 2048, 0, abi.SSMUL_PREC_FP32, 0)
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_BALANCED, balanced)
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_FP32_NIBBLES, nibbles)
        for dist in dists:
            limit, width = 0, 0.0
            for n in FP32_LIMIT_SIZES:
                good, w = True, 0.0
                for t in range(8 if dist == "uniform" else 1):
                    a, b = synth.operand_pair(synth.SEED_BASE + 1000 * n + t, n, n, dist)
                    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
                    dz = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
                    s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
                    w = max(w, r.max_width)
                    if s != abi.SSMUL_OK or not np.array_equal(dz.cpu().numpy(), E.long_mul(a, b)):
                        good = False
                        break
                if not good:
                    break
                limit, width = n, w
            out[f"{mode}_{dist}"] = {"largest_square_digits": limit, "max_width_there": width}
        abi.ssmul_plan_destroy(plan)
    out["note"] = ("sizes 1..64, then every 8 to 512, then every 32 to 2048; 8 uniform "
                   "products (1 all-0xFF) per size, all isolated and exact up to the size given")
    return out


# ---- C4 and C5: batches of many products -------------------------------------------

def _batch_report(ctx, seed, na, nb, dists, lanes, one_lane=False) -> dict:
    torch, abi = ctx.torch, ctx.abi
    batch = Batch(torch, abi, seed, na, nb, dists)
    max_n = int(max(batch.na.max(), batch.nb.max()))
    stream = torch.cuda.Stream()
    out = {"count": batch.count, "output_digits_total": int(batch.nz.sum()), "lanes": lanes}
    runs = [("ladder_batched", abi.SSMUL_PREC_LADDER), ("fp64_batched", abi.SSMUL_PREC_FP64),
            ("ladder_fast_batched", abi.SSMUL_PREC_LADDER_FAST)]
    # the GPU runs first, then the oracle (no host load during the timings)
    digits = {}
    for key, prec in runs:
        digits[key] = _batched_gpu(ctx, batch, max_n, prec, stream, lanes)
    if one_lane:
        digits["ladder_batched_one_lane"] = _batched_gpu(ctx, batch, max_n, abi.SSMUL_PREC_LADDER,
                                                         stream, 1)
    batch.clear()
    el, rs1 = _one_at_a_time(torch, abi, batch, max_n, abi.SSMUL_PREC_FP64)
    digits["fp64_one_at_a_time"] = (el, rs1, [digest(z) for z in batch.digits()])
    pool = ctx.pool()
    t0 = time.perf_counter()
    expected = pool.digests(batch.jobs())
    t_oracle = time.perf_counter() - t0
    # the oracle's own throughput on the host cores (exact convolution + carry per product)
    out["oracle_cpu"] = {"s_total": t_oracle, "digits_per_s": float(batch.nz.sum()) / t_oracle,
                         "cores": pool.processes, "kind": "oracle",
                         "sample": "every product of the batch (its operands drawn again in the worker), "
                                   "one worker process per core"}
    for key, (t, rs, dg) in digits.items():
        n_ver = d_ver = 0
        for r, d, e, nz in zip(rs, dg, expected, batch.nz):
            if r.status == abi.SSMUL_OK and d == e:
                n_ver += 1
                d_ver += int(nz)
        fp32 = sum(1 for r in rs if r.status == abi.SSMUL_OK and
                   r.precision_used == abi.SSMUL_PREC_FP32)
        entry = {("s_total" if key == "fp64_one_at_a_time" else "s_per_batch"): t,
                 "verified_digits_per_s": d_ver / t, "verified": f"{n_ver}/{batch.count}",
                 "statuses": _statuses(abi, rs), "deciding_rung": _used(abi, rs)}
        if key.startswith("ladder"):
            entry["fraction_fp32"] = fp32 / batch.count
            entry["fraction_fp32_by_output_digits"] = _fp32_fraction_by_size(abi, rs, batch.nz)
        out[key] = entry
    base = out["fp64_one_at_a_time"]["verified_digits_per_s"]
    for key in ("ladder_batched", "fp64_batched", "ladder_fast_batched"):
        out["speedup_" + key + "_vs_fp64_one_at_a_time"] = \
            out[key]["verified_digits_per_s"] / base if base else None
    if one_lane:
        t1 = out["ladder_batched_one_lane"]["s_per_batch"]
        out["lanes_saving"] = 1.0 - out["ladder_batched"]["s_per_batch"] / t1
    return out


def _batched_gpu(ctx, batch, max_n, prec, stream, lanes):
    """(seconds per graph-replayed batched call, results, digit digests)."""
    torch, abi = ctx.torch, ctx.abi
    plan = abi.ssmul_plan(max_n, max_n, batch.count, prec, stream.cuda_stream)
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_GRAPH, 1)
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_LANES, lanes)
    batch.clear()
    t = _time_batch(torch, plan, batch, 3, stream)
    abi.ssmul_plan_destroy(plan)
    return t, batch.results(), [digest(z) for z in batch.digits()]


def c4(ctx) -> dict:
    seed = synth.SEED_BASE + 4
    na, nb, dists = synth.ladder_batch(seed, count=4096)
    out = _batch_report(ctx, seed, na, nb, dists, ctx.lanes)
    out["workload"] = ("4,096 square products, n ~ U{512..32768}, 10% all-0xFF; batched calls "
                       "replay a CUDA graph")
    return out


def c5(ctx, one_lane=True) -> dict:
    seed = synth.SEED_BASE + 5
    na, nb, dists = synth.uneven_batch(seed, count=20000)
    out = _batch_report(ctx, seed, na, nb, dists, ctx.lanes, one_lane=one_lane)
    out["workload"] = ("20,000 products, na and nb independent, log-uniform in [64, 131072], "
                       "uniform bytes; batched calls replay a CUDA graph")
    return out


# ---- products past the rectangles' isolation limit ------------------------------

def split(ctx) -> dict:
    torch, abi = ctx.torch, ctx.abi
    part = 1 << 18
    seed = synth.SEED_BASE + 6
    rows, got = [], []
    sizes = [1 << k for k in (19, 20, 21, 22)]
    for n in sizes:
        a, b = synth.operand_pair(seed, n, n)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
        for name, prec, split_m in (("fp64", abi.SSMUL_PREC_FP64, 0),
                                    ("fp64_split_2^18", abi.SSMUL_PREC_FP64, part),
                                    ("disc64", abi.SSMUL_PREC_DISC64, 0)):
            plan = abi.ssmul_plan(n, n, 0, prec, 0)
            if split_m:
                assert abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_SPLIT_DIGITS, split_m) == 0
            abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
            el = (time.perf_counter() - t0) / reps
            abi.ssmul_plan_destroy(plan)
            row = {"digits": n, "method": name, "status": abi.status_string(s),
                   "max_width": r.max_width, "N": r.fft_odd << r.fft_log2, "ms": 1e3 * el}
            rows.append(row)
            got.append((row, n, s, digest(dz.cpu().numpy())))
    expected = dict(zip(sizes, ctx.pool().digests([("pair", seed, n, n, "uniform", "ntt")
                                                   for n in sizes])))
    for row, n, s, dg in got:
        row["verified"] = bool(s == abi.SSMUL_OK and dg == expected[n])
        row["verified_digits_per_s"] = (2 * n / (row["ms"] / 1e3)) if row["verified"] else 0.0
    return {"part_digits": part, "rows": rows}


def run(args):
    ctx = Ctx(lanes=args.lanes)
    try:
        if args.workload == "sweep":
            out = {"report": "sweep", **c3(ctx, dists=("uniform", "ff"), balanced=args.balanced)}
        elif args.workload == "ladder":
            out = {"report": "ladder", **c4(ctx)}
        elif args.workload == "uneven":
            out = {"report": "uneven", **c5(ctx)}
        elif args.workload == "c1":
            out = {"report": "c1", **c1(ctx)}
        else:
            out = {"report": "split", **split(ctx)}
    finally:
        ctx.close()
    print(json.dumps(out), flush=True)
