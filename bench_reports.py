"""Report workloads of bench.py (`--workload sweep | ladder | uneven`).

sweep   square products of 2^k uniform digits, k = 10 .. 22, and the
        unbalanced pair 2^20 x 2^12, in binary64: status, largest interval
        width, time per product; the largest length at which every
        coefficient is still isolated.  Also the binary32 isolation limit
        (square sizes 2 .. 64 digits).
ladder  4,096 square products, n ~ U{512..32768}, 10% all-0xFF: the ladder
        (binary32 first, binary64 on failure) in one batched call, plain
        binary64 batched, and plain binary64 one product at a time; verified
        digits/s of each and the fraction resolved in binary32.
uneven  20,000 products with na, nb independent and log-uniform in
        [64, 131072]: the ladder in one graph-captured batched call against
        the same set one product at a time in binary64.
split   square products of 2^19 .. 2^22 uniform digits, past the binary64
        rectangles' isolation limit: rectangles on the whole product, the
        same cut into parts of 2^18 digits (SSMUL_OPT_SPLIT_DIGITS, Section
        1's "different algorithm"), and binary64 discs on the whole product;
        status, time per product and residue verification of each.

Verification is against the CPU oracle: every product's digits against the
exact product for sweep and ladder; for the uneven batch every product's
residues modulo two primes plus the full digits of a seeded 5% sample.
Each workload prints one JSON line.
"""
from __future__ import annotations

import ctypes
import json
import time

import numpy as np

import synth

PRIMES = (2**61 - 1, 1_000_000_007)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the report workloads need a CUDA device")
    return torch


class Batch:
    """Device pools and descriptors of a batch."""

    def __init__(self, torch, seed, na, nb, dists):
        self.na = np.asarray(na, np.int64)
        self.nb = np.asarray(nb, np.int64)
        (self.a_pool, self.b_pool, self.a_off, self.b_off, self.z_off) = \
            synth.batch_operands(seed, self.na, self.nb, dists)
        self.nz = self.na + self.nb
        self.count = len(self.na)
        self.da = torch.from_numpy(self.a_pool).cuda()
        self.db = torch.from_numpy(self.b_pool).cuda()
        self.dz = torch.zeros(int(self.nz.sum()), dtype=torch.uint8, device="cuda")
        from paper_1006_0405_gb300 import abi
        self.abi = abi
        self.res_bytes = ctypes.sizeof(abi.ssmul_result) * self.count
        self.dres = torch.zeros(self.res_bytes, dtype=torch.uint8, device="cuda")
        self.descs = (abi.ssmul_desc * self.count)()
        for i in range(self.count):
            self.descs[i] = abi.ssmul_desc(int(self.a_off[i]), int(self.b_off[i]),
                                           int(self.z_off[i]), int(self.na[i]), int(self.nb[i]))

    def a(self, i):
        return self.a_pool[self.a_off[i]:self.a_off[i] + self.na[i]]

    def b(self, i):
        return self.b_pool[self.b_off[i]:self.b_off[i] + self.nb[i]]

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


def _time_batch(torch, plan, batch, reps, stream):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        batch.run(plan)                     # warm-up (and graph capture)
        stream.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            batch.run(plan)
        ev1.record(stream)
        stream.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / reps


def _one_at_a_time(torch, abi, batch, max_n, prec):
    plan = abi.ssmul_plan(max_n, max_n, 0, prec, 0)
    torch.cuda.synchronize()
    outs = []
    t0 = time.perf_counter()
    for i in range(batch.count):
        dz = batch.dz[batch.z_off[i]:batch.z_off[i] + batch.nz[i]]
        s, r = abi.ssmul_mul(plan, batch.da.data_ptr() + int(batch.a_off[i]), int(batch.na[i]),
                             batch.db.data_ptr() + int(batch.b_off[i]), int(batch.nb[i]),
                             dz.data_ptr())
        outs.append((s, r.precision_used))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    abi.ssmul_plan_destroy(plan)
    return el, outs


def _expected(batch, idx=None):
    """Exact products from the CPU oracle (NTT convolution and carry)."""
    from oracle import exact as E
    idx = range(batch.count) if idx is None else idx
    return {i: E.carry(E.conv_ntt(batch.a(i), batch.b(i)), int(batch.nz[i])) for i in idx}


def _verify_full(rs, zs, expect):
    return sum(1 for i, e in expect.items() if rs[i].status == 0 and np.array_equal(zs[i], e))


def _verify_residues(batch, rs, zs):
    from oracle import exact as E
    ok = np.zeros(batch.count, bool)
    for i in range(batch.count):
        if rs[i].status != 0:
            continue
        good = True
        for q in PRIMES:
            if E.residue(zs[i], q) != E.residue(batch.a(i), q) * E.residue(batch.b(i), q) % q:
                good = False
                break
        ok[i] = good
    return ok


def sweep(args):
    torch = _torch()
    from oracle import exact as E
    from paper_1006_0405_gb300 import abi
    abi.load()
    sizes = [(1 << k, 1 << k) for k in range(10, 23)] + [(1 << 20, 1 << 12)]
    prec = {"fp64": abi.SSMUL_PREC_FP64, "disc64": abi.SSMUL_PREC_DISC64,
            "naive64": abi.SSMUL_PREC_NAIVE64, "disc32x2": abi.SSMUL_PREC_DISC32X2,
            "ladder_fast": abi.SSMUL_PREC_LADDER_FAST}[args.precision]
    rows = []
    largest = None
    for na, nb in sizes:
        for dist in ("uniform", "ff"):
            a, b = synth.operand_pair(synth.SEED_BASE + 3, na, nb, dist)
            plan = abi.ssmul_plan(na, nb, 0, prec, 0)
            if args.balanced:
                abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_BALANCED, 1)
            da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
            dz = torch.zeros(na + nb, dtype=torch.uint8, device="cuda")
            abi.ssmul_mul(plan, da.data_ptr(), na, db.data_ptr(), nb, dz.data_ptr())
            reps = 3
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                s, r = abi.ssmul_mul(plan, da.data_ptr(), na, db.data_ptr(), nb, dz.data_ptr())
            el = (time.perf_counter() - t0) / reps
            abi.ssmul_plan_destroy(plan)
            z = dz.cpu().numpy()
            exact = bool(s in (abi.SSMUL_OK, abi.SSMUL_UNVERIFIED) and
                         np.array_equal(z, E.carry(E.conv_ntt(a, b), na + nb)))
            rows.append({"na": na, "nb": nb, "dist": dist, "log2_N": r.fft_log2, "N": r.fft_odd << r.fft_log2,
                         "status": abi.status_string(s), "max_width": r.max_width,
                         "n_unisolated": r.n_unisolated, "verified": exact, "ms": 1e3 * el})
            if na == nb and dist == "uniform" and exact and (largest == na // 2 or largest is None):
                largest = na
    # binary32 isolation limit
    f32_ok = []
    plan = abi.ssmul_plan(64, 64, 0, abi.SSMUL_PREC_FP32, 0)
    for n in range(1, 65):
        good = True
        for t in range(8):
            a, b = synth.operand_pair(synth.SEED_BASE + 1000 * n + t, n, n)
            da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
            dz = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
            s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
            if s != abi.SSMUL_OK or not np.array_equal(dz.cpu().numpy(), E.product(a, b)):
                good = False
        f32_ok.append(good)
    abi.ssmul_plan_destroy(plan)
    f32_limit = 0
    for n, g in enumerate(f32_ok, start=1):
        if not g:
            break
        f32_limit = n
    print(json.dumps({"report": "sweep", "precision": args.precision,
                      "balanced_digits": bool(args.balanced), "rows": rows,
                      "largest_isolated_square_digits": largest,
                      "largest_isolated_square_digits_fp32": f32_limit,
                      "fp32_note": "8 uniform products per size, all isolated up to this size"}),
          flush=True)


def ladder(args):
    torch = _torch()
    from paper_1006_0405_gb300 import abi
    abi.load()
    seed = synth.SEED_BASE + 4
    na, nb, dists = synth.ladder_batch(seed, count=4096)
    batch = Batch(torch, seed, na, nb, dists)
    max_n = int(max(na.max(), nb.max()))
    stream = torch.cuda.Stream()
    expect = _expected(batch)
    out = {"report": "ladder", "count": batch.count, "digits_total": int(batch.nz.sum())}
    for name, prec in (("ladder_batched", abi.SSMUL_PREC_LADDER), ("fp64_batched", abi.SSMUL_PREC_FP64),
                       ("ladder_fast_batched", abi.SSMUL_PREC_LADDER_FAST)):
        plan = abi.ssmul_plan(max_n, max_n, batch.count, prec, stream.cuda_stream)
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_GRAPH, 1)
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_LANES, args.lanes)
        t = _time_batch(torch, plan, batch, 3, stream)
        rs, zs = batch.results(), batch.digits()
        ok = _verify_full(rs, zs, expect)
        fp32 = sum(1 for r in rs if r.status == 0 and r.precision_used == abi.SSMUL_PREC_FP32)
        used = {}
        for r in rs:
            used[r.precision_used] = used.get(r.precision_used, 0) + 1
        out[name] = {"s_per_batch": t, "verified": ok, "precision_used": used,
                     "verified_digits_per_s": float(sum(batch.nz[i] for i in range(batch.count)
                                                        if rs[i].status == 0)) / t,
                     "resolved_fp32": fp32, "fraction_fp32": fp32 / batch.count}
        abi.ssmul_plan_destroy(plan)
    el, outs = _one_at_a_time(torch, abi, batch, max_n, abi.SSMUL_PREC_FP64)
    zs = batch.digits()
    rs1 = [type("R", (), {"status": s})() for s, _ in outs]
    ok = _verify_full(rs1, zs, expect)
    out["fp64_one_at_a_time"] = {"s_total": el, "verified": ok,
                                 "verified_digits_per_s": float(batch.nz.sum()) / el}
    print(json.dumps(out), flush=True)


def uneven(args):
    torch = _torch()
    from paper_1006_0405_gb300 import abi
    abi.load()
    seed = synth.SEED_BASE + 5
    na, nb, dists = synth.uneven_batch(seed, count=20000)
    batch = Batch(torch, seed, na, nb, dists)
    max_n = int(max(na.max(), nb.max()))
    stream = torch.cuda.Stream()
    out = {"report": "uneven", "count": batch.count, "digits_total": int(batch.nz.sum()),
           "lanes": args.lanes}
    for name, prec in (("ladder_graph_batched", abi.SSMUL_PREC_LADDER),
                       ("ladder_fast_graph_batched", abi.SSMUL_PREC_LADDER_FAST)):
        out[name] = _uneven_batched(torch, abi, batch, max_n, prec, stream, seed, args.lanes)
    el, outs = _one_at_a_time(torch, abi, batch, max_n, abi.SSMUL_PREC_FP64)
    zs = batch.digits()
    rs1 = [type("R", (), {"status": s})() for s, _ in outs]
    ok1 = _verify_residues(batch, rs1, zs)
    out["fp64_one_at_a_time"] = {"s_total": el,
                                 "verified_digits_per_s": float(sum(batch.nz[i] for i in range(batch.count) if ok1[i])) / el,
                                 "residue_verified": int(ok1.sum())}
    for name in ("ladder_graph_batched", "ladder_fast_graph_batched"):
        out["speedup_" + name] = out[name]["verified_digits_per_s"] / \
            out["fp64_one_at_a_time"]["verified_digits_per_s"]
    print(json.dumps(out), flush=True)


def _uneven_batched(torch, abi, batch, max_n, prec, stream, seed, lanes=1):
    plan = abi.ssmul_plan(max_n, max_n, batch.count, prec, stream.cuda_stream)
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_GRAPH, 1)
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_LANES, lanes)
    abi.ssmul_debug_kernel_stats(plan, False)
    t = _time_batch(torch, plan, batch, 3, stream)
    _, kst = abi.ssmul_debug_kernel_stats(plan, False)
    # the same batch once more without the graph and with every launch timed:
    # the summed kernel time against the graph-replayed wall time shows how
    # much of a batched call the GPU spends outside the kernels
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_GRAPH, 0)
    abi.ssmul_debug_kernel_stats(plan, True)
    with torch.cuda.stream(stream):
        batch.run(plan)
        stream.synchronize()
    _, kt = abi.ssmul_debug_kernel_stats(plan, False)
    kernel_s = sum(ms for _, ms in kt.values()) / 1e3
    abi.ssmul_plan_destroy(plan)
    rs, zs = batch.results(), batch.digits()
    res_ok = _verify_residues(batch, rs, zs)
    rng = np.random.default_rng(seed)
    sample = sorted(rng.choice(batch.count, size=batch.count // 20, replace=False).tolist())
    full_ok = _verify_full(rs, zs, _expected(batch, sample))
    statuses = {}
    for r in rs:
        k = abi.status_string(r.status)
        statuses[k] = statuses.get(k, 0) + 1
    ver_digits = float(sum(batch.nz[i] for i in range(batch.count) if res_ok[i]))
    used = {}
    for r in rs:
        used[r.precision_used] = used.get(r.precision_used, 0) + 1
    return {
        "s_per_batch": t, "verified_digits_per_s": ver_digits / t, "statuses": statuses,
        "residue_verified": int(res_ok.sum()), "full_sample": len(sample),
        "full_sample_verified": full_ok, "precision_used": used,
        "launches_per_batch": {k: v[0] // 4 for k, v in kst.items() if v[0]},
        "kernel_s_per_batch": kernel_s, "kernel_time_fraction": kernel_s / t}


def split(args):
    torch = _torch()
    from oracle import exact as E
    from paper_1006_0405_gb300 import abi
    abi.load()
    part = 1 << 18
    rows = []
    for k in (19, 20, 21, 22):
        n = 1 << k
        a, b = synth.operand_pair(synth.SEED_BASE + 6, n, n)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        dz = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
        want = [E.residue(a, q) * E.residue(b, q) % q for q in PRIMES]
        for name, prec, split_m in (("fp64", abi.SSMUL_PREC_FP64, 0),
                                    ("fp64_split_2^18", abi.SSMUL_PREC_FP64, part),
                                    ("disc64", abi.SSMUL_PREC_DISC64, 0)):
            plan = abi.ssmul_plan(n, n, 0, prec, 0)
            if split_m:
                assert abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_SPLIT_DIGITS, split_m) == 0
            s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
            reps = 3
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                s, r = abi.ssmul_mul(plan, da.data_ptr(), n, db.data_ptr(), n, dz.data_ptr())
            el = (time.perf_counter() - t0) / reps
            abi.ssmul_plan_destroy(plan)
            z = dz.cpu().numpy()
            ok = bool(s == abi.SSMUL_OK and
                      all(E.residue(z, q) == w for q, w in zip(PRIMES, want)))
            rows.append({"digits": n, "method": name, "status": abi.status_string(s),
                         "max_width": r.max_width, "N": r.fft_odd << r.fft_log2,
                         "residue_verified": ok, "ms": 1e3 * el,
                         "verified_digits_per_s": (2 * n / el) if ok else 0.0})
    print(json.dumps({"report": "split", "part_digits": part, "rows": rows}), flush=True)


def run(args):
    {"sweep": sweep, "ladder": ladder, "uneven": uneven, "split": split}[args.workload](args)
