"""Benchmark: verified interval-FFT multiplications on one GB300 (or N replicas).

Workload (default): the paper-scale binary64 interval method, products of
two 75,000-digit base-256 operands (FFT length 5 2^15).  One step is one
ssmul_mul_batched call over a batch of B such products (B - 1 with uniform
random digits, one with every digit 0xFF, the worst case of coefficient
size), i.e. one pass of the whole path: interval transforms, pointwise
products, isolation and the carry scan.  Metric: verified multiplies/s
(status OK and digits equal to the CPU oracle, checked after timing).

Contract: `python bench.py --gpus N --steps K --warmup W` prints one JSON
line on rank 0.  Under torchrun every rank runs its own batch (products are
independent: weak scaling, no collective on the data path); value = all
products of all ranks / the slowest rank's time.  `--impl reference` times
the CPU oracle (long multiplication, Section 2.1) on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "verified multiplies/s at 75k base-256 digits"


def _hbm_peak() -> float:
    """Measured HBM copy bandwidth (GB/s) of the GB300s, else the
    fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak()
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=256,
                    help="products per step (every 64th all-0xFF, the rest uniform)")
    ap.add_argument("--digits", type=int, default=75000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="time budget of the CPU oracle sample")
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "disc64", "naive64", "disc32x2", "ladder_fast"],
                    help="rung of the paper workload: binary64 rectangles (default), binary64 "
                         "discs, the unverified naive transform, double-binary32 discs, or the "
                         "fast ladder (double-binary32 discs, escalating to binary64)")
    ap.add_argument("--lanes", type=int, default=4,
                    help="streams over which batched calls spread their length groups "
                         "(SSMUL_OPT_LANES)")
    ap.add_argument("--host-pieces", type=int, default=4,
                    help="pieces of the end-to-end host-buffer call (SSMUL_OPT_HOST_PIECES)")
    ap.add_argument("--no-alternates", action="store_true",
                    help="skip the extra lines for the other rungs (disc64, naive64)")
    ap.add_argument("--balanced", action="store_true",
                    help="balanced digits (the transforms carry digit - 128)")
    ap.add_argument("--lengths", type=int, default=3, choices=[0, 1, 2, 3],
                    help="transform length families besides 2^k (SSMUL_OPT_LENGTHS bit mask: "
                         "1 = 3 2^k, 2 = 5 2^k)")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "c1", "sweep", "ladder", "uneven", "split", "probe"],
                    help="paper: the headline line (with the c1, c3, c4 and c5 reports unless "
                         "--no-reports); c1 / sweep / ladder / uneven / split: one report line "
                         "(one 4096-digit product, the size sweep, the precision ladder, the "
                         "uneven batch, the products past the isolation limit)")
    ap.add_argument("--autotune", action="store_true",
                    help="time the candidate four-step geometries of the plan's lengths first "
                         "(SSMUL_OPT_AUTOTUNE), outside every timed region")
    ap.add_argument("--no-reports", action="store_true",
                    help="headline line only (no c1 / c3 / c4 / c5 reports)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- workload ---------------------------------------------------------------

def make_batch(rank: int, batch: int, n: int):
    seed = synth.SEED_BASE + 1 + 1000 * rank
    # one product in 64 (and the last of a smaller batch) has all digits 0xFF
    dists = ["ff" if i % 64 == 63 or i == batch - 1 else "uniform" for i in range(batch)]
    na = [n] * batch
    return synth.batch_operands(seed, na, na, dists), dists


# ---- algorithmic work model ------------------------------------------------------
#
# binary64 operations of each building block: rectangles (inf-sup, 4 per
# complex add, 8 per twiddle product, 12 per general product, 4 to scale,
# 1 per coefficient width) and discs / points (2, 4, 4, 2; isolation of a
# disc: 2 bounds + 1 width per coefficient)
COSTS = {
    # stw: a product by a real or pure imaginary scalar (radix-3, radix-5);
    # scale 0: the rectangles and binary64 discs fold the 1/N scaling into
    # the isolation's integer conversion
    "fp64": dict(add=4, bfly=32, tw=8, stw=4, mul=12, scale=0, iso=1),
    "disc64": dict(add=2, bfly=16, tw=4, stw=2, mul=4, scale=0, iso=3),
    "naive64": dict(add=2, bfly=16, tw=4, stw=2, mul=4, scale=2, iso=0),
    # double-binary32 discs count binary32 operations: a pair sum is TwoSum,
    # two adds and FastTwoSum (11); a complex add is two pair sums and its
    # radius (2 x 11 + 6); the radix-4 butterfly's eight sums share one
    # radius (8 x 22 + 13); a twiddle product is four pair products (4 x 7),
    # two pair sums and 5 radius operations (the terms in the table's radius
    # alone are loop invariants); a general product 28 + 22 + 10; the binary32
    # isolation of a component 12 (two roundings to integers, the
    # remainders' sum and its bounds, the width, two magic-number roundings);
    # a product by a real or imaginary scalar is two pair products and 5
    # radius operations
    "disc32x2": dict(add=28, bfly=189, tw=55, stw=19, mul=60, scale=6, iso=12),
}
TAGS = {"fp64": "double", "disc64": "disc", "naive64": "naive", "disc32x2": "disc32x2"}
SETS = {"fp64": "binary64 inf-sup intervals", "disc64": "binary64 midpoint-radius discs",
        "naive64": "unverified binary64 points", "disc32x2": "double-binary32 midpoint-radius discs",
        "ladder_fast": "ladder of double-binary32 then binary64 discs"}


def _fft_ops(logL: int, nl: int, c: dict, exact_first: bool = False) -> int:
    """exact_first: the first step's 4-point sums are integer arithmetic on
    the digits (forward column transforms), only its twiddle products count"""
    L = 1 << logL
    ops = 0
    logn, logs = logL, 0
    while logn >= 2:
        s = 1 << logs
        sums = 0 if (exact_first and logs == 0) else nl * (L // 4) * c["bfly"]
        ops += sums + nl * (L // 4 - s) * 3 * c["tw"]
        logn -= 2
        logs += 2
    if logn == 1:
        ops += nl * (L // 2) * 2 * c["add"]
    return ops


def _fft_odd_ops(R: int, loga: int, nl: int, c: dict, exact_first: bool = False) -> int:
    """lines of length R 2^loga (R = 3 or 5, loga even): radix-4 steps, then
    one radix-R step: radix 3 = 6 adds, a scaling by 1/2 and one product by
    a pure imaginary scalar per butterfly; radix 5 = 14 adds and 8 products
    by a real or pure imaginary scalar"""
    L = R << loga
    ops = 0
    logn2, logs = loga, 0
    while logn2 >= 2:
        s = 1 << logs
        sums = 0 if (exact_first and logs == 0) else nl * (L // 4) * c["bfly"]
        ops += sums + nl * (L // 4 - s) * 3 * c["tw"]
        logn2 -= 2
        logs += 2
    last = (6 * c["add"] + c["scale"] + c["stw"]) if R == 3 else (14 * c["add"] + 8 * c["stw"])
    return ops + nl * (L // R) * last


LENGTHS = 3          # SSMUL_OPT_LENGTHS of the plans this run makes


def length_code(na: int, nb: int, mask: int | None = None) -> tuple[int, int]:
    """(R, k): the transform length R 2^k the library picks under the
    length mask (default: this run's)."""
    mask = LENGTHS if mask is None else mask
    L = na + nb - 1
    k = max(2, (L - 1).bit_length())
    if mask & 2 and 10 <= k - 3 <= 19 and (5 << (k - 3)) >= L:
        return 5, k - 3
    if mask & 1 and 11 <= k - 2 <= 21 and (3 << (k - 2)) >= L:
        return 3, k - 2
    return 1, k


def geometry(R: int, k: int):
    """(log2 N1 / R, log2 N2, log2 C1, log2 C3) of the default four-step split"""
    if R == 1:
        b = min((k + 1) // 2, 11)
        a = k - b
        c = max(0, 11 - a)
    else:
        amax = 10 if R == 3 else 8
        b = (k + 1) // 2
        a = k - b
        if a & 1:
            a, b = a - 1, b + 1
        while b > 11:
            a, b = a + 2, b - 2
        while a > amax:
            a, b = a - 2, b + 2
        c = max(0, 10 - a - (1 if R == 3 else 2))
    return a, b, min(c, b), min(c, b - 1)


def kernel_ops(na: int, nb: int, precision: str = "fp64") -> dict:
    """arithmetic operations per product of each four-step kernel (N > 4096):
    radix-4 butterfly (8 adds) + 3 twiddle products unless p = 0; radix-2 =
    2 adds; radix-3 and radix-5 as in _fft_odd_ops; pair product =
    2 adds + 1 general product; packing = 3 adds + 1 twiddle product;
    four-step twiddles; scaling and isolation."""
    c = COSTS[precision]
    tag = TAGS[precision]
    R, k = length_code(na, nb)
    n1l, n2l, c1l, c3l = geometry(R, k)
    N1, N2 = R << n1l, 1 << n2l
    M2 = N2 // 2
    def col(nl, exact_first=False):
        if R == 1:
            return _fft_ops(n1l, nl, c, exact_first and n1l >= 2)
        return _fft_odd_ops(R, n1l, nl, c, exact_first)
    fwd = (N2 >> c1l) * col(1 << c1l, True) + (N1 - 1) * (N2 - 1) * c["tw"]
    rows = 0
    for k1 in range(N1 // 2 + 1):
        nl = 1 if k1 == (N1 - k1) % N1 else 2
        rows += _fft_ops(n2l, nl, c) + _fft_ops(n2l - 1, nl, c)
        rows += (nl * N2 // 2) * (2 * c["add"] + c["mul"]) + nl * M2 * (3 * c["add"] + c["tw"])
        rows += nl * (M2 - 1) * c["tw"] if k1 else 0
    inv = (M2 >> c3l) * col(1 << c3l) + (N1 * M2) * (c["scale"] + 2 * c["iso"])
    return {f"k_fwd_cols<{tag}>": fwd, f"k_rows<{tag}>": rows, f"k_inv_cols<{tag}>": inv}


# DRAM bytes per product of one launch of the dominant kernels, from ncu
# captures (16 products of 75k x 75k digits per launch, spectra larger than
# L2): dram__bytes_read.sum + dram__bytes_write.sum divided by 16.  They hold
# only for the kernel sources they were captured with (the hash of the
# device headers csrc/*.cuh) and the four-step geometry of the 75k length
# (log2(N1 / 5), log2 N2, log2 column CTA elements); the bench checks both
# at run time and reports null traffic when either differs.
NCU_TRAFFIC = {
    "cuh_sha256_16": "749fe2a5f42a1d8c",
    "geometry_75k": (6, 9, 10),
    "per_product": {
        "k_rows<double>": (84.413696e6 + 9.755648e6) / 16,
        "k_rows<disc>": (63.517952e6 + 3.389696e6) / 16,
        "k_rows<disc32x2>": (63.329536e6 + 4.898816e6) / 16,
    },
}

def kernel_source_hash() -> str:
    """sha256 (first 16 hex digits) of the device headers the kernels are built from."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1006_0405_gb300", "csrc", "*.cuh"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str, n: int, geometry) -> tuple:
    """(bytes per product, why) of the ncu capture, or (None, reason) when the
    workload, the kernel sources or the geometry differ from the captured ones."""
    if n != 75000 or kernel not in NCU_TRAFFIC["per_product"]:
        return None, "no ncu capture of this kernel at this size"
    if kernel_source_hash() != NCU_TRAFFIC["cuh_sha256_16"]:
        return None, "kernel sources changed since the ncu capture"
    if tuple(geometry) != NCU_TRAFFIC["geometry_75k"]:
        return None, "four-step geometry differs from the ncu capture"
    return NCU_TRAFFIC["per_product"][kernel], "ncu capture of the same kernel sources and geometry"


def algorithmic_bytes(n: int) -> float:
    """HBM bytes one product's passes must move at minimum (binary64
    rectangles, N = 5 2^15 for 75k digits): digits in, Z written and read,
    W written and read, coefficients written and read, digits out."""
    R, k = length_code(n, n)
    N = R << k
    return 2 * n + 32 * N * 2 + 16 * N * 2 + 8 * N * 2 + 2 * n


def fft_len_str(n: int) -> str:
    R, k = length_code(n, n)
    return f"2^{k}" if R == 1 else f"{R}*2^{k}"


def pipe_rates() -> dict:
    """Measured throughput (G operations/s) of each operation of the
    library's pipe probe (ssmul_debug_pipe_rate): the ceilings the kernels'
    operation mixes run against, beside the nominal peaks."""
    from paper_1006_0405_gb300 import abi
    out = {}
    for i, name in enumerate(abi.PIPE_OPS):
        st, g = abi.ssmul_debug_pipe_rate(i)
        out[name] = g if st == abi.SSMUL_OK else None
    return out


def run_probe(args):
    import torch
    from paper_1006_0405_gb300 import abi
    if not torch.cuda.is_available():
        raise SystemExit("the probe needs a CUDA device")
    abi.load()
    prop = torch.cuda.get_device_properties(0)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    rates = pipe_rates()
    t1 = time.perf_counter()
    clk = clocks.stop(t0, t1)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    print(json.dumps({"report": "pipe_probe", "device": prop.name, "sms": prop.multi_processor_count,
                      "gops": rates, "clocks": clk,
                      "nominal_gops": {"f64": fp64_peak_gops(sm_mhz, prop.multi_processor_count),
                                       "f32": fp32_peak_gops(sm_mhz, prop.multi_processor_count)}}),
          flush=True)


def fp64_peak_gops(sm_mhz: float, sms: int) -> float:
    """sms SMs x 2 binary64 operations per clock (GB300's nominal 1.25 TFLOP/s
    counts an fma as 2 flops: 152 SMs * 2 * 2 * 2.07 GHz)."""
    return sms * 2 * sm_mhz * 1e6 / 1e9


def fp32_peak_gops(sm_mhz: float, sms: int) -> float:
    """sms SMs x 128 binary32 lanes per clock."""
    return sms * 128 * sm_mhz * 1e6 / 1e9


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between t0 and t1 (perf_counter
        seconds; sampling lags by up to one period, so the window is widened
        by 0.15 s at its end); all samples when no window is given."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for t, ln in self.lines
                 if t0 is None or (t0 <= t <= t1 + 0.15)]
        if not lines and self.lines:
            # nearest sample to the window
            lines = [min(self.lines, key=lambda x: abs(x[0] - (t0 or 0)))[1]]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- multi-rank aggregation -------------------------------------------------------

def aggregate_ranks(step_seconds: float, verified: int, e2e_seconds: float, products: int,
                    world: int, device):
    """Whole-job numbers from every rank's own measurement (products are
    independent: no collective on the data path, only these three numbers):
    value = all verified products / the slowest rank's timed seconds,
    e2e = all products / the slowest rank's end-to-end seconds per step."""
    if world == 1:
        return verified / step_seconds, products / e2e_seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([step_seconds, float(verified), e2e_seconds], dtype=torch.float64,
                     device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return sm[1].item() / mx[0].item(), world * products / mx[2].item()


# ---- CPU oracle ---------------------------------------------------------------

def cpu_oracle_rate(n: int, budget_s: float, rank: int = 0):
    """Products/s of the CPU oracle (long multiplication: exact convolution
    sums of Section 2.1 and the carry of Section 2.4) on the host cores."""
    from oracle import exact as E
    E.lib()
    (a_pool, b_pool, a_off, b_off, _), _ = make_batch(rank, 2, n)
    a, b = a_pool[:n], b_pool[:n]
    done, t0 = 0, time.perf_counter()
    while True:
        E.product(a, b)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return done / el, done, el, E.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import exact as E
    E.lib()
    n = args.digits
    (a_pool, b_pool, *_), _ = make_batch(0, 2, n)
    a, b = a_pool[:n], b_pool[:n]
    for _ in range(args.warmup):
        E.product(a, b)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E.product(a, b)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "multiplies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{n}x{n} base-256 digits, uniform bytes; CPU oracle "
                               f"long multiplication, one product per step"},
        "cpu_baseline": {"value": v, "unit": "multiplies/s", "cores": E.num_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} products of {n}x{n} digits"},
        "e2e": {"value": v, "unit": "multiplies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- our arm --------------------------------------------------------------------

def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device; the GPU path has no CPU fallback")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_1006_0405_gb300 import abi
    abi.load()
    n, B = args.digits, args.batch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    (a_pool, b_pool, a_off, b_off, z_off), dists = make_batch(rank, B, n)
    nz = 2 * n
    stream = torch.cuda.Stream(device=dev)
    PRECS = {"fp64": abi.SSMUL_PREC_FP64, "disc64": abi.SSMUL_PREC_DISC64,
             "naive64": abi.SSMUL_PREC_NAIVE64, "disc32x2": abi.SSMUL_PREC_DISC32X2,
             "ladder_fast": abi.SSMUL_PREC_LADDER_FAST}
    prec = PRECS[args.precision]
    t_plan = time.perf_counter()
    plan = abi.ssmul_plan(n, n, B, prec, stream.cuda_stream)
    stream.synchronize()
    plan_first_ms = 1e3 * (time.perf_counter() - t_plan)
    abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_HOST_PIECES, args.host_pieces)
    if args.balanced:
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_BALANCED, 1)
    if args.lengths != 3:
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_LENGTHS, args.lengths)
    if args.autotune:
        abi.ssmul_plan_set_option(plan, abi.SSMUL_OPT_AUTOTUNE, 1)
    descs = (abi.ssmul_desc * B)()
    for i in range(B):
        descs[i] = abi.ssmul_desc(int(a_off[i]), int(b_off[i]), int(z_off[i]), n, n)
    da = torch.from_numpy(a_pool).to(dev)
    db = torch.from_numpy(b_pool).to(dev)
    dz = torch.zeros(B * nz, dtype=torch.uint8, device=dev)
    res_bytes = ctypes.sizeof(abi.ssmul_result) * B
    dres = torch.zeros(res_bytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step(z_target=None, r_target=None):
        s = abi.ssmul_mul_batched(plan, descs, da.data_ptr(), db.data_ptr(),
                                  (z_target if z_target is not None else dz).data_ptr(),
                                  (r_target if r_target is not None else dres).data_ptr())
        if s != abi.SSMUL_OK:
            raise RuntimeError(abi.status_string(s))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        zs = [torch.empty_like(dz) for _ in range(args.steps)]
        rs = [torch.empty_like(dres) for _ in range(args.steps)]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        abi.ssmul_debug_kernel_stats(plan, True)        # reset; time kernels from here
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.5)                                   # sampler running before timing
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                                 # L2 flushed between timed steps
            ev[k][0].record(stream)
            step(zs[k], rs[k])
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t_end = time.perf_counter()
        wall = t_end - t_wall
        clk = clocks.stop(t_wall, t_end)
        _, kstats = abi.ssmul_debug_kernel_stats(plan, False)
        step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]

    torch.cuda.synchronize()

    # the exact products, from the CPU oracle (NTT convolution and carry)
    from oracle import exact as E
    expect = []
    for i in range(B):
        a = a_pool[a_off[i]:a_off[i] + n]
        b = b_pool[b_off[i]:b_off[i] + n]
        expect.append(E.carry(E.conv_ntt(a, b), nz))

    # end to end through the library's host-buffer call: every step hands
    # the operands in page-locked host memory to ssmul_mul_batched_host,
    # which uploads them, runs the batch in pieces whose copies overlap the
    # computation, and returns once the digits and outcomes are back in host
    # memory; each step is timed on the host around that call (it waits)
    ha = torch.from_numpy(a_pool).pin_memory()
    hb = torch.from_numpy(b_pool).pin_memory()
    hz = torch.empty(B * nz, dtype=torch.uint8).pin_memory()
    hres = torch.empty(res_bytes, dtype=torch.uint8).pin_memory()
    e2e_steps = max(4, min(args.steps, 12))
    e2e_times, e2e_ok = [], True

    def host_step():
        s_ = abi.ssmul_mul_batched_host(plan, descs, ha.data_ptr(), hb.data_ptr(), hz.data_ptr(),
                                        hres.data_ptr())
        if s_ != abi.SSMUL_OK:
            raise RuntimeError(abi.status_string(s_))

    with torch.cuda.stream(stream):
        host_step()                                   # warm-up: the plan's device copies grow
        for k in range(e2e_steps):
            hz.zero_()
            flush.zero_()                             # L2 flushed between steps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_step()
            e2e_times.append(time.perf_counter() - t0)
            rr = (abi.ssmul_result * B)()
            ctypes.memmove(rr, hres.numpy().ctypes.data, res_bytes)
            zh = hz.numpy()
            e2e_ok &= all(rr[i].status == abi.SSMUL_OK and
                          np.array_equal(zh[z_off[i]:z_off[i] + nz], expect[i]) for i in range(B))
    e2e_s = sum(e2e_times) / len(e2e_times)

    # verification of every timed step against the CPU oracle: a product is
    # verified when its status is SSMUL_OK and its digits are the oracle's
    # (the naive transform's digits can match without being verified)
    verified, matched = 0, 0
    widths = []
    statuses = {}
    for k in range(args.steps):
        z = zs[k].cpu().numpy()
        rr = (abi.ssmul_result * B)()
        host = rs[k].cpu().numpy()
        ctypes.memmove(rr, host.ctypes.data, res_bytes)
        for i in range(B):
            st = rr[i].status
            statuses[abi.status_string(st)] = statuses.get(abi.status_string(st), 0) + 1
            same = bool(np.array_equal(z[z_off[i]:z_off[i] + nz], expect[i]))
            verified += int(st == abi.SSMUL_OK and same)
            matched += int(same)
            if k == 0:
                widths.append((dists[i], rr[i].max_width))

    # the other rungs on the same batch (context for the headline rung)
    alternatives = {}
    if world == 1 and not args.no_alternates:
        for alt in ("fp64", "disc64", "naive64", "disc32x2", "ladder_fast"):
            if alt == args.precision:
                continue
            aplan = abi.ssmul_plan(n, n, B, PRECS[alt], stream.cuda_stream)
            if args.balanced:
                abi.ssmul_plan_set_option(aplan, abi.SSMUL_OPT_BALANCED, 1)
            if args.lengths != 3:
                abi.ssmul_plan_set_option(aplan, abi.SSMUL_OPT_LENGTHS, args.lengths)
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    s_ = abi.ssmul_mul_batched(aplan, descs, da.data_ptr(), db.data_ptr(),
                                               dz.data_ptr(), dres.data_ptr())
                stream.synchronize()
                abi.ssmul_debug_kernel_stats(aplan, True)
                aev = []
                for k in range(args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s_ = abi.ssmul_mul_batched(aplan, descs, da.data_ptr(), db.data_ptr(),
                                               zs[k].data_ptr(), rs[k].data_ptr())
                    e1.record(stream)
                    aev.append((e0, e1))
                stream.synchronize()
                _, akst = abi.ssmul_debug_kernel_stats(aplan, False)
            abi.ssmul_plan_destroy(aplan)
            a_ok, a_match, a_w = 0, 0, 0.0
            for k in range(args.steps):
                z = zs[k].cpu().numpy()
                rr = (abi.ssmul_result * B)()
                host = rs[k].cpu().numpy()
                ctypes.memmove(rr, host.ctypes.data, res_bytes)
                for i in range(B):
                    same = bool(np.array_equal(z[z_off[i]:z_off[i] + nz], expect[i]))
                    a_ok += int(rr[i].status == abi.SSMUL_OK and same)
                    a_match += int(same)
                    a_w = max(a_w, rr[i].max_width)
            a_t = sum(e0.elapsed_time(e1) for e0, e1 in aev) / 1e3
            amodel = "disc32x2" if alt == "ladder_fast" else alt
            aops = kernel_ops(n, n, amodel)
            adom = max(aops, key=lambda kk: akst.get(kk, (0, 0.0))[1])
            ala, ams = akst[adom]
            aach = aops[adom] * B / (ams / ala * 1e-3) / 1e9 if ala else 0.0
            alternatives[alt] = {
                "value": a_ok / a_t, "unit": "verified multiplies/s",
                "ms_per_step": 1e3 * a_t / args.steps,
                "verified": f"{a_ok}/{args.steps * B}", "max_width": a_w,
                "dominant_kernel": adom,
                ("fp32_gops" if amodel == "disc32x2" else "fp64_gops"): aach}
            if alt == "naive64":
                # never verified (status SSMUL_UNVERIFIED): its speed is that of
                # the products whose digits happened to equal the oracle's
                alternatives[alt]["unverified_digits_matched"] = f"{a_match}/{args.steps * B}"
                alternatives[alt]["unverified_multiplies_per_s"] = a_match / a_t

    # the other configurations of the method, each verified bit-exact against
    # the oracle (single GPU only: they are reports, not the weak-scaled step)
    reports = None
    if world == 1 and not args.no_reports:
        import bench_reports
        ctx = bench_reports.Ctx(lanes=args.lanes)
        t_rep = time.perf_counter()
        try:
            reports = {"c1": bench_reports.c1(ctx), "c3": bench_reports.c3(ctx),
                       "c4": bench_reports.c4(ctx), "c5": bench_reports.c5(ctx)}
        finally:
            ctx.close()
        reports["wall_s"] = time.perf_counter() - t_rep

    t_steps = sum(step_ms) / 1e3
    value, e2e_value = aggregate_ranks(t_steps, verified, e2e_s, B, world, dev)
    if not e2e_ok:
        e2e_value = 0.0

    if rank == 0:
        # roofline of the dominant kernel: binary64 pipe (an ALU bound)
        model = "disc32x2" if args.precision == "ladder_fast" else args.precision
        ops = kernel_ops(n, n, model)
        dom = max(ops, key=lambda k: kstats.get(k, (0, 0.0))[1])
        launches, ms = kstats[dom]
        # one launch covers all B products of the batch
        achieved = ops[dom] * B / (ms / launches * 1e-3) / 1e9 if launches else 0.0
        sm_mhz = clk.get("sm_mhz") or 2070.0
        peak = (fp32_peak_gops(sm_mhz, sms) if model == "disc32x2"
                else fp64_peak_gops(sm_mhz, sms))
        R_, k_ = length_code(n, n)
        geo = abi.ssmul_debug_geometry(plan, (64 if R_ == 5 else 32 if R_ == 3 else 0) + k_)[1]
        traffic_pp, traffic_why = captured_traffic(dom, n, geo)
        rates = pipe_rates() if world == 1 else None
        total_ms = sum(v[1] for v in kstats.values())
        shares = {k: round(v[1] / total_ms, 4) for k, v in kstats.items() if v[0]}
        cpu = None
        if world == 1:
            cpu_v, cpu_n, cpu_el, cores = cpu_oracle_rate(n, args.cpu_seconds)
            cpu = {"value": cpu_v, "unit": "multiplies/s", "cores": cores, "kind": "oracle",
                   "sample": f"{cpu_n} products of {n}x{n} digits in {cpu_el:.1f} s "
                             f"(long multiplication + carry)"}
        gpu_launches = sum(v[0] for v in kstats.values())
        # plan creation (twiddle tables, workspace) outside every timed region: the first
        # plan of the process (module load included), then the same plan again
        t_plan = time.perf_counter()
        plan2 = abi.ssmul_plan(n, n, B, prec, stream.cuda_stream)
        stream.synchronize()
        plan_warm_ms = 1e3 * (time.perf_counter() - t_plan)
        abi.ssmul_plan_destroy(plan2)
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "multiplies/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t_steps / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"disc32x2": "f32", "ladder_fast": "f32+f64"}.get(args.precision, "f64"),
            "precision": args.precision,
            "balanced_digits": bool(args.balanced),
            "data": "synthetic",
            "config": {"workload": f"{n}x{n} base-256 digits, {SETS[args.precision]}, "
                                   f"FFT length {fft_len_str(n)}; batch of {B} per step "
                                   f"({dists.count('uniform')} uniform random, {dists.count('ff')} "
                                   f"all-0xFF) per GPU",
                       "batch_per_gpu": B, "digits": n, "precision": args.precision,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas x{world}",
                       "geometry": {"log_n1": geo[0], "log_n2": geo[1], "log_cta": geo[2],
                                    "autotuned": bool(args.autotune)}},
            "verified": f"{verified}/{args.steps * B} per rank 0",
            "digits_matched": f"{matched}/{args.steps * B} per rank 0",
            "statuses": statuses,
            "max_width": {"uniform": max(w for d, w in widths if d == "uniform"),
                          "all_ff": max((w for d, w in widths if d == "ff"), default=None)},
            "e2e": {"value": e2e_value, "unit": "multiplies/s",
                    "h2d_bytes_per_step": int(a_pool.nbytes + b_pool.nbytes + ctypes.sizeof(descs)),
                    "d2h_bytes_per_step": int(B * nz + res_bytes),
                    "call": "ssmul_mul_batched_host (page-locked host pools in, host digits out)",
                    "host_pieces": int(args.host_pieces), "steps": e2e_steps,
                    "verified": "all" if e2e_ok else "not all products SSMUL_OK and exact"},
            "gpu_launches": int(gpu_launches),
            "alternatives": alternatives,
            "kernel_ms_share": shares,
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "fp32 Gop/s" if model == "disc32x2" else "fp64 Gop/s",
                         "frac": achieved / peak,
                         "traffic": traffic_pp * B if traffic_pp is not None else None,
                         "traffic_note": "bytes per launch: ncu DRAM bytes of a 16-product launch "
                                         "scaled to the B products of this launch; " + traffic_why,
                         "peak_note": (f"binary32 pipe: {sms} SMs x 128 lanes/clk"
                                       if model == "disc32x2" else
                                       f"binary64 pipe: {sms} SMs x 2 ops/clk")
                                      + " at the median sampled SM clock (recipe unit counts "
                                        "and clocks)",
                         "measured_op_gops": rates},
            "hbm_roofline": {"achieved_gbs": value * algorithmic_bytes(n) / 1e9,
                             "peak_gbs": HBM_PEAK_GBS,
                             "frac": value * algorithmic_bytes(n) / 1e9 / HBM_PEAK_GBS,
                             "note": "minimum pass traffic per product x products/s over the "
                                     "measured copy bandwidth; the path is arithmetic-pipe "
                                     "bound"},
            "cpu_baseline": cpu,
            "plan_ms": {"first_in_process": plan_first_ms, "warm": plan_warm_ms},
            "reports": reports,
            "clocks": clk,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    abi.ssmul_plan_destroy(plan)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    global LENGTHS
    args = parse()
    LENGTHS = args.lengths
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "probe":
        run_probe(args)
    elif args.workload == "paper":
        run_ours(args)
    else:
        import bench_reports
        bench_reports.run(args)


if __name__ == "__main__":
    main()
