"""ctypes binding of the ssmul C ABI (include/ssmul.h, include/ssmul_debug.h).

Argument marshalling only: every step of the multiplication runs in the
CUDA library libssmul.so.  Loading fails loudly when the library is
missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

# ssmul_status
SSMUL_OK = 0
SSMUL_ISOLATION_FAILED = 1
SSMUL_CONTAINMENT_FAILED = 2
SSMUL_INVALID_ARG = 3
SSMUL_TOO_LARGE = 4
SSMUL_CUDA_ERROR = 5
SSMUL_OUT_OF_MEMORY = 6
SSMUL_TIMEOUT = 7
SSMUL_UNVERIFIED = 8

# ssmul_precision
SSMUL_PREC_FP64 = 0
SSMUL_PREC_FP32 = 1
SSMUL_PREC_LADDER = 2
SSMUL_PREC_DISC64 = 3
SSMUL_PREC_NAIVE64 = 4
SSMUL_PREC_LADDER_DISC = 5
SSMUL_PREC_DISC32X2 = 6
SSMUL_PREC_LADDER_FAST = 7
#: ssmul_debug_mul_intervals only: binary32 rectangles on 4-bit digits
SSMUL_DEBUG_PREC_FP32_NIBBLES = 100

#: every symbol the headers declare
EXPORTS = (
    "ssmul_plan", "ssmul_plan_set_option", "ssmul_mul", "ssmul_mul_host", "ssmul_mul_batched",
    "ssmul_mul_batched_host", "ssmul_mul_noalloc",
    "ssmul_plan_destroy", "ssmul_status_string",
    "ssmul_debug_twiddles", "ssmul_debug_mul_intervals", "ssmul_debug_ci_op", "ssmul_debug_disc_op",
    "ssmul_debug_ddisc_op", "ssmul_debug_isolate", "ssmul_debug_floor_ceil",
    "ssmul_debug_kernel_stats", "ssmul_debug_geometry", "ssmul_debug_set_fault",
    "ssmul_debug_pipe_rate",
)

# ssmul_option
SSMUL_OPT_GRAPH = 0
SSMUL_OPT_AUTOTUNE = 1
SSMUL_OPT_FP32_MAX_DIGITS = 2
SSMUL_OPT_BALANCED = 3
SSMUL_OPT_SPLIT_DIGITS = 4
SSMUL_OPT_LENGTHS = 5
SSMUL_OPT_HOST_PIECES = 6
SSMUL_OPT_LANES = 7
SSMUL_OPT_FP32_NIBBLES = 8

#: kernel kinds of ssmul_debug_kernel_stats, in index order
KERNEL_KINDS = tuple(f"{k}<{r}>" for k in ("k_small", "k_fwd_cols", "k_rows", "k_inv_cols")
                     for r in ("float", "double", "disc", "naive", "disc32x2")) + (
    "k_carry", "k_finalize", "k_prefix", "k_gate_list")


class ssmul_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("precision_used", ctypes.c_int32),
        ("fft_log2", ctypes.c_uint32),
        ("n_unisolated", ctypes.c_uint32),
        ("n_empty", ctypes.c_uint32),
        ("fft_odd", ctypes.c_uint32),
        ("max_width", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ssmul_desc(ctypes.Structure):
    _fields_ = [
        ("a_off", ctypes.c_uint64),
        ("b_off", ctypes.c_uint64),
        ("z_off", ctypes.c_uint64),
        ("na", ctypes.c_uint32),
        ("nb", ctypes.c_uint32),
    ]


_lib = None


class LibraryMissing(RuntimeError):
    pass


def load(path: str | None = None, build_if_missing: bool = True):
    """Load libssmul.so (building it first when absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if build_if_missing:
            try:
                _build.build()
            except Exception as e:  # no nvcc: fall through to the existence check
                if not os.path.exists(path):
                    raise LibraryMissing(f"libssmul.so could not be built: {e}") from e
    if not os.path.exists(path):
        raise LibraryMissing(f"CUDA library not found: {path}")
    L = ctypes.CDLL(path)
    vp, sz, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    L.ssmul_plan.argtypes = [ctypes.POINTER(vp), sz, sz, sz, ctypes.c_int, vp]
    L.ssmul_plan.restype = st
    L.ssmul_plan_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    L.ssmul_plan_set_option.restype = st
    L.ssmul_debug_geometry.argtypes = [vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    L.ssmul_debug_geometry.restype = st
    L.ssmul_debug_set_fault.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    L.ssmul_debug_set_fault.restype = st
    L.ssmul_mul.argtypes = [vp, vp, sz, vp, sz, vp, ctypes.POINTER(ssmul_result)]
    L.ssmul_mul.restype = st
    L.ssmul_mul_host.argtypes = [vp, vp, sz, vp, sz, vp, ctypes.POINTER(ssmul_result)]
    L.ssmul_mul_host.restype = st
    L.ssmul_mul_noalloc.argtypes = [vp, sz, vp, sz, vp, ctypes.POINTER(ssmul_result), vp]
    L.ssmul_mul_noalloc.restype = st
    L.ssmul_mul_batched.argtypes = [vp, sz, ctypes.POINTER(ssmul_desc), vp, vp, vp, vp]
    L.ssmul_mul_batched.restype = st
    L.ssmul_mul_batched_host.argtypes = [vp, sz, ctypes.POINTER(ssmul_desc), vp, vp, vp, vp]
    L.ssmul_mul_batched_host.restype = st
    L.ssmul_plan_destroy.argtypes = [vp]
    L.ssmul_plan_destroy.restype = None
    L.ssmul_status_string.argtypes = [ctypes.c_int]
    L.ssmul_status_string.restype = ctypes.c_char_p
    L.ssmul_debug_twiddles.argtypes = [vp, ctypes.c_int, vp, sz, ctypes.POINTER(ctypes.c_int)]
    L.ssmul_debug_twiddles.restype = st
    L.ssmul_debug_mul_intervals.argtypes = [vp, vp, sz, vp, sz, vp, ctypes.POINTER(ssmul_result),
                                            ctypes.c_int, vp]
    L.ssmul_debug_mul_intervals.restype = st
    L.ssmul_debug_ci_op.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, sz]
    L.ssmul_debug_ci_op.restype = st
    L.ssmul_debug_disc_op.argtypes = [ctypes.c_int, vp, vp, vp, sz]
    L.ssmul_debug_disc_op.restype = st
    L.ssmul_debug_ddisc_op.argtypes = [ctypes.c_int, vp, vp, vp, sz]
    L.ssmul_debug_ddisc_op.restype = st
    L.ssmul_debug_isolate.argtypes = [ctypes.c_int, vp, vp, vp, sz]
    L.ssmul_debug_isolate.restype = st
    L.ssmul_debug_floor_ceil.argtypes = [vp, vp, vp, sz]
    L.ssmul_debug_floor_ceil.restype = st
    L.ssmul_debug_kernel_stats.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
    L.ssmul_debug_kernel_stats.restype = st
    L.ssmul_debug_pipe_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.ssmul_debug_pipe_rate.restype = st
    _lib = L
    return L


def status_string(s: int) -> str:
    return load().ssmul_status_string(s).decode()


class SsmulError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)}")
        self.status = status


def _check(s: int, what: str):
    if s != SSMUL_OK:
        raise SsmulError(s, what)


# ---- the C calls, one Python function each -------------------------------------

def ssmul_plan(max_na: int, max_nb: int, max_products: int = 0,
               prec: int = SSMUL_PREC_FP64, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().ssmul_plan(ctypes.byref(h), max_na, max_nb, max_products, prec,
                             ctypes.c_void_p(stream or 0)), "ssmul_plan")
    return h.value


def ssmul_plan_set_option(plan: int, option: int, value: int) -> int:
    return load().ssmul_plan_set_option(ctypes.c_void_p(plan), option, value)


def ssmul_debug_set_fault(plan: int, kind: int, value: int = 0) -> int:
    return load().ssmul_debug_set_fault(ctypes.c_void_p(plan), kind, value)


def ssmul_debug_geometry(plan: int, log_n: int):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    s = load().ssmul_debug_geometry(ctypes.c_void_p(plan), log_n, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c))
    return s, (a.value, b.value, c.value)


def ssmul_plan_destroy(plan: int) -> None:
    load().ssmul_plan_destroy(ctypes.c_void_p(plan))


def ssmul_mul(plan: int, d_a: int, na: int, d_b: int, nb: int, d_z: int):
    """Returns (status, ssmul_result)."""
    r = ssmul_result()
    s = load().ssmul_mul(ctypes.c_void_p(plan), ctypes.c_void_p(d_a), na, ctypes.c_void_p(d_b),
                         nb, ctypes.c_void_p(d_z), ctypes.byref(r))
    return s, r


def ssmul_mul_host(plan: int, h_a: int, na: int, h_b: int, nb: int, h_z: int):
    r = ssmul_result()
    s = load().ssmul_mul_host(ctypes.c_void_p(plan), ctypes.c_void_p(h_a), na,
                              ctypes.c_void_p(h_b), nb, ctypes.c_void_p(h_z), ctypes.byref(r))
    return s, r


def ssmul_mul_noalloc(d_a: int, na: int, d_b: int, nb: int, d_z: int, stream: int | None = None):
    """The allocation-free product (na + nb <= 4097 digits).  Returns (status, ssmul_result)."""
    r = ssmul_result()
    s = load().ssmul_mul_noalloc(ctypes.c_void_p(d_a), na, ctypes.c_void_p(d_b), nb,
                                 ctypes.c_void_p(d_z), ctypes.byref(r), ctypes.c_void_p(stream or 0))
    return s, r


def ssmul_mul_batched(plan: int, descs, d_a_pool: int, d_b_pool: int, d_z_pool: int,
                      d_res: int) -> int:
    """descs: a ctypes array of ssmul_desc (or a sequence of 5-tuples)."""
    if not isinstance(descs, ctypes.Array):
        arr = (ssmul_desc * len(descs))()
        for i, (ao, bo, zo, na, nb) in enumerate(descs):
            arr[i] = ssmul_desc(ao, bo, zo, na, nb)
        descs = arr
    return load().ssmul_mul_batched(ctypes.c_void_p(plan), len(descs), descs,
                                    ctypes.c_void_p(d_a_pool), ctypes.c_void_p(d_b_pool),
                                    ctypes.c_void_p(d_z_pool), ctypes.c_void_p(d_res))


def ssmul_mul_batched_host(plan: int, descs, h_a_pool: int, h_b_pool: int, h_z_pool: int,
                           h_res) -> int:
    """Host pools in, host digits out.  descs: a ctypes array of ssmul_desc (or
    a sequence of 5-tuples); h_res: a ctypes array of len(descs) ssmul_result,
    or the address of host memory holding that many."""
    if not isinstance(descs, ctypes.Array):
        arr = (ssmul_desc * len(descs))()
        for i, (ao, bo, zo, na, nb) in enumerate(descs):
            arr[i] = ssmul_desc(ao, bo, zo, na, nb)
        descs = arr
    return load().ssmul_mul_batched_host(ctypes.c_void_p(plan), len(descs), descs,
                                         ctypes.c_void_p(h_a_pool), ctypes.c_void_p(h_b_pool),
                                         ctypes.c_void_p(h_z_pool),
                                         ctypes.c_void_p(h_res if isinstance(h_res, int)
                                                         else ctypes.addressof(h_res)))


def ssmul_debug_twiddles(plan: int, f32: int, h_out: int, cap: int):
    """f32: bit 0 binary32, bit 1 the table of the lengths 3 2^k, bit 2 of 5 2^k."""
    ln = ctypes.c_int()
    s = load().ssmul_debug_twiddles(ctypes.c_void_p(plan), int(f32), ctypes.c_void_p(h_out), cap,
                                    ctypes.byref(ln))
    return s, ln.value


def ssmul_debug_mul_intervals(plan: int, d_a: int, na: int, d_b: int, nb: int, d_z: int,
                              prec: int, d_iv: int):
    r = ssmul_result()
    s = load().ssmul_debug_mul_intervals(ctypes.c_void_p(plan), ctypes.c_void_p(d_a), na,
                                         ctypes.c_void_p(d_b), nb, ctypes.c_void_p(d_z),
                                         ctypes.byref(r), prec, ctypes.c_void_p(d_iv))
    return s, r


def ssmul_debug_disc_op(op: int, d_x: int, d_y: int, d_out: int, n: int) -> int:
    return load().ssmul_debug_disc_op(op, ctypes.c_void_p(d_x), ctypes.c_void_p(d_y),
                                      ctypes.c_void_p(d_out), n)


def ssmul_debug_isolate(path: int, d_x: int, d_value: int, d_class: int, n: int) -> int:
    return load().ssmul_debug_isolate(path, ctypes.c_void_p(d_x), ctypes.c_void_p(d_value),
                                      ctypes.c_void_p(d_class), n)


def ssmul_debug_floor_ceil(d_x: int, d_k: int, d_out: int, n: int) -> int:
    return load().ssmul_debug_floor_ceil(ctypes.c_void_p(d_x), ctypes.c_void_p(d_k),
                                         ctypes.c_void_p(d_out), n)


def ssmul_debug_ddisc_op(op: int, d_x: int, d_y: int, d_out: int, n: int) -> int:
    return load().ssmul_debug_ddisc_op(op, ctypes.c_void_p(d_x), ctypes.c_void_p(d_y),
                                       ctypes.c_void_p(d_out), n)


def ssmul_debug_ci_op(op: int, f32: bool, d_x: int, d_y: int, d_out: int, n: int) -> int:
    return load().ssmul_debug_ci_op(op, int(f32), ctypes.c_void_p(d_x), ctypes.c_void_p(d_y),
                                    ctypes.c_void_p(d_out), n)


def ssmul_debug_kernel_stats(plan: int, enable: bool):
    """Returns (status, {kind: (launches, ms)}) since the previous call."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    la = (ctypes.c_ulonglong * n)()
    s = load().ssmul_debug_kernel_stats(ctypes.c_void_p(plan), int(enable), ms, la, n)
    return s, {KERNEL_KINDS[i]: (int(la[i]), float(ms[i])) for i in range(n)}


#: operations of ssmul_debug_pipe_rate, in index order
PIPE_OPS = ("f64_add_rd", "f64_mul_ru", "f64_fma_rd", "f64_add_as_fma_rd", "f64_add_rn",
            "f32_add_rd", "f32_fma_rd")


def ssmul_debug_pipe_rate(op: int):
    """Returns (status, G operations per second) of one arithmetic operation."""
    g = ctypes.c_double()
    s = load().ssmul_debug_pipe_rate(op, ctypes.byref(g))
    return s, g.value
