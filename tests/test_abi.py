"""The C-ABI library builds, loads and exports every declared symbol (no GPU needed)."""
import os
import re

import pytest

from paper_1006_0405_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ssmul_\w+)\s*\(", src))
    return names


def test_headers_declare_the_boundary():
    d = _declared()
    for name in ("ssmul_plan", "ssmul_mul", "ssmul_mul_batched", "ssmul_plan_destroy",
                 "ssmul_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = abi.load(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(abi.EXPORTS) == _declared()


def test_status_strings_without_device():
    assert abi.status_string(abi.SSMUL_OK) == "SSMUL_OK"
    assert abi.status_string(abi.SSMUL_TIMEOUT) == "SSMUL_TIMEOUT"
    assert abi.status_string(99) == "SSMUL_UNKNOWN_STATUS"


def test_plan_argument_checks_without_device():
    # rejected before any device work
    import ctypes
    h = ctypes.c_void_p()
    L = abi.load()
    assert L.ssmul_plan(None, 1, 1, 0, 0, None) == abi.SSMUL_INVALID_ARG
    assert L.ssmul_plan(ctypes.byref(h), 0, 1, 0, 0, None) == abi.SSMUL_INVALID_ARG
    assert L.ssmul_plan(ctypes.byref(h), 1, 1, 0, 99, None) == abi.SSMUL_INVALID_ARG
    assert L.ssmul_plan(ctypes.byref(h), 1 << 24, 1 << 24, 0, 0, None) == abi.SSMUL_TOO_LARGE
    assert L.ssmul_mul(None, None, 1, None, 1, None, None) == abi.SSMUL_INVALID_ARG
    assert L.ssmul_mul_batched_host(None, 0, None, None, None, None, None) == abi.SSMUL_INVALID_ARG
    assert L.ssmul_mul_noalloc(None, 1, None, 1, None, None, None) == abi.SSMUL_INVALID_ARG


def test_cpu_has_no_compute_path():
    import paper_1006_0405_gb300 as P
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(RuntimeError):
        P.Multiplier(10, 10)
