"""Exact integer oracle: digits, convolution coefficients, carry, residues.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Functions and the passage each follows:
  long_mul(x, y)       Section 2.1, the long multiplication algorithm
  conv(x, y)           Section 2.1, c_i = sum_j x_j y_{i-j}
  conv_ntt(x, y)       exact convolution by an NTT mod 2^64-2^32+1 (a library-
                       style primitive used for sizes where conv is too slow)
  carry(c, nz)         Section 2.4, the carry loop of the SS algorithm
  product(x, y)        conv (or conv_ntt) followed by carry
  residue(x, p)        x mod p by Horner's rule
  to_int / from_int    Section 2 digit convention, via Python integers

Pins (tests/test_oracle_exact.py): brute force against Python's own integer
product, exhaustive 1x1 and 1x2 digit cases, residues mod four primes, the
all-0xFF closed forms, the DC and alternating-sum invariants, shifts by b^k.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        sz = ctypes.c_size_t
        L.oracle_long_mul.argtypes = [u8p, sz, u8p, sz, u8p]
        L.oracle_conv.argtypes = [u8p, sz, u8p, sz, u64p]
        L.oracle_conv_ntt.argtypes = [u8p, sz, u8p, sz, u64p]
        L.oracle_carry.argtypes = [u64p, sz, u8p, sz]
        L.oracle_residue.argtypes = [u8p, sz, ctypes.c_uint64]
        L.oracle_residue.restype = ctypes.c_uint64
        L.oracle_residue_coeffs.argtypes = [u64p, sz, ctypes.c_uint64]
        L.oracle_residue_coeffs.restype = ctypes.c_uint64
        L.oracle_ntt_prime.restype = ctypes.c_uint64
        L.oracle_ntt_root.argtypes = [ctypes.c_uint64]
        L.oracle_ntt_root.restype = ctypes.c_uint64
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def long_mul(x, y) -> np.ndarray:
    """Section 2.1 long multiplication: n + m output digits."""
    x, px = _u8(x)
    y, py = _u8(y)
    z = np.zeros(len(x) + len(y), np.uint8)
    rc = lib().oracle_long_mul(px, len(x), py, len(y), z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError(f"oracle_long_mul failed ({rc})")
    return z


def conv(x, y) -> np.ndarray:
    """Section 2.1: exact coefficients c_0 .. c_{n+m-2} (uint64)."""
    x, px = _u8(x)
    y, py = _u8(y)
    c = np.zeros(len(x) + len(y) - 1, np.uint64)
    if lib().oracle_conv(px, len(x), py, len(y), _u64(c)) != 0:
        raise ValueError("oracle_conv failed")
    return c


def conv_ntt(x, y) -> np.ndarray:
    """Exact coefficients via the NTT (same result as conv)."""
    x, px = _u8(x)
    y, py = _u8(y)
    c = np.zeros(len(x) + len(y) - 1, np.uint64)
    rc = lib().oracle_conv_ntt(px, len(x), py, len(y), _u64(c))
    if rc != 0:
        raise ValueError(f"oracle_conv_ntt failed ({rc})")
    return c


#: above this many digit products the plain sum is replaced by the NTT
SCHOOLBOOK_LIMIT = 1 << 33


def conv_auto(x, y) -> np.ndarray:
    return conv(x, y) if len(x) * len(y) <= SCHOOLBOOK_LIMIT else conv_ntt(x, y)


def carry(c, nz: int) -> np.ndarray:
    """Section 2.4: the coefficient vector evaluated at b = 256 as nz digits."""
    c = np.ascontiguousarray(c, dtype=np.uint64)
    z = np.zeros(nz, np.uint8)
    if lib().oracle_carry(_u64(c), len(c), z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nz) != 0:
        raise ValueError("oracle_carry: value does not fit")
    return z


def product(x, y) -> np.ndarray:
    """x * y as len(x) + len(y) base-256 digits (convolution, then carry)."""
    return carry(conv_auto(x, y), len(x) + len(y))


def residue(x, p: int) -> int:
    x, px = _u8(x)
    return int(lib().oracle_residue(px, len(x), p))


def residue_coeffs(c, p: int) -> int:
    c = np.ascontiguousarray(c, dtype=np.uint64)
    return int(lib().oracle_residue_coeffs(_u64(c), len(c), p))


def ntt_prime() -> int:
    return int(lib().oracle_ntt_prime())


def ntt_root(n: int) -> int:
    return int(lib().oracle_ntt_root(n))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def to_int(d) -> int:
    """Section 2: x = sum_i x_i 256^i."""
    return int.from_bytes(np.asarray(d, np.uint8).tobytes(), "little")


def from_int(v: int, n: int) -> np.ndarray:
    return np.frombuffer(v.to_bytes(n, "little"), dtype=np.uint8).copy()
