"""The paper's rigorous Schoenhage-Strassen multiplication, in the paper's order.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  fft(x, sign)      Section 2.2, the Cooley-Tukey FFT: split x into even and
                    odd entries, transform both halves, and combine
                    X_i = E_{i mod n/2} + omega^i O_{i mod n/2} for
                    i = 0 .. n-1 with omega = e^{2 pi i sign / n}.  Every
                    complex operation is a rectangular complex interval
                    operation with directed rounding (Section 2.5).  The
                    recursion is evaluated breadth first: all subproblems of
                    one size are transformed together as one batch, which
                    changes no arithmetic.
  convolve(a, b)    Section 2.3, the fast convolution algorithm: pad to
                    m = 2^k >= na + nb - 1 (the paper writes k =
                    ceil(log2(2n - 1)) for equal lengths), transform both,
                    multiply pointwise, transform back with omega^-1 and
                    divide by m (exact: m is a power of two).
  multiply(a, b)    Section 2.4 with Section 1's rule: isolate the unique
                    integer in every coefficient's containment set, report
                    an error when a set holds several integers (or none, or
                    its imaginary part excludes 0), and carry the integers
                    into na + nb base-256 digits.

Twiddles are the enclosures of oracle.twiddle (one per power omega^j).
Precision "f64" uses binary64 directed rounding; "f32" uses binary32
directed rounding with binary32 twiddle enclosures.

Parity: the digits are pinned to the exact product (oracle.exact); every
coefficient interval is pinned to contain the exact coefficient.  The
widths and the isolation limit of this radix-2 structure are the paper's
own structure; the GPU path's radix-4 transforms have other widths, so
widths are compared, not matched ("parity unpinned" for widths).
"""
from __future__ import annotations

import numpy as np

from . import exact as _exact
from . import interval as iv
from . import twiddle as tw

STATUS_OK, STATUS_ISOLATION_FAILED, STATUS_CONTAINMENT_FAILED = 0, 1, 2


def _twiddles(N: int, prec: str):
    c_lo, c_hi, s_lo, s_hi = tw.enclosures(N, f32=(prec == iv.F32))
    return c_lo, c_hi, s_lo, s_hi


def fft(x, sign: int, prec: str = iv.F64):
    """Interval DFT of x (tuple of 4 arrays of length n = 2^k), omega = e^{2 pi i sign/n}."""
    n = len(x[0])
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    c_lo, c_hi, s_lo, s_hi = _twiddles(max(n, 1), prec)
    # breadth-first recursion: level arrays have shape (batch, size)
    X = _fft_rec(tuple(np.asarray(c, np.float64)[None, :] for c in x), sign, prec,
                 n, (c_lo, c_hi, s_lo, s_hi))
    return tuple(c[0] for c in X)


def _fft_rec(x, sign, prec, N, tw_table):
    B, n = x[0].shape
    if n == 1:
        return x
    y = tuple(np.concatenate([c[:, 0::2], c[:, 1::2]], axis=0) for c in x)
    Y = _fft_rec(y, sign, prec, N, tw_table)
    E = tuple(c[:B] for c in Y)
    O = tuple(c[B:] for c in Y)
    return _combine(E, O, n, sign, prec, N, tw_table)


def _combine(E, O, n, sign, prec, N, tw_table):
    """X_i = E_{i mod n/2} + omega_n^i O_{i mod n/2}, i = 0 .. n-1."""
    c_lo, c_hi, s_lo, s_hi = tw_table
    i = np.arange(n)
    j = (i * (N // n)) % N                   # omega_n^i = omega_N^{i N / n}
    w = (c_lo[j], c_hi[j], s_lo[j], s_hi[j]) if sign > 0 else \
        (c_lo[j], c_hi[j], -s_hi[j], -s_lo[j])
    h = n // 2
    Eh = tuple(np.concatenate([c, c], axis=1) for c in E)
    Oh = tuple(np.concatenate([c, c], axis=1) for c in O)
    wb = tuple(np.broadcast_to(c[None, :], Oh[0].shape) for c in w)
    return iv.ic_add(Eh, iv.ic_mul(wb, Oh, prec), prec)


def fft_length(na: int, nb: int) -> int:
    """m = 2^k with k = ceil(log2(na + nb - 1)) (Section 2.3, generalised)."""
    L = na + nb - 1
    m = 1
    while m < L:
        m *= 2
    return m


def convolve(a, b, prec: str = iv.F64):
    """Section 2.3: interval enclosures of c = a * b, length m."""
    na, nb = len(a), len(b)
    m = fft_length(na, nb)
    ap = np.zeros(m)
    bp = np.zeros(m)
    ap[:na] = np.asarray(a, np.float64)
    bp[:nb] = np.asarray(b, np.float64)
    A = fft(iv.ic_point(ap), +1, prec)
    Bt = fft(iv.ic_point(bp), +1, prec)
    C = iv.ic_mul(A, Bt, prec)
    c = fft(C, -1, prec)
    k = m.bit_length() - 1
    return iv.ic_scale_pow2(c, k)


def multiply(a, b, prec: str = iv.F64):
    """Section 2.4 with the isolation rule of Section 1.

    Returns dict(status, digits (zero-filled unless OK), coeff (isolated
    integers), codes, intervals, max_width, max_width_imag, m)."""
    na, nb = len(a), len(b)
    L = na + nb - 1
    c = convolve(a, b, prec)
    re_lo, re_hi, im_lo, im_hi = (x[:L] for x in c)
    val, code = iv.isolate(re_lo, re_hi, im_lo, im_hi)
    if np.any(code >= iv.EMPTY):
        status = STATUS_CONTAINMENT_FAILED
    elif np.any(code == iv.AMBIGUOUS):
        status = STATUS_ISOLATION_FAILED
    else:
        status = STATUS_OK
    width = np.max(iv.sub_ru(re_hi, re_lo)) if L else 0.0
    width_im = np.max(iv.sub_ru(im_hi, im_lo)) if L else 0.0
    digits = np.zeros(na + nb, np.uint8)
    coeff = val.astype(np.uint64)
    if status == STATUS_OK:
        digits = _exact.carry(coeff, na + nb)
    return dict(status=status, digits=digits, coeff=coeff, codes=code,
                intervals=(re_lo, re_hi, im_lo, im_hi), max_width=float(width),
                max_width_imag=float(width_im), m=fft_length(na, nb))
