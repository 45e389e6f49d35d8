"""The exact correction of the binary32 rung's centred 4-bit digits, on the CPU.

The rung transforms e_j = a'_j - ma and f_j = b'_j - mb (a'_j the 4-bit
digits, ma and mb their rounded means) and adds back
    mb Wa_i + ma Wb_i - ma mb |J_i|
to each isolated coefficient, where J_i holds the pairs (j, i - j) that meet
in coefficient i and Wa_i, Wb_i are the digit sums over J_i, read from one
prefix array Q over a's then b's digits.  Here the same window bounds and Q
indices are evaluated in exact integers and the result is compared with the
oracle's convolution of the uncentred 4-bit digits (the product identity of
Section 2.1 in base 16), which must come out equal for every operand.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E


def _nibbles(x):
    x = np.asarray(x, np.uint8)
    return np.stack([x & 15, x >> 4], axis=1).reshape(-1).astype(np.int64)


def _centred_coefficients(a, b):
    """c'_i rebuilt the way the kernel does: the centred convolution plus the
    window-sum correction."""
    na2, nb2 = 2 * len(a), 2 * len(b)
    da, db = _nibbles(a), _nibbles(b)
    Q = np.concatenate([[0], np.cumsum(np.concatenate([da, db]))])
    ma = (2 * int(Q[na2]) + na2) // (2 * na2)                  # rounded means
    mb = (2 * int(Q[na2 + nb2] - Q[na2]) + nb2) // (2 * nb2)
    e, f = da - ma, db - mb
    cc = np.convolve(e, f)                                      # c''_i, exact in int64
    out = np.empty(na2 + nb2 - 1, np.int64)
    for i in range(na2 + nb2 - 1):
        ja_lo, ja_hi = max(i - nb2 + 1, 0), min(i, na2 - 1)
        jb_lo, jb_hi = max(i - na2 + 1, 0), min(i, nb2 - 1)
        wa = int(Q[ja_hi + 1] - Q[ja_lo])
        wb = int(Q[na2 + jb_hi + 1] - Q[na2 + jb_lo])
        out[i] = cc[i] + mb * wa + ma * wb - ma * mb * (ja_hi - ja_lo + 1)
    return out, ma, mb


@pytest.mark.parametrize("na,nb,dist", [(1, 1, "uniform"), (1, 7, "uniform"), (5, 3, "ff"),
                                        (17, 40, "raw"), (64, 63, "uniform"), (200, 1, "ff"),
                                        (256, 256, "uniform"), (3, 3, "zero")])
def test_centred_correction_gives_the_base16_convolution(na, nb, dist):
    a, b = synth.operand_pair(synth.SEED_BASE + 4000 + 7 * na + nb, na, nb, dist)
    got, ma, mb = _centred_coefficients(a, b)
    want = E.conv(_nibbles(a).astype(np.uint8), _nibbles(b).astype(np.uint8))
    assert np.array_equal(got, np.asarray(want, np.int64))
    # and those coefficients give the product (Section 2.1 in base 16)
    assert sum(int(c) << (4 * i) for i, c in enumerate(got)) == E.to_int(a) * E.to_int(b)
    assert 0 <= ma <= 15 and 0 <= mb <= 15


def test_centres_of_the_extreme_operands():
    """All-0xFF operands centre on 15 (their centred digits are all zero),
    zero operands on 0, sparse ones on 0, uniform ones near 7.5."""
    ff = np.full(100, 0xFF, np.uint8)
    zero = np.zeros(100, np.uint8)
    sparse = zero.copy()
    sparse[[3, 50, 99]] = [0x12, 0xF0, 0x07]
    uni = synth.operand_pair(synth.SEED_BASE + 4100, 1000, 1)[0]
    assert _centred_coefficients(ff, zero)[1:] == (15, 0)
    assert _centred_coefficients(sparse, uni)[1] == 0
    assert _centred_coefficients(sparse, uni)[2] in (7, 8)


def test_a_wrong_window_bound_is_caught():
    """The identity is sensitive to the window bounds: dropping the last pair
    of J_i breaks it for a generic operand pair."""
    a, b = synth.operand_pair(synth.SEED_BASE + 4200, 30, 20)
    na2, nb2 = 60, 40
    da, db = _nibbles(a), _nibbles(b)
    Q = np.concatenate([[0], np.cumsum(np.concatenate([da, db]))])
    ma, mb = 7, 8
    cc = np.convolve(da - ma, db - mb)
    want = np.asarray(E.conv(da.astype(np.uint8), db.astype(np.uint8)), np.int64)
    bad = 0
    for i in range(na2 + nb2 - 1):
        ja_lo, ja_hi = max(i - nb2 + 1, 0), min(i, na2 - 1) - 1     # one pair short
        jb_lo, jb_hi = max(i - na2 + 1, 0), min(i, nb2 - 1)
        wa = int(Q[ja_hi + 1] - Q[ja_lo])
        wb = int(Q[na2 + jb_hi + 1] - Q[na2 + jb_lo])
        v = cc[i] + mb * wa + ma * wb - ma * mb * (ja_hi - ja_lo + 1)
        bad += int(v != want[i])
    assert bad > (na2 + nb2) // 2
