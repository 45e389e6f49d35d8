"""The bench's cost model (bench.py) against the library's documented rules:
the transform length the library picks (ssmul.h, SSMUL_OPT_LENGTHS), the
default four-step geometry (column length R 2^a with a even and R 2^a <=
4096, rows 2^b with 2 <= b <= 11), and the operation counts' basic
properties.  CPU only."""
import pytest

import bench


def documented_length(na, nb):
    L = na + nb - 1
    k = max(2, (L - 1).bit_length())
    cands = [(1, k)]
    if 10 <= k - 3 <= 19:
        cands.append((5, k - 3))
    if 11 <= k - 2 <= 21:
        cands.append((3, k - 2))
    ok = [(R << j, R, j) for R, j in cands if (R << j) >= L]
    n, R, j = min(ok)
    return R, j


@pytest.mark.parametrize("na,nb", [(75000, 75000), (3000, 2500), (2600, 2400), (49153, 49152),
                                   (49153, 49153), (60000, 4000), (1 << 20, 1 << 12),
                                   (300000, 300000), (5000, 3000), (4097, 1)])
def test_length_rule(na, nb):
    assert bench.length_code(na, nb) == documented_length(na, nb)
    R, k = bench.length_code(na, nb)
    assert (R << k) >= na + nb - 1


def test_length_rule_sweep():
    for L in range(4000, 2_000_000, 997):
        na = L // 2 + 1
        nb = L + 1 - na
        R, k = bench.length_code(na, nb)
        assert (R, k) == documented_length(na, nb)
        # never longer than the next power of two, and within 1.6x of L
        assert (R << k) >= L and (R << k) <= (1 << max(2, (L - 1).bit_length()))
        if L > 4096:
            assert (R << k) < 1.6 * L


@pytest.mark.parametrize("R,k", [(1, 13), (1, 18), (1, 23), (3, 11), (3, 16), (3, 21),
                                 (5, 10), (5, 15), (5, 19)])
def test_geometry_bounds(R, k):
    a, b, c1, c3 = bench.geometry(R, k)
    assert a + b == k and 2 <= b <= 11
    if R > 1:
        assert a % 2 == 0 and a >= 2 and (R << a) <= 4096
    assert 0 <= c1 <= b and 0 <= c3 <= b - 1


def test_op_counts_at_75k():
    # 5 2^15 at 75k: fewer operations than 3 2^16 and 2^18 would take
    ops = {p: sum(bench.kernel_ops(75000, 75000, p).values())
           for p in ("fp64", "disc64", "disc32x2")}
    assert abs(ops["fp64"] / 1e6 - 31.46) < 0.05
    assert abs(ops["disc64"] / 1e6 - 15.97) < 0.05
    assert ops["disc64"] < ops["fp64"] < ops["disc32x2"]
    assert bench.fft_len_str(75000) == "5*2^15"
