"""Transform lengths N = 3 * 2^k and 5 * 2^k (SSMUL_OPT_LENGTHS).

The zero padding of Section 2.3 may stop at the shortest allowed length of
the families 2^k, 3 * 2^k and 5 * 2^k.  The odd families need their own
root-of-unity enclosures (their arguments 2j/N are not binary fractions),
a radix-3 or radix-5 step in the column transforms and a division by 3
or 5 in the isolation.  Checked here: each family's twiddle table against
the oracle's rigorous enclosures; the lengths and geometries the plan
picks; every rung bit-exact under every length mask, on the same inputs;
every coefficient interval containing the exact coefficient.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import twiddle as tw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan, batched  # noqa: E402

OK = abi.SSMUL_OK


def expect_len(na, nb, mask=3):
    """(odd, log2) of the length the library must pick (its documented rule)."""
    L = na + nb - 1
    k = max(2, (L - 1).bit_length())
    if mask & 2 and 10 <= k - 3 <= 19 and (5 << (k - 3)) >= L:
        return 5, k - 3
    if mask & 1 and 11 <= k - 2 <= 21 and (3 << (k - 2)) >= L:
        return 3, k - 2
    return 1, k


@pytest.mark.parametrize("odd,K", [(3, 14), (5, 13)])
def test_odd_family_twiddles_contain_exact(odd, K):
    n = 1 << 15                        # plan length 2^16: families 3 2^14 and 5 2^13
    with Plan(n, n) as p:
        ln, cl, ch, sl, sh = p.twiddles(False, odd=odd)
        assert ln == K
        o = tw.octant_table(odd << ln)
        assert np.all(cl <= o[0]) and np.all(o[1] <= ch)
        assert np.all(sl <= o[2]) and np.all(o[3] <= sh)
        for lo, hi in ((cl, ch), (sl, sh)):          # 2 * 6 ulps plus rounding at most
            ulp = np.spacing(np.maximum(np.abs(lo), np.abs(hi)))
            assert np.all(hi - lo <= 13 * ulp)
        assert (cl[0], ch[0], sl[0], sh[0]) == (1.0, 1.0, 0.0, 0.0)
        ln32, fcl, fch, fsl, fsh = p.twiddles(True, odd=odd)
        assert ln32 == ln
        assert np.all(fcl <= cl) and np.all(ch <= fch) and np.all(fsl <= sl) and np.all(sh <= fsh)


@pytest.mark.parametrize("odd,K", [(1, 16), (3, 14), (5, 13)])
def test_twiddle_bounds_are_the_widened_values(odd, K):
    """The binary64 table keeps the values before the widening and rebuilds
    the bounds where they are read: every entry j >= 1 spans exactly 2 w
    binary64 steps (w = 4 where the argument 2 j / Ntab is exact, R = 1 or R
    divides j; 6 otherwise), or fewer only where it was clamped at 1, and
    entry 0 is the exact point (1, 0)."""
    n = 1 << 15
    with Plan(n, n) as p:
        ln, cl, ch, sl, sh = p.twiddles(False, odd=odd)
    assert ln == K
    j = np.arange(len(cl))
    w = np.where((odd == 1) | (j % odd == 0), 4, 6)
    for lo, hi in ((cl, ch), (sl, sh)):
        steps = hi.view(np.int64) - lo.view(np.int64)
        clamped = hi == 1.0
        assert np.all(steps[1:][~clamped[1:]] == 2 * w[1:][~clamped[1:]])
        assert np.all(steps[1:][clamped[1:]] <= 2 * w[1:][clamped[1:]])
        assert np.all(lo[1:] > 0.0)
    assert (cl[0], ch[0], sl[0], sh[0]) == (1.0, 1.0, 0.0, 0.0)


def test_short_plans_have_no_odd_tables():
    with Plan(2000, 2000) as p:
        buf = np.zeros(64)
        for flags in (2, 4, 6):
            s, _ = abi.ssmul_debug_twiddles(p.h, flags, buf.ctypes.data, 64)
            assert s == abi.SSMUL_INVALID_ARG


def test_odd_geometries():
    with Plan(1 << 22, 1 << 22) as p:
        for base, R, lo, hi in ((32, 3, 11, 21), (64, 5, 10, 19)):
            for k in range(lo, hi + 1):
                s, (a, b, cta) = abi.ssmul_debug_geometry(p.h, base + k)
                assert s == OK
                assert a + b == k and a % 2 == 0 and a >= 2 and (R << a) <= 4096 and 2 <= b <= 11
            assert abi.ssmul_debug_geometry(p.h, base + lo - 1)[0] == abi.SSMUL_INVALID_ARG
            assert abi.ssmul_debug_geometry(p.h, base + hi + 1)[0] == abi.SSMUL_INVALID_ARG


SIZES = [(3000, 2500), (2600, 2400), (4097, 1), (40000, 30000), (75000, 75000), (60000, 4000),
         (49153, 49152), (49153, 49153), (3000, 1000)]
RUNGS = [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_DISC32X2,
         abi.SSMUL_PREC_NAIVE64, abi.SSMUL_PREC_LADDER]


def test_length_rule_examples():
    assert expect_len(75000, 75000) == (5, 15)
    assert expect_len(3000, 2500) == (3, 11)
    assert expect_len(2600, 2400) == (5, 10)
    assert expect_len(49153, 49152) == (3, 15)
    assert expect_len(49153, 49153) == (1, 17)
    assert expect_len(75000, 75000, 1) == (3, 16)
    assert expect_len(75000, 75000, 0) == (1, 18)


@pytest.mark.parametrize("na,nb", SIZES)
def test_lengths_and_products(na, nb):
    L = na + nb - 1
    a, b = synth.operand_pair(synth.SEED_BASE + 300 + na + 7 * nb, na, nb)
    exact = E.product(a, b)
    for prec in RUNGS:
        with Plan(na, nb, 0, prec) as p:
            runs = {}
            for mask in (3, 0, 1, 2):
                assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_LENGTHS, mask) == OK
                runs[mask] = p.mul(a, b)
        want = abi.SSMUL_UNVERIFIED if prec == abi.SSMUL_PREC_NAIVE64 else OK
        for mask, (s, r, z) in runs.items():
            assert (r.fft_odd, r.fft_log2) == expect_len(na, nb, mask), (prec, mask)
            assert r.fft_odd << r.fft_log2 >= L
            assert s in (want, abi.SSMUL_ISOLATION_FAILED), (prec, mask, abi.status_string(s))
            if s == OK:
                assert np.array_equal(z, exact), (prec, mask)
            if prec in (abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_LADDER):
                assert s == OK
        r0, r3 = runs[0][1], runs[3][1]
        if r3.fft_odd > 1 and prec != abi.SSMUL_PREC_NAIVE64:
            # the odd families' twiddles are wider (6 ulps against 4 where R does
            # not divide j), the transform shorter
            assert 0 < r3.max_width <= r0.max_width * 2.5


@pytest.mark.parametrize("na,nb", [(3000, 2500), (2600, 2400), (40000, 30000)])
@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_FP32, abi.SSMUL_PREC_DISC64,
                                  abi.SSMUL_PREC_DISC32X2])
def test_intervals_contain_exact(na, nb, prec):
    a, b = synth.operand_pair(synth.SEED_BASE + 77 + na, na, nb, "ff" if na == 3000 else "uniform")
    with Plan(na, nb) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, prec)
    assert (r.fft_odd, r.fft_log2) == expect_len(na, nb)
    c = E.conv_ntt(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi)), prec
    assert r.n_empty == 0


def test_batched_mix_of_families():
    pairs = [synth.operand_pair(synth.SEED_BASE + 900 + i, na, nb) for i, (na, nb) in
             enumerate([(3000, 2500), (5000, 3000), (40000, 30000), (70000, 60000), (20, 30),
                        (75000, 75000), (3000, 2600), (2600, 2400)])]
    with Plan(75000, 75000, 16, abi.SSMUL_PREC_LADDER) as p:
        s, res, digits = batched(p, pairs)
    assert s == OK
    seen = set()
    for (a, b), r, z in zip(pairs, res, digits):
        assert r.status == OK and np.array_equal(z, E.product(a, b))
        if r.precision_used == abi.SSMUL_PREC_FP32:
            # binary32 on 4-bit digits: 2 (na + nb) - 1 coefficients, powers of two
            assert (r.fft_odd, r.fft_log2) == (1, (2 * (len(a) + len(b)) - 2).bit_length())
        else:
            assert (r.fft_odd, r.fft_log2) == expect_len(len(a), len(b))
        seen.add(r.fft_odd)
    assert seen == {1, 3, 5}


@pytest.mark.parametrize("odd,K", [(3, 21), (5, 19)])
def test_largest_odd_families_contain_exact_sampled(odd, K):
    """The largest odd-family tables (a plan of 2^22 x 2^22 digits), sampled:
    the first and last octant entries and a stride through the rest."""
    from fractions import Fraction as Fr
    n = 1 << 22
    with Plan(n, n) as p:
        ln, cl, ch, sl, sh = p.twiddles(False, odd=odd)
        assert ln == K
        N = odd << ln
        m = N // 8
        for j in list(range(0, 30)) + list(range(m - 30, m + 1)) + list(range(1, m, 7919)):
            (c, ec), (s, es) = tw.exact_fraction(N, j)
            assert Fr(float(cl[j])) <= c - ec and c + ec <= Fr(float(ch[j])), j
            assert Fr(float(sl[j])) <= s - es and s + es <= Fr(float(sh[j])), j
