"""Transform lengths N = 3 * 2^k (SSMUL_OPT_RADIX3).

The zero padding of Section 2.3 may stop at the next length of either
family 2^k or 3 * 2^k.  The second family needs its own root-of-unity
enclosures (its arguments 2j/N are not binary fractions), a radix-3 step
in the column transforms and a division by 3 in the isolation.  Checked
here: the family's twiddle table against the oracle's rigorous
enclosures; the lengths and geometries the plan picks; every rung
bit-exact with the option on and off, on the same inputs; every
coefficient interval containing the exact coefficient.
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
from tests.gpu_util import Plan  # noqa: E402

OK = abi.SSMUL_OK


def test_family3_twiddles_contain_exact():
    n = 1 << 15                        # plan length 2^16: the family 3 2^14
    with Plan(n, n) as p:
        ln, cl, ch, sl, sh = p.twiddles(False, three=True)
        assert ln == 14
        N = 3 << ln
        o = tw.octant_table(N)
        assert np.all(cl <= o[0]) and np.all(o[1] <= ch)
        assert np.all(sl <= o[2]) and np.all(o[3] <= sh)
        for lo, hi in ((cl, ch), (sl, sh)):          # 2 * 6 ulps plus rounding at most
            ulp = np.spacing(np.maximum(np.abs(lo), np.abs(hi)))
            assert np.all(hi - lo <= 13 * ulp)
        assert (cl[0], ch[0], sl[0], sh[0]) == (1.0, 1.0, 0.0, 0.0)
        ln32, fcl, fch, fsl, fsh = p.twiddles(True, three=True)
        assert ln32 == ln
        assert np.all(fcl <= cl) and np.all(ch <= fch) and np.all(fsl <= sl) and np.all(sh <= fsh)
    with Plan(2000, 2000) as p:                  # too short for the family: no table
        buf = np.zeros(64)
        s, _ = abi.ssmul_debug_twiddles(p.h, 2, buf.ctypes.data, 64)
        assert s == abi.SSMUL_INVALID_ARG


def test_family3_geometry():
    with Plan(1 << 22, 1 << 22) as p:
        for k in range(11, 22):
            s, (a, b, cta) = abi.ssmul_debug_geometry(p.h, 32 + k)
            assert s == OK
            assert a + b == k and a % 2 == 0 and 2 <= a <= 10 and 2 <= b <= 11
        assert abi.ssmul_debug_geometry(p.h, 32 + 10)[0] == abi.SSMUL_INVALID_ARG
        assert abi.ssmul_debug_geometry(p.h, 32 + 22)[0] == abi.SSMUL_INVALID_ARG


# (na, nb) -> expected (times3, log2 part) with the option on
SIZES = [((3000, 2500), (1, 11)), ((4097, 1), (1, 11)), ((2049, 2049), (1, 11)),
         ((40000, 30000), (1, 15)), ((75000, 75000), (1, 16)), ((60000, 4000), (0, 16)),
         ((49153, 49152), (1, 15)), ((49153, 49153), (0, 17)), ((3000, 1000), (0, 12))]
RUNGS = [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_DISC32X2,
         abi.SSMUL_PREC_NAIVE64, abi.SSMUL_PREC_LADDER]


@pytest.mark.parametrize("sizes,expect", SIZES)
def test_lengths_and_products(sizes, expect):
    na, nb = sizes
    L = na + nb - 1
    a, b = synth.operand_pair(synth.SEED_BASE + 300 + na + 7 * nb, na, nb)
    exact = E.product(a, b)
    for prec in RUNGS:
        with Plan(na, nb, 0, prec) as p:
            s1, r1, z1 = p.mul(a, b)
            assert abi.ssmul_plan_set_option(p.h, abi.SSMUL_OPT_RADIX3, 0) == OK
            s0, r0, z0 = p.mul(a, b)
        assert (r1.fft_times3, r1.fft_log2) == expect, prec
        assert (r0.fft_times3, r0.fft_log2) == (0, (L - 1).bit_length()), prec
        assert (3 if r1.fft_times3 else 1) << r1.fft_log2 >= L
        want = abi.SSMUL_UNVERIFIED if prec == abi.SSMUL_PREC_NAIVE64 else OK
        for s, z in ((s1, z1), (s0, z0)):
            assert s in (want, abi.SSMUL_ISOLATION_FAILED), (prec, abi.status_string(s))
            if s == want and prec != abi.SSMUL_PREC_NAIVE64:
                assert np.array_equal(z, exact), prec
        if prec in (abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_DISC64, abi.SSMUL_PREC_LADDER):
            assert s1 == OK and s0 == OK
        if r1.fft_times3 and prec != abi.SSMUL_PREC_NAIVE64:
            # the family-3 twiddles are wider (6 ulps against 4 where 3 does
            # not divide j), the transform shorter
            assert 0 < r1.max_width <= r0.max_width * 2.0


@pytest.mark.parametrize("na,nb", [(3000, 2500), (40000, 30000)])
@pytest.mark.parametrize("prec", [abi.SSMUL_PREC_FP64, abi.SSMUL_PREC_FP32, abi.SSMUL_PREC_DISC64,
                                  abi.SSMUL_PREC_DISC32X2])
def test_intervals_contain_exact(na, nb, prec):
    a, b = synth.operand_pair(synth.SEED_BASE + 77 + na, na, nb, "ff" if na == 3000 else "uniform")
    with Plan(na, nb) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, prec)
    assert r.fft_times3 == 1
    c = E.conv_ntt(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi)), prec
    assert r.n_empty == 0


def test_batched_mix_of_families():
    from tests.gpu_util import batched
    pairs = [synth.operand_pair(synth.SEED_BASE + 900 + i, na, nb) for i, (na, nb) in
             enumerate([(3000, 2500), (5000, 3000), (40000, 30000), (70000, 60000), (20, 30),
                        (75000, 75000), (3000, 2600)])]
    with Plan(75000, 75000, 16, abi.SSMUL_PREC_LADDER) as p:
        s, res, digits = batched(p, pairs)
    assert s == OK
    seen = set()
    for (a, b), r, z in zip(pairs, res, digits):
        assert r.status == OK and np.array_equal(z, E.product(a, b))
        seen.add(r.fft_times3)
    assert seen == {0, 1}
