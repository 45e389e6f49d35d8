"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar: product digits bit-exact (integer work); every coefficient enclosure
contains the exact coefficient (the rigor of Section 2.5); the device
interval primitives bit-exact against exact directed rounding where the
formula is the same, and between the exact hull and the paper's formula
where the device fuses a multiply-add.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import interval as iv
from oracle import twiddle as tw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402
from tests.gpu_util import Plan, batched, dev  # noqa: E402

OK = abi.SSMUL_OK


def _pair(seed, na, nb, dist="uniform"):
    return synth.operand_pair(synth.SEED_BASE + seed, na, nb, dist)


# ---- twiddle enclosures ---------------------------------------------------------

@pytest.mark.parametrize("log_n", [4, 10, 16])
def test_twiddles_contain_exact_all_entries(log_n):
    n = 1 << log_n
    with Plan(n // 2, n // 2) as p:
        ln, cl, ch, sl, sh = p.twiddles(False)
        # the table also serves 4-bit digits: up to 4 N, at most 2^12
        assert ln == max(log_n, min(12, log_n + 2))
        o = tw.octant_table(1 << ln)
        assert np.all(cl <= o[0]) and np.all(o[1] <= ch)
        assert np.all(sl <= o[2]) and np.all(o[3] <= sh)
        # documented bound widened: at most 2 * 4 ulps wide
        for lo, hi in ((cl, ch), (sl, sh)):
            wide = hi - lo
            ulp = np.spacing(np.maximum(np.abs(lo), np.abs(hi)))
            assert np.all(wide <= 9 * ulp)
        assert (cl[0], ch[0], sl[0], sh[0]) == (1.0, 1.0, 0.0, 0.0)
        ln32, fcl, fch, fsl, fsh = p.twiddles(True)
        assert np.all(fcl <= cl) and np.all(ch <= fch) and np.all(fsl <= sl) and np.all(sh <= fsh)
        assert np.all(fcl.astype(np.float32).astype(np.float64) == fcl)


def test_twiddles_contain_exact_sampled_2_23():
    n = 1 << 23
    with Plan(n // 2, n // 2) as p:
        ln, cl, ch, sl, sh = p.twiddles(False)
        assert ln == 23
        from fractions import Fraction as Fr
        for j in list(range(0, 40)) + list(range(n // 8 - 40, n // 8 + 1)) + \
                list(range(1, n // 8, 9973)):
            (c, ec), (s, es) = tw.exact_fraction(n, j)
            assert Fr(float(cl[j])) <= c - ec and c + ec <= Fr(float(ch[j]))
            assert Fr(float(sl[j])) <= s - es and s + es <= Fr(float(sh[j]))


# ---- interval primitives -------------------------------------------------------

def _rand_ci(rng, n, f32=False, sign_definite=False):
    lo_r = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 6, n)
    lo_i = rng.standard_normal(n) * 10.0 ** rng.integers(-3, 6, n)
    w_r = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-12, 1, n) * np.abs(lo_r)
    w_i = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-12, 1, n) * np.abs(lo_i)
    x = np.stack([lo_r, lo_r + w_r, lo_i, lo_i + w_i], axis=1)
    if sign_definite:
        x = np.stack([lo_r, lo_r * (1 + 1e-15 * np.sign(lo_r)), lo_i, lo_i * (1 + 1e-15 * np.sign(lo_i))], 1)
        x[:, 0], x[:, 1] = np.minimum(x[:, 0], x[:, 1]), np.maximum(x[:, 0], x[:, 1])
        x[:, 2], x[:, 3] = np.minimum(x[:, 2], x[:, 3]), np.maximum(x[:, 2], x[:, 3])
        x[:8] = [[1, 1, 0, 0], [0, 0, 1, 1], [-1, -1, 0, 0], [0, 0, -1, -1],
                 [0.5, 0.5000000000000001, -0.8660254037844387, -0.8660254037844386],
                 [-0.7071067811865477, -0.7071067811865475, 0.7071067811865475, 0.7071067811865477],
                 [1, 1, 0, 0], [0, 0, 1, 1]]
    if f32:
        x[:, 0] = iv.to32_rd(x[:, 0])
        x[:, 1] = iv.to32_ru(x[:, 1])
        x[:, 2] = iv.to32_rd(x[:, 2])
        x[:, 3] = iv.to32_ru(x[:, 3])
    return x


def _run_op(op, f32, x, y):
    dx, dy = dev(x.ravel()), dev(y.ravel())
    out = torch.zeros_like(dx)
    assert abi.ssmul_debug_ci_op(op, f32, dx.data_ptr(), dy.data_ptr(), out.data_ptr(), len(x)) == OK
    return out.cpu().numpy().reshape(-1, 4)


@pytest.mark.parametrize("f32", [False, True])
def test_ci_add_sub_mul_bit_exact(f32):
    rng = np.random.default_rng(7 + f32)
    x, y = _rand_ci(rng, 4000, f32), _rand_ci(rng, 4000, f32)
    # straddling and sign-mixed cases
    y[:100, 0] = -np.abs(y[:100, 1]); y[:100, 1] = np.abs(y[:100, 1])
    x[50:150, 2] = -np.abs(x[50:150, 3]); x[50:150, 3] = np.abs(x[50:150, 3])
    prec = iv.F32 if f32 else iv.F64
    X = tuple(x[:, k] for k in range(4))
    Y = tuple(y[:, k] for k in range(4))
    for op, ref in ((0, iv.ic_add), (1, iv.ic_sub), (3, iv.ic_mul)):
        got = _run_op(op, f32, x, y)
        want = np.stack(ref(X, Y, prec), axis=1)
        assert np.array_equal(got, want), f"op {op}"


@pytest.mark.parametrize("f32", [False, True])
def test_ci_twiddle_product_between_hull_and_paper_formula(f32):
    from fractions import Fraction as Fr
    rng = np.random.default_rng(11)
    x = _rand_ci(rng, 2000, f32)
    w = _rand_ci(rng, 2000, f32, sign_definite=True)
    got = _run_op(2, f32, x, w)
    prec = iv.F32 if f32 else iv.F64
    paper = np.stack(iv.ic_mul(tuple(x[:, k] for k in range(4)), tuple(w[:, k] for k in range(4)), prec), 1)
    # no wider than the paper's formula (the fused multiply-add rounds once)
    assert np.all(got[:, 0] >= paper[:, 0]) and np.all(got[:, 1] <= paper[:, 1])
    assert np.all(got[:, 2] >= paper[:, 2]) and np.all(got[:, 3] <= paper[:, 3])
    # and still containing the exact hull over the corners
    for i in range(0, 2000, 7):
        xr = [Fr(float(v)) for v in x[i, :2]]
        xi = [Fr(float(v)) for v in x[i, 2:]]
        wr = [Fr(float(v)) for v in w[i, :2]]
        wi = [Fr(float(v)) for v in w[i, 2:]]
        re = [a * c - b * d for a in xr for b in xi for c in wr for d in wi]
        im = [a * d + b * c for a in xr for b in xi for c in wr for d in wi]
        assert Fr(float(got[i, 0])) <= min(re) and max(re) <= Fr(float(got[i, 1]))
        assert Fr(float(got[i, 2])) <= min(im) and max(im) <= Fr(float(got[i, 3]))


@pytest.mark.parametrize("f32", [False, True])
def test_ci_real_and_imaginary_scalar_products_equal_paper_formula(f32):
    """The radix-3 and radix-5 steps multiply by real enclosures (cos) and
    pure imaginary ones (i sin) in 4 directed products: the result must be
    the paper's interval product (Section 2.5) with the zero part taken as
    the point 0, bit for bit."""
    rng = np.random.default_rng(12 + f32)
    x = _rand_ci(rng, 3000, f32)
    x[:200, 0] = -np.abs(x[:200, 1]); x[:200, 1] = np.abs(x[:200, 1])       # straddling 0
    w = _rand_ci(rng, 3000, f32, sign_definite=True)
    prec = iv.F32 if f32 else iv.F64
    X = tuple(x[:, k] for k in range(4))
    for op, keep in ((4, (0, 1)), (5, (2, 3))):
        wz = w.copy()
        zero = (2, 3) if op == 4 else (0, 1)
        wz[:, zero[0]] = 0.0
        wz[:, zero[1]] = 0.0
        ok = (wz[:, keep[0]] > 0) | (wz[:, keep[1]] < 0)                   # sign-definite part
        got = _run_op(op, f32, x, wz)[ok]
        want = np.stack(iv.ic_mul(X, tuple(wz[:, k] for k in range(4)), prec), axis=1)[ok]
        assert ok.sum() > 2500
        assert np.array_equal(got, want), f"op {op}"


# ---- end-to-end parity ---------------------------------------------------------

SMALL_SIZES = [(1, 1), (1, 2), (2, 1), (2, 2), (3, 1), (1, 7), (5, 5), (8, 9), (17, 16), (31, 33),
               (64, 64), (100, 3), (255, 257), (1000, 1000), (1024, 1025), (2048, 2048), (2049, 2000)]


@pytest.mark.parametrize("na,nb", SMALL_SIZES)
def test_small_products_bit_exact(na, nb):
    a, b = _pair(na * 7 + nb, na, nb)
    with Plan(na, nb) as p:
        s, r, z = p.mul(a, b)
    assert s == OK, abi.status_string(s)
    assert np.array_equal(z, E.product(a, b))
    assert r.precision_used == abi.SSMUL_PREC_FP64 and r.n_unisolated == 0 and r.n_empty == 0


def test_exhaustive_short_lengths():
    with Plan(40, 40) as p:
        for na in range(1, 41):
            for nb in range(1, 41, 3):
                a, b = _pair(na * 100 + nb, na, nb, "raw")
                s, r, z = p.mul(a, b)
                assert s == OK and np.array_equal(z, E.product(a, b)), (na, nb)


FOURSTEP_SIZES = [(2049, 2049), (4096, 4096), (4097, 100), (3, 5000), (10000, 7777),
                  (16384, 16384), (32768, 32767), (65536, 1), (65535, 65537), (100000, 31)]


@pytest.mark.parametrize("na,nb", FOURSTEP_SIZES)
def test_fourstep_products_bit_exact(na, nb):
    a, b = _pair(na + 3 * nb, na, nb)
    with Plan(na, nb) as p:
        s, r, z = p.mul(a, b)
    assert s == OK, abi.status_string(s)
    assert np.array_equal(z, E.product(a, b))


@pytest.mark.parametrize("dist", ["uniform", "ff"])
def test_paper_scale_75000(dist):
    # the paper's largest double-precision size (75,000 base-256 digits)
    a, b = _pair(2, 75000, 75000, dist)
    with Plan(75000, 75000) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, abi.SSMUL_PREC_FP64)
    assert (r.fft_odd, r.fft_log2) == (5, 15)           # N = 5 2^15 >= 149,999
    assert s == OK, abi.status_string(s)
    assert np.array_equal(z, E.product(a, b))
    c = E.conv_ntt(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi))
    assert 0 < r.max_width < 1.0
    if dist == "ff":
        assert c.max() == 4_876_875_000.0


@pytest.mark.parametrize("na,nb,prec", [(1, 1, 0), (7, 9, 0), (1000, 1000, 0), (4096, 4096, 0),
                                        (5000, 3000, 0), (3, 3, 1), (10, 10, 1), (512, 512, 1)])
def test_every_interval_contains_exact_coefficient(na, nb, prec):
    a, b = _pair(na * 5 + nb + prec, na, nb)
    with Plan(na, nb) as p:
        s, r, z, lo, hi = p.mul_intervals(a, b, prec)
    c = E.conv(a, b).astype(np.float64)
    assert np.all((lo <= c) & (c <= hi))
    assert r.n_empty == 0
    if s == OK:
        assert np.array_equal(z, E.product(a, b))
    else:
        assert s == abi.SSMUL_ISOLATION_FAILED and not z.any()


def test_fp32_failure_is_reported_and_zero_filled():
    a, b = _pair(9, 512, 512)
    with Plan(512, 512, 0, abi.SSMUL_PREC_FP32) as p:
        s, r, z = p.mul(a, b)
    assert s == abi.SSMUL_ISOLATION_FAILED
    assert r.n_unisolated > 0 and r.precision_used == abi.SSMUL_PREC_FP32
    assert not z.any()


def test_ladder_resolves_small_in_fp32_and_escalates():
    with Plan(3000, 3000, 0, abi.SSMUL_PREC_LADDER) as p:
        a, b = _pair(1, 4, 3)
        s, r, z = p.mul(a, b)
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP32
        assert np.array_equal(z, E.product(a, b))
        a, b = _pair(2, 20, 20)
        s, r, z = p.mul(a, b)
        assert s == OK and np.array_equal(z, E.product(a, b))
        a, b = _pair(3, 3000, 2999)
        s, r, z = p.mul(a, b)
        assert s == OK and r.precision_used == abi.SSMUL_PREC_FP64
        assert np.array_equal(z, E.product(a, b))


def test_edge_operands():
    with Plan(5000, 5000) as p:
        z0 = np.zeros(5000, np.uint8)
        a = synth.uniform_digits(3, 4000)
        s, r, z = p.mul(z0, a)
        assert s == OK and not z.any()
        one = np.zeros(300, np.uint8); one[0] = 1          # leading zeros allowed
        s, r, z = p.mul(one, a)
        assert s == OK and np.array_equal(z, E.product(one, a))
        shift = np.zeros(1000, np.uint8); shift[999] = 1   # 256^999
        s, r, z = p.mul(a, shift)
        assert s == OK and np.array_equal(z[999:999 + 4000], a) and not z[:999].any()
        ff = np.full(5000, 0xFF, np.uint8)
        s, r, z = p.mul(ff, ff)
        assert s == OK and np.array_equal(z, E.product(ff, ff))


def test_invalid_arguments():
    with Plan(100, 100) as p:
        a = dev(np.ones(10, np.uint8))
        z = torch.zeros(300, dtype=torch.uint8, device="cuda")
        s, _ = abi.ssmul_mul(p.h, a.data_ptr(), 0, a.data_ptr(), 10, z.data_ptr())
        assert s == abi.SSMUL_INVALID_ARG
        s, _ = abi.ssmul_mul(p.h, a.data_ptr(), 101, a.data_ptr(), 10, z.data_ptr())
        assert s == abi.SSMUL_TOO_LARGE
        s, _ = abi.ssmul_mul(p.h, 0, 10, a.data_ptr(), 10, z.data_ptr())
        assert s == abi.SSMUL_INVALID_ARG


def test_host_buffers():
    a, b = _pair(21, 30000, 20000)
    with Plan(30000, 30000) as p:
        z = np.zeros(50000, np.uint8)
        s, r = abi.ssmul_mul_host(p.h, a.ctypes.data, len(a), b.ctypes.data, len(b), z.ctypes.data)
    assert s == OK and np.array_equal(z, E.product(a, b))


def test_batched_mixed_sizes():
    rng = np.random.default_rng(3)
    pairs = []
    for i in range(40):
        na, nb = (int(v) for v in np.exp(rng.uniform(0, np.log(20000), 2)).astype(int) + 1)
        pairs.append(_pair(100 + i, na, nb, "ff" if i % 10 == 0 else "uniform"))
    pairs.append(_pair(999, 3, 2))
    mx = max(max(len(a), len(b)) for a, b in pairs)
    with Plan(mx, mx, len(pairs), abi.SSMUL_PREC_LADDER) as p:
        s, res, digits = batched(p, pairs)
    assert s == OK
    for (a, b), r, z in zip(pairs, res, digits):
        assert r.status == OK
        assert np.array_equal(z, E.product(a, b))


@pytest.mark.parametrize("na,nb", [(1 << 20, 1 << 12), (1 << 19, 1 << 19)])
def test_large_products_residues(na, nb):
    a, b = _pair(na ^ nb, na, nb)
    with Plan(na, nb) as p:
        s, r, z = p.mul(a, b)
    assert s == OK, abi.status_string(s)
    assert np.array_equal(z, E.carry(E.conv_ntt(a, b), na + nb))
    for q in (2**61 - 1, 1_000_000_007):
        assert E.residue(z, q) == E.residue(a, q) * E.residue(b, q) % q


def test_largest_plan_size_discs_and_empty_batch():
    """The largest transform the plans support (2^22 x 2^22 digits, N = 2^23)
    under the binary64 discs, which isolate it: bit-exact; and a batched call
    with no products is a no-op that succeeds."""
    n = 1 << 22
    a, b = _pair(4242, n, n)
    with Plan(n, n, 4, abi.SSMUL_PREC_DISC64) as p:
        s, r, z = p.mul(a, b)
        assert s == OK, abi.status_string(s)
        assert (r.fft_odd, r.fft_log2) == (1, 23)
        assert np.array_equal(z, E.carry(E.conv_ntt(a, b), 2 * n))
        assert abi.ssmul_mul_batched(p.h, [], 0, 0, 0, 0) == OK
