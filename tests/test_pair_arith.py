"""The pair sum of the double-binary32 discs, checked on the CPU in binary32
arithmetic (numpy float32 operations round to nearest): its final
FastTwoSum(s, v) must be exact, i.e. give the same pair as the always-exact
TwoSum, for normalised operands (h = RN(h + l)), including the cancelling
high parts and half-ulp low parts where |v| comes closest to |s|.  This
pins the derivation the kernels rely on, not the kernels."""
import numpy as np

F = np.float32


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fast_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def normalised_low(rng, h):
    ulp = np.spacing(np.abs(h))
    lo = (rng.uniform(-0.5, 0.5, h.size) * ulp).astype(F)
    edge = rng.random(h.size) < 0.5
    lo[edge] = (np.sign(rng.uniform(-1, 1, edge.sum())) * ulp[edge].astype(np.float64)
                * (0.5 - 2.0 ** -22)).astype(F)
    return lo, (h + lo) == h


def check(xh, xl, yh, yl):
    with np.errstate(over="ignore", invalid="ignore"):
        s, e = two_sum(xh, yh)
        v = e + (xl + yl)
        f = fast_two_sum(s, v)
        t = two_sum(s, v)
    ok = np.isfinite(xh) & np.isfinite(yh)
    same = (f[0] == t[0]) & (f[1] == t[1])
    assert np.all(same[ok]), np.flatnonzero(~same & ok)[:5]
    # normalised result
    assert np.all(((f[0] + f[1]) == f[0])[ok])
    return int(ok.sum())


def test_fast_two_sum_exact_for_cancelling_pairs():
    rng = np.random.default_rng(2024)
    n = 2_000_000
    total = 0
    for scale_exp in (-30, 0, 20):
        xh = (rng.uniform(0.5, 4.0, n) * 2.0 ** scale_exp).astype(F)
        mix = rng.random(n)
        f = np.where(mix < 0.4, rng.uniform(0.5, 2.0, n),                   # Sterbenz range
                     np.where(mix < 0.8, 1.0 + rng.integers(-64, 65, n) * 2.0 ** -23,
                              rng.uniform(-8.0, 8.0, n)))                   # anything
        yh = (-(xh.astype(np.float64) * f)).astype(F)
        xl, k1 = normalised_low(rng, xh)
        yl, k2 = normalised_low(rng, yh)
        k = k1 & k2
        total += check(xh[k], xl[k], yh[k], yl[k])
    assert total > 4_000_000


def test_fast_two_sum_exact_near_subnormal_range():
    rng = np.random.default_rng(7)
    n = 500_000
    xh = (rng.uniform(0.5, 4.0, n) * 2.0 ** -125).astype(F)
    yh = (-(xh.astype(np.float64) * rng.uniform(0.5, 2.0, n))).astype(F)
    xl, k1 = normalised_low(rng, xh)
    yl, k2 = normalised_low(rng, yh)
    k = k1 & k2
    assert check(xh[k], xl[k], yh[k], yl[k]) > n // 4


def test_plain_fast_two_sum_would_fail_without_normalisation():
    """The same rule is not exact once |v| exceeds |s| by about 2^24 (low
    parts of 2^24 ulps of their high parts, far from normalised): the check
    above has power to see a failure."""
    rng = np.random.default_rng(3)
    n = 200_000
    xh = rng.uniform(1.0, 2.0, n).astype(F)
    yh = (-xh.astype(np.float64) * (1.0 + rng.integers(-2, 3, n) * 2.0 ** -23)).astype(F)
    xl = (np.spacing(xh) * rng.uniform(2.0 ** 24, 2.0 ** 26, n)).astype(F)     # not normalised
    yl = (np.spacing(np.abs(yh)) * rng.uniform(2.0 ** 24, 2.0 ** 26, n)).astype(F)
    s, e = two_sum(xh, yh)
    v = e + (xl + yl)
    f = fast_two_sum(s, v)
    t = two_sum(s, v)
    assert np.any((f[0] != t[0]) | (f[1] != t[1]))
