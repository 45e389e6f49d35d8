"""The binary64 twiddle table's bound rebuild, restated on the CPU.

The table keeps each entry's cosine and sine before the widening; every
reader moves each value w binary64 steps down and up by integer steps of its
bit pattern and clamps to [0, 1].  For the positive finite values of the
first octant that must equal w applications of nextafter toward -inf and
+inf followed by the clamp, which is how the widening of the enclosures is
defined.  Here both are evaluated with numpy on values that cover the octant,
the steps across a power of two and the clamp at 1.
"""
import numpy as np
import pytest

ONE_BITS = np.float64(1.0).view(np.int64)


def _rebuild(v, w):
    """Integer steps of the bit pattern and the clamp, as the kernels do."""
    b = np.asarray(v, np.float64).view(np.int64)
    lo = np.maximum(b - w, 0).view(np.float64)
    hi = np.minimum(b + w, ONE_BITS).view(np.float64)
    return lo, hi


def _nextafter(v, w):
    lo = np.asarray(v, np.float64).copy()
    hi = lo.copy()
    for _ in range(w):
        lo = np.nextafter(lo, -np.inf)
        hi = np.nextafter(hi, np.inf)
    return np.maximum(lo, 0.0), np.minimum(hi, 1.0)


def _first_octant_values(n):
    j = np.arange(1, n // 8 + 1)
    x = 2.0 * np.pi * j / n
    return np.concatenate([np.cos(x), np.sin(x)])


@pytest.mark.parametrize("w", [4, 6])
@pytest.mark.parametrize("n", [8, 1 << 10, 5 << 12, 3 << 14])
def test_bit_steps_equal_nextafter_on_the_octant(n, w):
    v = _first_octant_values(n)
    assert np.all(v > 0.0) and np.all(v <= 1.0)
    lo, hi = _rebuild(v, w)
    lo2, hi2 = _nextafter(v, w)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    assert np.all(lo < v) and np.all((hi > v) | (v == 1.0))


@pytest.mark.parametrize("w", [1, 4, 6])
def test_steps_across_powers_of_two_and_the_clamp(w):
    """Values within a few steps of 1/2, 1/4 and 1 (where the step size
    changes), and 1 itself, whose upper bound is clamped."""
    edges = []
    for p in (0.5, 0.25, 1.0 / 1024):
        x = np.float64(p)
        for _ in range(8):
            x = np.nextafter(x, -np.inf)
        for _ in range(16):
            edges.append(x)
            x = np.nextafter(x, np.inf)
    x = np.float64(1.0)
    for _ in range(8):
        edges.append(x)
        x = np.nextafter(x, -np.inf)
    v = np.array(edges)
    lo, hi = _rebuild(v, w)
    lo2, hi2 = _nextafter(v, w)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    assert np.all(hi <= 1.0)
    assert hi[np.argmax(v)] == 1.0


def test_the_exact_point_keeps_zero_width():
    """Entry 0 is the point (1, 0) and takes no widening (w = 0)."""
    lo, hi = _rebuild(np.array([1.0, 0.0]), 0)
    assert lo.tolist() == [1.0, 0.0] and hi.tolist() == [1.0, 0.0]
    assert np.signbit(lo[1]) == False  # noqa: E712  (+0, not -0)
