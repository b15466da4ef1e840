"""The TF32 rounding the TF32 tensor-core route applies to its operands.

The kernels round an FP32 value x to TF32 (10 explicit mantissa bits) by
adding half a TF32 unit to the bit pattern and clearing the 13 dropped bits:
    bits(x) + 0x1000, then AND 0xFFFFE000.
This test pins that identity against an independent construction on the
CPU: the result must be the nearer of the two TF32 neighbours of x, and on
an exact tie the one of larger magnitude (round to nearest, ties away from
zero), for finite values, both signs, subnormals and carries into the
exponent."""

import numpy as np


def add_and_mask(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def reference_tf32(x):
    """Nearest TF32 value, ties away from zero, built from the two TF32
    neighbours of |x| (truncation and the next TF32 value up) in FP64."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32)
    sign = b & np.uint32(0x80000000)
    mag = b & np.uint32(0x7FFFFFFF)
    lo = mag & np.uint32(0xFFFFE000)                 # truncated magnitude
    hi = lo + np.uint32(0x2000)                      # next TF32 magnitude up
    v = mag.view(np.float32).astype(np.float64)
    vlo = lo.view(np.float32).astype(np.float64)
    vhi = hi.view(np.float32).astype(np.float64)
    pick_hi = (vhi - v) <= (v - vlo)                 # nearer, ties to the larger magnitude
    out = np.where(pick_hi, hi, lo) | sign
    return out.view(np.float32)


def test_random_finite_values():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 0x7F7FFFFF, size=200_000, dtype=np.uint64).astype(np.uint32)
    bits[::2] |= np.uint32(0x80000000)               # both signs
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < np.float32(3.0e38))]
    np.testing.assert_array_equal(add_and_mask(x).view(np.uint32), reference_tf32(x).view(np.uint32))


def test_exact_ties_go_away_from_zero():
    # low 13 bits exactly 0x1000: half a TF32 unit above a TF32 value
    base = np.array([1.0, 1.5, 3.0, 1234.5, 1e-20, 6.5e4], dtype=np.float32).view(np.uint32)
    tie = (base & np.uint32(0xFFFFE000)) | np.uint32(0x1000)
    for s in (0, 0x80000000):
        x = (tie | np.uint32(s)).view(np.float32)
        got = add_and_mask(x).view(np.uint32)
        want = ((tie & np.uint32(0xFFFFE000)) + np.uint32(0x2000)) | np.uint32(s)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got, reference_tf32(x).view(np.uint32))


def test_carry_into_the_exponent_and_small_values():
    # mantissa all ones above the cut: rounding up carries into the exponent
    x = np.array([np.nextafter(np.float32(2.0), np.float32(0.0)), -np.nextafter(np.float32(4.0), np.float32(0.0))],
                 dtype=np.float32)
    np.testing.assert_array_equal(add_and_mask(x), np.array([2.0, -4.0], dtype=np.float32))
    # subnormals and zero keep the same rule
    sub = np.array([0.0, -0.0, 1e-45, 3e-39, -5e-40], dtype=np.float32)
    np.testing.assert_array_equal(add_and_mask(sub).view(np.uint32), reference_tf32(sub).view(np.uint32))
    # values already in TF32 are unchanged
    t = add_and_mask(np.linspace(-100, 100, 1001, dtype=np.float32))
    np.testing.assert_array_equal(add_and_mask(t), t)
