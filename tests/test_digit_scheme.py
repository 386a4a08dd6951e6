"""The exact-digit scheme behind the tensor-core double-float projections, checked on the CPU.

The GPU kernels (oz_gemm.cu) write each row of 49-bit fixed-point values as seven balanced
base-128 digits and sum digit products by group g = t + u in FP32 chains of 512 values. The claims
their exactness rests on are checked here with exact integer arithmetic (Python ints / int64):

* the digits reconstruct the integer exactly, |m_0| <= 128 and |m_t| <= 64 for t >= 1, so every
  digit is exact in bf16 (8 significant bits);
* the worst-case magnitude of a group's sum over a 512-value chain stays below 2^24 for g <= 3 (so
  FP32 accumulation of integers is exact), and the int32 totals over 127 chains stay below 2^31;
* the scheme's dot product (groups 0..6, products t + u >= 7 dropped) is within its stated bound
  of the exact dot product of the fixed-point inputs, and within ~2^-46 of the exact dot product
  of the double inputs relative to max|a| max|b| K, on rows with a realistic spread of magnitudes.
"""

from fractions import Fraction

import numpy as np

T, BITS, CHAIN = 7, 7, 512


def digits(I):
    """Balanced base-128 digits m_0 .. m_{T-1} of an integer (most significant first)."""
    d = [0] * T
    for t in range(T - 1, 0, -1):
        m = ((I + 64) & 127) - 64
        d[t] = m
        I = (I - m) >> 7
    d[0] = I
    return d


def row_digits(v):
    """Exponent E (every |v| < 2^E) and the digits of round(v 2^(7T - E)) for one row."""
    m = float(np.max(np.abs(v)))
    E = int(np.frexp(m)[1]) if m > 0 else 0  # m < 2^E
    ints = [int(round(Fraction(float(x)) * Fraction(2) ** (BITS * T - E))) for x in v]
    return E, ints, np.array([digits(i) for i in ints], dtype=np.int64)


def test_digits_reconstruct_and_fit_bf16():
    rng = np.random.default_rng(1)
    for I in list(rng.integers(-(2 ** 49), 2 ** 49, 20000)) + [2 ** 49, -(2 ** 49), 0, 1, -1, 63, 64, -64, -65]:
        I = int(I)
        d = digits(I)
        assert sum(m * 128 ** (T - 1 - t) for t, m in enumerate(d)) == I
        assert abs(d[0]) <= 128 and all(-64 <= m <= 63 for m in d[1:])


def test_group_chains_are_exact_in_fp32():
    # largest |sum over a chain| of the products of group g, digits at their bounds
    top, rest = 128, 64
    for g in range(4):
        per_value = sum((top if t == 0 else rest) * (top if g - t == 0 else rest) for t in range(g + 1))
        assert per_value * CHAIN < 2 ** 24, g
    assert 127 * 2 ** 24 < 2 ** 31  # int32 totals of a split's chains


def scheme_dot(a, b):
    """The kernels' arithmetic for one output: exact group sums, groups 0..6, scaled back."""
    Ea, _, da = row_digits(a)
    Eb, _, db = row_digits(b)
    total = Fraction(0)
    for g in range(T):
        s = 0
        for t in range(g + 1):
            s += int(np.dot(da[:, t], db[:, g - t]))
        total += Fraction(s) * Fraction(2) ** (Ea + Eb - 14 - BITS * g)
    return total, Ea, Eb


def test_dot_products_meet_their_bound():
    rng = np.random.default_rng(7)
    K = 1500  # three chains, the last ragged
    for trial in range(6):
        # plane-wave-like rows: magnitudes decaying over three decades, random signs
        a = rng.standard_normal(K) * np.exp(-np.linspace(0, 7, K)) * (10.0 ** rng.integers(-5, 5))
        b = rng.standard_normal(K) * np.exp(-np.linspace(0, 4, K)[::-1])
        if trial == 5:
            b[: K // 2] = 0.0
        got, Ea, Eb = scheme_dot(a, b)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        scale = Fraction(float(np.max(np.abs(a)))) * Fraction(float(np.max(np.abs(b)))) * K
        err = abs(got - exact) / scale
        # fixed-point rounding of both inputs (2^-49 of 2^E each) and the dropped products (t + u >= 7,
        # at most 6 x 64 x 64 x 2^-63 of 2^(Ea + Eb) per value): ~2^-46 of max|a| max|b| per value
        assert float(err) < 2.0 ** -46, (trial, float(err))
