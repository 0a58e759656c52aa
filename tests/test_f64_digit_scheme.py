"""The FP64 emulation of the tensor-core passes, checked on the CPU from its
definition (exact rational arithmetic, no GPU).

Each value a of a row with scale 2^r >= max |a| is written with six
balanced base-256 digits,
    a = 2^r (sum_{s=0..5} d_s 2^(-7-8s) + rho),  |d_s| <= 128,  |rho| <= 2^-48,
so every digit is an integer exactly representable in BF16.  A product of
two such expansions keeps the 21 digit products d_s e_t with s + t <= 5
(weights 2^(-14-8(s+t))) and drops the rest; each kept product is an exact
integer.  The result of a K-term dot product is then within
2^-43 K 2^(r_a + r_x) of the exact one, the bound the GPU tests hold every
output to.
"""
from fractions import Fraction

import numpy as np


def digits(y_num, y_exp):
    """Balanced base-256 digits of y = y_num 2^y_exp in [-1, 1] (exact ints):
    N = round(y 2^47), then digits from the bottom with carries."""
    shift = 47 + y_exp
    if shift >= 0:
        N = y_num << shift
    else:
        q, r = divmod(y_num, 1 << -shift)         # round to nearest, halves upward
        N = q + (1 if 2 * r >= (1 << -shift) else 0)
    d = [0] * 6
    for s in range(5, 0, -1):
        low = ((N + 128) % 256) - 128
        d[s] = low
        N = (N - low) // 256
    d[0] = N                          # the top digit takes the last carry: |d_0| <= 128
    assert abs(N) <= 128
    return d


def as_fraction(x):
    return Fraction(float(x))


def split(values, scale_exp):
    """Digits of every value relative to the power-of-two scale 2^scale_exp."""
    out = []
    for v in values:
        f = as_fraction(v) / Fraction(2) ** scale_exp
        num, den = f.numerator, f.denominator
        e = -(den.bit_length() - 1)
        assert den == 1 << -e
        out.append(digits(num, e))
    return out


def scale_exp_of(values):
    m = max(abs(float(v)) for v in values)
    return int(np.ceil(np.log2(m))) if m > 0 else 0


def test_digits_reconstruct_within_rho():
    rng = np.random.default_rng(0)
    vals = rng.standard_normal(500) * np.exp2(rng.integers(-30, 30, 500))
    r = scale_exp_of(vals)
    for v, d in zip(vals, split(vals, r)):
        assert all(abs(x) <= 128 for x in d)
        approx = sum(Fraction(x) * Fraction(2) ** (-7 - 8 * s) for s, x in enumerate(d))
        rho = as_fraction(v) / Fraction(2) ** r - approx
        assert abs(rho) <= Fraction(2) ** -48


def test_kept_digit_products_meet_the_bound():
    rng = np.random.default_rng(1)
    for K in (1, 7, 64, 256):
        a = rng.standard_normal(K) * np.exp2(rng.integers(-8, 8, K))
        x = rng.standard_normal(K) * np.exp2(rng.integers(-8, 8, K))
        ra, rx = scale_exp_of(a), scale_exp_of(x)
        da, dx = split(a, ra), split(x, rx)
        kept = Fraction(0)
        for ds, es in zip(da, dx):
            for s in range(6):
                for t in range(6 - s):
                    kept += Fraction(ds[s] * es[t]) * Fraction(2) ** (-14 - 8 * (s + t))
        kept *= Fraction(2) ** (ra + rx)
        exact = sum(as_fraction(p) * as_fraction(q) for p, q in zip(a, x))
        bound = Fraction(2) ** -43 * K * Fraction(2) ** (ra + rx)
        assert abs(kept - exact) <= bound


def test_dropping_a_kept_weight_breaks_the_bound():
    """Keeping only s + t <= 4 (15 products) drops the weight-5 products, up to
    2^-40 of the scales each: over 256 positive terms the error exceeds 2^-43 of
    the scales, which the 21-product form stays far below."""
    rng = np.random.default_rng(2)
    K = 256
    a = rng.uniform(0.5, 1.0, K)
    x = rng.uniform(0.5, 1.0, K)
    ra, rx = scale_exp_of(a), scale_exp_of(x)
    da, dx = split(a, ra), split(x, rx)
    kept = Fraction(0)
    for ds, es in zip(da, dx):
        for s in range(5):
            for t in range(5 - s):
                kept += Fraction(ds[s] * es[t]) * Fraction(2) ** (-14 - 8 * (s + t))
    kept *= Fraction(2) ** (ra + rx)
    exact = sum(as_fraction(p) * as_fraction(q) for p, q in zip(a, x))
    assert abs(kept - exact) > Fraction(2) ** -43 * Fraction(2) ** (ra + rx)
