"""The numerical scheme of the FP32 tensor engine, checked on the CPU.

An FP32 value v splits into three BF16 values v = v1 + v2 + v3 (v1 = bf16(v),
v2 = bf16(v - v1), v3 = bf16(v - v1 - v2), round to nearest even, each
remainder exact in FP32).  The split is exact while v3 is a normal BF16
number, |v| >= 2^-110; below that BF16's subnormal step (2^-133) limits v3,
and the split's error is at most 2^-134 absolute.  A product keeps the six slice
products a_i x_j with i + j <= 4.  The dropped terms a2 x3 + a3 x2 + a3 x3
are below 2^-23 of |a x|, so a dot product of length K computed that way
differs from the exact one by at most 2^-23 sum |a_k x_k| before any
accumulation rounding.  BF16 rounding is written out here from the format's
definition (the top 16 bits of an FP32 word, round to nearest even).
"""
import numpy as np


def bf16_rn(v):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    b = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, dtype=np.float32)
    v1 = bf16_rn(v)
    r1 = (v - v1).astype(np.float32)
    v2 = bf16_rn(r1)
    r2 = (r1 - v2).astype(np.float32)
    v3 = bf16_rn(r2)
    return v1, v2, v3


def finite_fp32(rng, n, lo=-60, hi=60):
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return (mant * np.exp2(rng.integers(lo, hi, n))).astype(np.float32)


def test_bf16_rounding_matches_definition():
    # values exactly halfway between two BF16 numbers go to the even one
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)
    assert bf16_rn(one + ulp / 2) == one                       # 1 is even
    assert bf16_rn(one + ulp + ulp / 2) == one + 2 * ulp       # 1 + ulp is odd
    assert bf16_rn(np.float32(-1.5)) == np.float32(-1.5)       # representable stays
    x = finite_fp32(np.random.default_rng(0), 10000)
    r = bf16_rn(x)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)            # 8 significant bits
    assert np.all(np.abs(r.astype(np.float64) - x) <= np.abs(x) * 2.0 ** -8)


def test_three_slices_are_exact_above_the_subnormal_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([finite_fp32(rng, 200000), finite_fp32(rng, 1000, -140, -120),
                        np.array([0.0, -0.0, 1.0, 3.0e38, -3.0e38], np.float32)])
    v1, v2, v3 = split3(x)
    for s in (v1, v2, v3):
        assert np.all((s.view(np.uint32) & 0xFFFF) == 0)        # each slice is a BF16 value
    total = v1.astype(np.float64) + v2.astype(np.float64) + v3.astype(np.float64)
    big = np.abs(x) >= 2.0 ** -110
    assert big.sum() > 200000 and (~big).sum() >= 1000
    assert np.array_equal(total[big], x[big].astype(np.float64))
    assert np.all(np.abs(total[~big] - x[~big].astype(np.float64)) <= 2.0 ** -134)
    normal = np.abs(x) > 2.0 ** -100
    assert np.all(np.abs(v2[normal]) <= np.abs(x[normal]) * 2.0 ** -8)
    assert np.all(np.abs(v3[normal]) <= np.abs(x[normal]) * 2.0 ** -16)


def test_six_slice_products_bound():
    rng = np.random.default_rng(2)
    for K in (1, 16, 1000, 4096):
        a = finite_fp32(rng, K, -20, 20)
        x = finite_fp32(rng, K, -20, 20)
        a1, a2, a3 = (s.astype(np.float64) for s in split3(a))
        x1, x2, x3 = (s.astype(np.float64) for s in split3(x))
        # each slice product is exact in FP64 (8 x 8 significant bits)
        six = a1 * (x1 + x2 + x3) + a2 * (x1 + x2) + a3 * x1
        dropped = a2 * x3 + a3 * x2 + a3 * x3
        exact = a.astype(np.float64) * x.astype(np.float64)
        assert np.allclose(six + dropped, exact, rtol=0, atol=0) or \
            np.all(np.abs(six + dropped - exact) <= np.abs(exact) * 2.0 ** -52)
        assert np.all(np.abs(dropped) <= np.abs(exact) * 2.0 ** -23)
        dot_err = abs(six.sum() - exact.sum())
        assert dot_err <= 2.0 ** -23 * np.abs(exact).sum() + 1e-300


def test_a_planted_mistake_is_caught():
    """Keeping only a1 x1 + a1 x2 + a2 x1 (dropping the 2^-16 terms) breaks the bound."""
    rng = np.random.default_rng(3)
    a = finite_fp32(rng, 4096, -5, 5)
    x = finite_fp32(rng, 4096, -5, 5)
    a1, a2, a3 = (s.astype(np.float64) for s in split3(a))
    x1, x2, x3 = (s.astype(np.float64) for s in split3(x))
    exact = a.astype(np.float64) * x.astype(np.float64)
    three = a1 * x1 + a1 * x2 + a2 * x1
    assert np.max(np.abs(three - exact) / np.abs(exact)) > 2.0 ** -23
