"""Pins of the FP8 (E4M3 + per-tile scale) dequantisation used by the oracle.

The decoder follows the format's definition (sign, 4-bit exponent of bias 7,
3-bit mantissa, subnormals at exponent field 0, S.1111.111 NaN, no
infinities); it is pinned to hand-derived values of that definition, to a
library decoder (torch.float8_e4m3fn) over all 256 codes, and to the
format's order.  Dequantisation is pinned on tiles of known scale.
"""
import numpy as np
import pytest

from oracle import fp8


@pytest.mark.parametrize("code,value", [
    (0x00, 0.0), (0x01, 2.0 ** -9), (0x07, 7 * 2.0 ** -9), (0x08, 2.0 ** -6),
    (0x38, 1.0), (0x3C, 1.5), (0x40, 2.0), (0x7E, 448.0), (0xFE, -448.0),
    (0xB8, -1.0), (0x30, 0.5), (0x39, 1.125),
])
def test_decode_known_codes(code, value):
    assert fp8.decode_e4m3(np.array([code], dtype=np.uint8))[0] == value


def test_decode_nan_and_signed_zero():
    v = fp8.decode_e4m3(np.array([0x7F, 0xFF, 0x80], dtype=np.uint8))
    assert np.isnan(v[0]) and np.isnan(v[1])
    assert v[2] == 0.0 and np.signbit(v[2])


def test_decode_matches_library_for_all_codes():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ours = fp8.decode_e4m3(codes)
    lib = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(ours), np.isnan(lib))
    ok = ~np.isnan(ours)
    assert np.array_equal(ours[ok], lib[ok])


def test_positive_codes_increase_strictly():
    v = fp8.decode_e4m3(np.arange(0x00, 0x7F, dtype=np.uint8))
    assert np.all(np.diff(v) > 0)


def test_dequantize_applies_the_tile_scale():
    m, n = 300, 260
    codes = np.full((m, n), 0x38, dtype=np.uint8)      # every code is 1.0
    scales = np.array([[2.0 ** (i + 3 * j) for j in range(3)] for i in range(3)])
    A = fp8.dequantize_tiles(codes, scales, m, n)
    for i in (0, 127, 128, 255, 256, 299):
        for j in (0, 127, 128, 259):
            assert A[i, j] == scales[i // 128, j // 128]


def test_dequantize_row_per_column_layout():
    rng = np.random.default_rng(0)
    m, n, lda = 150, 140, 160
    codes = rng.integers(0, 0x7E, size=(m, n)).astype(np.uint8)
    stored = np.zeros((n, lda), dtype=np.uint8)       # row j = column j of A
    stored[:, :m] = codes.T
    scales = np.array([[0.5, 4.0], [2.0, 0.25]])
    a = fp8.dequantize_tiles(codes, scales, m, n)
    b = fp8.dequantize_tiles(stored, scales, m, n, columns_as_rows=True)
    assert np.array_equal(a, b)
