"""FP8 E4M3 storage of A with per-tile scales -- TEST INFRASTRUCTURE ONLY.

The mixed form may read A stored as 8-bit floats in the E4M3 format with one
FP32 scale per 128 x 128 tile (the compressed-storage variant of the mixed
workload; the thesis itself stores A in full precision, Section 3.3).  The
oracle computes on the exactly dequantised matrix

    A[i, j] = e4m3(code[i, j]) * scale[i // 128, j // 128]

in FP64, so a GPU result is compared with the randomized SVD of the very
matrix it was given.

E4M3 (the OCP 8-bit floating-point format, "E4M3FN"): bit 7 sign, bits 6-3
exponent field e with bias 7, bits 2-0 mantissa m.
    e = 0:        (-1)^s * m/8 * 2^(1-7)        (subnormals, zero)
    1 <= e <= 15: (-1)^s * (1 + m/8) * 2^(e-7)  (normals)
except e = 15, m = 7, which is NaN; there are no infinities.  The largest
finite magnitude is 1.75 * 2^8 = 448.
"""
from __future__ import annotations

import numpy as np

TILE = 128


def decode_e4m3(codes) -> np.ndarray:
    """FP64 values of E4M3 codes (uint8 array), by the format definition."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    s = (c >> 7) & 1
    e = (c >> 3) & 15
    m = c & 7
    sign = np.where(s == 1, -1.0, 1.0)
    sub = sign * (m / 8.0) * 2.0 ** (1 - 7)
    nor = sign * (1.0 + m / 8.0) * np.power(2.0, (e - 7).astype(np.float64))
    out = np.where(e == 0, sub, nor)
    out = np.where((e == 15) & (m == 7), np.nan, out)
    return out


def dequantize_tiles(codes, scales, m: int, n: int, columns_as_rows: bool = False) -> np.ndarray:
    """A (m x n, FP64) from E4M3 codes and per-tile scales.

    codes: an m x n uint8 array, or (columns_as_rows=True) the device layout
    of a column-major matrix, an (n, lda) array whose row j is column j.
    scales: (m_tiles, n_tiles), tile (I, J) scaling rows 128 I .. 128 I + 127
    and columns 128 J .. 128 J + 127."""
    codes = np.asarray(codes)
    vals = decode_e4m3(codes[:, :m]).T if columns_as_rows else decode_e4m3(codes[:m, :n])
    s = np.asarray(scales, dtype=np.float64)
    rows = np.arange(m) // TILE
    cols = np.arange(n) // TILE
    return vals * s[np.ix_(rows, cols)]
