"""The tensor engine's work schedule (host logic, no GPU): rsvd_grouped_schedule.

Every output tile of every product is covered exactly once, by units whose
contraction ranges partition the product's 64-deep blocks; split tiles get
distinct partial slots; column tiles follow the product's own N; units are
dealt longest first, so no CTA carries more than the average load plus one
unit; and a product's units do not depend on what else is scheduled with it
(the property that keeps a batched result the same alone and in a mix).
"""
import math

import numpy as np
import pytest

from paper_2402_17794_gb300 import _build, rsvd as R


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        _build.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not available")
    _build.build()


def tile_of(N):
    tiles = math.ceil(N / 80)
    return math.ceil(math.ceil(N / tiles) / 16) * 16


def shapes_of(rng, count, trans):
    out = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(256), np.log(4096))))
        n = int(rng.integers(256, 2049))
        l = int(rng.integers(20, 75))
        out.append((n, m, l) if trans else (m, n, l))
    out += [(0, 500, 40), (300, 9000, 150), (129, 77, 288), (1, 1, 1)]
    return out


@pytest.mark.parametrize("trans", [0, 1])
def test_units_cover_every_tile_once(trans):
    rng = np.random.default_rng(3 + trans)
    shapes = shapes_of(rng, 60, trans)
    units, cta, info = R.rsvd_grouped_schedule(shapes, trans, 152)
    assert info[0] == len(units) and info[1] == len(cta) - 1 and cta[0] == 0 and cta[-1] == len(units)
    cover = {}
    slots = []
    for (p, r0, c0, k0, k1, slot, t) in units:
        M, K, N = shapes[p]
        assert M > 0 and 0 <= r0 < M and r0 % 128 == 0
        assert t == tile_of(N) and 0 <= c0 < N and c0 % t == 0
        assert 0 <= k0 < k1 <= math.ceil(K / 64)
        cover.setdefault((p, r0, c0), []).append((k0, k1, slot))
        if slot >= 0:
            slots.append(slot)
    assert len(slots) == len(set(slots)) == info[2]
    for p, (M, K, N) in enumerate(shapes):
        if M == 0:
            assert not any(key[0] == p for key in cover)
            continue
        t = tile_of(N)
        for r0 in range(0, M, 128):
            for c0 in range(0, N, t):
                parts = sorted(cover.pop((p, r0, c0)))
                assert parts[0][0] == 0 and parts[-1][1] == math.ceil(K / 64)
                for a, b in zip(parts, parts[1:]):
                    assert a[1] == b[0]
                if len(parts) == 1:
                    assert parts[0][2] == -1
                else:
                    assert all(s >= 0 for (_, _, s) in parts)
    assert not cover
    assert info[3] == max(tile_of(N) for (M, K, N) in shapes if M > 0)


def test_long_contractions_split_into_default_chunks():
    units, _, info = R.rsvd_grouped_schedule([(300, 9000, 20), (300, 4096, 20)], 0, 8)
    kbs = sorted((k0, k1) for (p, r0, c0, k0, k1, s, t) in units if p == 0 and r0 == 0)
    assert kbs == [(0, 47), (47, 94), (94, 141)]          # 141 blocks in 3 chunks of <= 64
    assert all(s == -1 for (p, *_r, s, t) in units if p == 1)   # 64 blocks: one unit
    assert info[2] == 3 * 3                                 # three row tiles of product 0


@pytest.mark.parametrize("num_sms", [152, 37, 1])
def test_longest_first_dealing_balances_the_load(num_sms):
    rng = np.random.default_rng(9)
    shapes = shapes_of(rng, 200, 0)
    units, cta, info = R.rsvd_grouped_schedule(shapes, 0, num_sms)
    cost = [k1 - k0 + 2 for (p, r0, c0, k0, k1, s, t) in units]
    loads = [sum(cost[cta[c]:cta[c + 1]]) for c in range(info[1])]
    assert info[1] == min(num_sms, len(units))
    assert max(loads) <= sum(cost) / info[1] + max(cost)


@pytest.mark.parametrize("trans", [0, 1])
def test_a_products_units_do_not_depend_on_the_mix(trans):
    rng = np.random.default_rng(21)
    shapes = shapes_of(rng, 40, trans)
    mixed, _, _ = R.rsvd_grouped_schedule(shapes, trans, 152)
    for p in (0, 7, len(shapes) - 3):
        alone, _, _ = R.rsvd_grouped_schedule([shapes[p]], trans, 152)
        want = sorted((r0, c0, k0, k1, s >= 0, t) for (_, r0, c0, k0, k1, s, t) in alone)
        got = sorted((r0, c0, k0, k1, s >= 0, t) for (q, r0, c0, k0, k1, s, t) in mixed if q == p)
        assert got == want


def test_schedule_rejects_bad_arguments():
    import ctypes
    lib = R._lib.load()
    info = (ctypes.c_int * 4)()
    shp = (ctypes.c_int64 * 3)(10, 10, 10)
    assert lib.rsvd_grouped_schedule(0, shp, 0, 8, None, 0, None, info) == -1
    assert lib.rsvd_grouped_schedule(1, None, 0, 8, None, 0, None, info) == -2
    assert lib.rsvd_grouped_schedule(1, shp, 0, 0, None, 0, None, info) == -3
    bad = (ctypes.c_int64 * 3)(10, 10, 300)
    assert lib.rsvd_grouped_schedule(1, bad, 0, 8, None, 0, None, info) == -100
    small = (ctypes.c_int * 7)()
    two = (ctypes.c_int64 * 3)(300, 10, 10)
    assert lib.rsvd_grouped_schedule(1, two, 0, 8, small, 1, None, info) == 4
    assert info[0] == 3
