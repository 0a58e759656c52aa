"""The tensor engine of FP32 batches (tcgen05 grouped products) through the C ABI.

Each FP32 operand enters the MMAs as three BF16 slices (exact split) and the
six slice products with i + j <= 4 are summed in FP32, so every entry of
C = op(A) X must lie within the FP32 bound (K + 8) u32 (|op(A)| |X|)_ij of
the FP64 product of the same FP32 inputs (u32 = 2^-24).  Uneven products of
both forms, ragged tiles, odd leading dimensions, triangular X, skipped
entries, several column tiles and split contractions are covered; a product
must be bitwise the same alone and in the group, and from run to run.
"""
import numpy as np
import pytest
import torch

from paper_2402_17794_gb300 import rsvd as R

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _dev(a):
    """Column-major FP32 device copy of a 2-D float array (padded ld allowed)."""
    return torch.from_numpy(np.ascontiguousarray(a.T, dtype=np.float32)).cuda()


def _case(rng, M, K, N, trans, x_upper=False, pad=0):
    rows = K if trans else M
    cols = M if trans else K
    A = rng.standard_normal((rows + pad, cols)).astype(np.float32)
    X = rng.standard_normal((K + pad, N)).astype(np.float32)
    if x_upper:
        X[:K, :N] = np.triu(X[:K, :N])
    return A, X


def _run(plan, cases, trans):
    """cases: list of (A host (ld x cols), X host (ldx x N), M, K, N, x_upper)."""
    gemms, outs, keep = [], [], []
    for (A, X, M, K, N, xu) in cases:
        dA, dX = _dev(A), _dev(X)
        C = torch.full((N, max(M, 1) + 3), float("nan"), dtype=torch.float32, device="cuda")
        keep += [dA, dX]
        gemms.append((dA, A.shape[0], dX, X.shape[0], C, C.shape[1], M, K, N, xu))
        outs.append(C)
    plan.grouped_gemm(gemms, trans)
    torch.cuda.synchronize()
    assert R.rsvd_plan_status(plan.handle) == 0
    return [C.cpu().numpy().T for C in outs]   # (ldc x N)


def _check(cases, outs, trans):
    for (A, X, M, K, N, xu), C in zip(cases, outs):
        if M == 0:
            continue
        A64 = A.astype(np.float64)
        X64 = X[:K, :N].astype(np.float64)
        if xu:
            X64 = np.triu(X64)
        opA = A64[:K, :M].T if trans else A64[:M, :K]
        ref = opA @ X64
        bound = (K + 8) * U32 * (np.abs(opA) @ np.abs(X64))
        got = C[:M, :N].astype(np.float64)
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref)
        assert np.all(err <= bound), (M, K, N, trans, float((err / np.maximum(bound, 1e-300)).max()))


def _plan(max_count=16, rows=40000, cols=40000, l_max=288):
    return R.BatchPlan(max_count, rows, cols, l_max, R.F32)


@pytest.mark.parametrize("trans", [0, 1])
def test_grouped_products_within_fp32_bound(trans):
    rng = np.random.default_rng(10 + trans)
    shapes = [(128, 64, 16, False, 0), (300, 1000, 74, False, 3), (1, 5, 1, False, 0),
              (129, 77, 80, False, 1), (4099, 700, 33, False, 5), (777, 2500, 150, False, 0),
              (200, 200, 200, True, 0), (64, 9000, 20, False, 2), (0, 100, 10, False, 0),
              (513, 333, 288, False, 7)]
    cases = []
    for (M, K, N, xu, pad) in shapes:
        A, X = _case(rng, max(M, 1), K, N, trans, xu, pad)
        cases.append((A, X, M, K, N, xu))
    plan = _plan()
    outs = _run(plan, cases, trans)
    _check(cases, outs, trans)


@pytest.mark.parametrize("trans", [0, 1])
def test_grouped_product_same_alone_and_in_group(trans):
    rng = np.random.default_rng(20 + trans)
    shapes = [(1000, 3000, 40), (130, 9000, 74), (2048, 256, 64), (77, 77, 77), (5000, 120, 16)]
    cases = []
    for (M, K, N) in shapes:
        A, X = _case(rng, M, K, N, trans, False, 1)
        cases.append((A, X, M, K, N, False))
    plan = _plan()
    together = _run(plan, cases, trans)
    again = _run(plan, cases, trans)
    for c, a, b in zip(cases, together, again):
        assert np.array_equal(a[:c[2], :c[4]], b[:c[2], :c[4]])
    for i, c in enumerate(cases):
        alone = _run(plan, [c], trans)[0]
        M, N = c[2], c[4]
        assert np.array_equal(alone[:M, :N], together[i][:M, :N]), i


def test_grouped_product_rejects_bad_arguments():
    plan = _plan(max_count=2)
    a = torch.zeros(4, 4, dtype=torch.float32, device="cuda")
    good = (a, 4, a, 4, a, 4, 4, 4, 4, 0)
    bad_ld = (a, 2, a, 4, a, 4, 4, 4, 4, 0)
    arr = [R._lib.RsvdGemm(R._ptr(g[0]), g[1], R._ptr(g[2]), g[3], R._ptr(g[4]), g[5], g[6], g[7],
                           g[8], g[9]) for g in (good, bad_ld)]
    assert R.rsvd_grouped_gemm_f32(plan.handle, arr, 0) == -101
    assert R.rsvd_grouped_gemm_f32(plan.handle, arr * 2, 0) == -2
    p64 = R.BatchPlan(2, 100, 100, 16, R.F64)
    assert R.rsvd_grouped_gemm_f32(p64.handle, arr[:1], 0) == -1
    assert R.rsvd_batch_set_engine(p64.handle, R.BATCH_ENGINE_TENSOR) == 7


def test_grouped_product_wait_limit_expires_and_recovers():
    """A wait limit of a few cycles makes the pipeline waits expire: the launch
    reports RSVD_ERR_TIMEOUT through rsvd_plan_status and leaves the context
    usable; with the default limit the same products are correct again."""
    rng = np.random.default_rng(30)
    A, X = _case(rng, 3000, 2000, 64, 0)
    cases = [(A, X, 3000, 2000, 64, False)]
    plan = _plan(max_count=2)
    assert R.rsvd_plan_set_wait_limit(plan.handle, 8) == 0
    gem = [(_dev(A), A.shape[0], _dev(X), X.shape[0],
            torch.zeros(64, 3000, dtype=torch.float32, device="cuda"), 3000, 3000, 2000, 64, False)]
    plan.grouped_gemm(gem, 0)
    torch.cuda.synchronize()
    assert R.rsvd_plan_status(plan.handle) == 3
    assert R.rsvd_plan_set_wait_limit(plan.handle, 0) == 0
    outs = _run(plan, cases, 0)
    _check(cases, outs, 0)


def test_tensor_engine_batch_matches_simt_engine():
    """The same FP32 batch on both engines: sigma agree to FP32 accuracy."""
    from paper_2402_17794_gb300 import synthetic as syn
    rng = np.random.default_rng(40)
    items = []
    for i in range(12):
        m = int(rng.integers(200, 3000))
        n = int(rng.integers(200, 1500))
        k = int(rng.integers(10, 60))
        A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n, 300), r=30.0), seed=500 + i)
        items.append((R.from_numpy_f(A, dtype=torch.float32), m, n, k, 10, 1, 90 + i))
    rows = sum(it[1] for it in items)
    cols = sum(it[2] for it in items)
    res = {}
    for eng in (R.BATCH_ENGINE_SIMT, R.BATCH_ENGINE_TENSOR):
        plan = R.BatchPlan(len(items), rows, cols, 74, R.F32)
        plan.set_engine(eng)
        out = plan.solve(items)
        torch.cuda.synchronize()
        assert plan.status() == [0] * len(items)
        res[eng] = [o[1].cpu().numpy() for o in out]
    for s0, s1 in zip(res[R.BATCH_ENGINE_SIMT], res[R.BATCH_ENGINE_TENSOR]):
        assert np.max(np.abs(s0 - s1)) <= 1e-5 * s0[0]


def test_autotune_then_alone_equals_mix():
    """After rsvd_batch_autotune a problem's schedule depends only on its own
    shape: solved alone it gives the same bits as inside the tuned batch."""
    from paper_2402_17794_gb300 import synthetic as syn
    rng = np.random.default_rng(50)
    items = []
    for i in range(10):
        m = int(rng.integers(300, 5000))
        n = int(rng.integers(300, 2000))
        k = int(rng.integers(10, 60))
        A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n, 300), r=20.0), seed=700 + i)
        items.append((R.from_numpy_f(A, dtype=torch.float32), m, n, k, 10, 1, 30 + i))
    rows = sum(it[1] for it in items)
    cols = sum(it[2] for it in items)
    plan = R.BatchPlan(len(items), rows, cols, 74, R.F32)
    plan.autotune(items)
    mix = plan.solve(items)
    torch.cuda.synchronize()
    assert plan.status() == [0] * len(items)
    for i in (0, 3, 9):
        alone = plan.solve([items[i]])
        torch.cuda.synchronize()
        assert plan.status() == [0]
        for a, b in zip(alone[0], mix[i]):
            assert torch.equal(a, b), i


@pytest.mark.parametrize("trans", [0, 1])
def test_grouped_product_has_no_accumulation_bias(trans):
    """Positive operands over a long contraction (K = 16384, 256 blocks): the
    tensor cores round their internal sums toward zero, so an accumulator
    kept across the whole contraction would drift low by hundreds of u32.
    With one accumulator per 64-deep block and round-to-nearest running
    sums, the mean relative error stays within a few u32."""
    rng = np.random.default_rng(60 + trans)
    M, K, N = 256, 16384, 64
    A = rng.random((K, M) if trans else (M, K)).astype(np.float32)
    X = rng.random((K, N)).astype(np.float32)
    plan = _plan(rows=40000, cols=40000)
    out = _run(plan, [(A, X, M, K, N, False)], trans)[0][:M, :N].astype(np.float64)
    opA = A.astype(np.float64).T if trans else A.astype(np.float64)
    ref = opA @ X.astype(np.float64)
    e = (out - ref) / ref
    assert abs(e.mean()) <= 24 * U32, e.mean() / U32
    assert np.abs(e).max() <= 96 * U32, np.abs(e).max() / U32


def test_graph_replays_match_direct_solves():
    """rsvd_batch_set_graphs: the first solve captures the grouped solve as a
    CUDA graph, later solves of the same shapes replay it with new operands
    and seeds; every result equals the same solve launched directly."""
    from paper_2402_17794_gb300 import synthetic as syn
    rng = np.random.default_rng(70)
    shapes = [(int(rng.integers(300, 3000)), int(rng.integers(300, 1500)), int(rng.integers(10, 60)))
              for _ in range(8)]

    def batch(seed0):
        return [(R.from_numpy_f(syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n, 300), r=25.0),
                                                   seed=seed0 + i), dtype=torch.float32),
                 m, n, k, 10, 1, seed0 + 7 * i) for i, (m, n, k) in enumerate(shapes)]

    a, b = batch(100), batch(200)
    rows = sum(s[0] for s in shapes)
    cols = sum(s[1] for s in shapes)
    stream = torch.cuda.Stream()
    direct = R.BatchPlan(len(shapes), rows, cols, 74, R.F32, stream=stream)
    out = direct.solve(a)
    stream.synchronize()
    ref_a = [tuple(t.clone() for t in o) for o in out]
    out = direct.solve(b)
    stream.synchronize()
    ref_b = [tuple(t.clone() for t in o) for o in out]
    graph = R.BatchPlan(len(shapes), rows, cols, 74, R.F32, stream=stream)
    graph.set_graphs(True)
    for items, ref in ((a, ref_a), (b, ref_b), (a, ref_a)):
        out = graph.solve(items)
        stream.synchronize()
        assert graph.status() == [0] * len(shapes)
        for o, r in zip(out, ref):
            for x, y in zip(o, r):
                assert torch.equal(x, y)
    p64 = R.BatchPlan(2, 100, 100, 16, R.F64, stream=stream)
    assert R.rsvd_batch_set_graphs(p64.handle, 1) == 7
    nostream = R.BatchPlan(2, 100, 100, 16, R.F32)
    assert R.rsvd_batch_set_graphs(nostream.handle, 1) == -2
