"""The allocation-free FP64 Y = A X entry point (GPU required).

For callers that may not allocate device memory (they run inside a host
framework that owns the device memory, or were handed only inputs and
outputs), rsvd_apply_a_f64_static keeps its split-K partials in a fixed
array inside the library.  This checks, through the C ABI, that two calls in
a row give the host's FP64 product a @ x (numpy, independent of the GPU) and
the plan-based rsvd_apply_a, both within the FP64 test tolerance (64 ulps of
max |A||X|), and that a size beyond the fixed array is refused.  The file
sorts last so a stop-at-first-failure run has already run every other test;
it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2402_17794_gb300 import rsvd as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_static_scratch_product_matches_host_product_and_plan_entry_point():
    m, n, l = 12000, 9000, 80          # m * l = 960000 <= 4 Mi: several split-K slices fit
    rng = np.random.default_rng(123)
    lda = m + 5
    A = torch.zeros(n, lda, dtype=torch.float64, device="cuda")
    A[:, :m] = torch.from_numpy(rng.standard_normal((n, m))).cuda()
    X = torch.from_numpy(rng.standard_normal((l, n))).cuda()
    plan = R.Plan(m, n, l)
    Y_ref = torch.empty(l, m, dtype=torch.float64, device="cuda")
    assert R.rsvd_apply_a(plan.handle, A, m, n, lda, X, n, l, Y_ref, m) == 0
    assert plan.status() == 0
    a = A[:, :m].cpu().numpy().T
    x = X.cpu().numpy().T
    tol = 64 * 2.0 ** -52 * (np.abs(a) @ np.abs(x)).max()
    host = (a @ x).T                   # (l, m): the layout of the device output
    ref = Y_ref.cpu().numpy()
    for _ in range(2):
        Y = torch.full((l, m), float("nan"), dtype=torch.float64, device="cuda")
        assert R.rsvd_apply_a_f64_static(A, m, n, lda, X, n, l, Y, m) == 0
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - host).max() <= tol
        assert np.abs(got - ref).max() <= tol


def test_static_scratch_rejects_sizes_beyond_its_array():
    m, n, l = (1 << 16) + 1, 64, 64    # m * l > 4 Mi
    A = torch.zeros(n, m, dtype=torch.float64, device="cuda")
    X = torch.zeros(l, n, dtype=torch.float64, device="cuda")
    Y = torch.full((l, m), 7.0, dtype=torch.float64, device="cuda")
    assert R.rsvd_apply_a_f64_static(A, m, n, m, X, n, l, Y, m) == 4
    torch.cuda.synchronize()
    assert bool((Y == 7.0).all())
