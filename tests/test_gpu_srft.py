"""Parity of the SRFT sketch and FastRandRF (the toolbox's SRFT and
FastRandRF; Halko, Martinsson and Tropp 2011, Algorithm 4.5) with the CPU
oracle through the C ABI (GPU required).

Same seed on both sides: the same phases D (Philox stream 2) and the same
Floyd sample R (Philox stream 3), each side implementing the generator from
its definition.  The sample R is integer work and must match exactly; the
GPU returns it through the sketch's columns, so a wrong coordinate shows as
an O(1) column mismatch.  Y = A Omega within 1e-12 of max |Y| (FP64
products over n terms).  Q columns are Gram-Schmidt vectors with
q_c^H y_c > 0 on both sides (the oracle's Householder Q is rotated to that
normalisation): elementwise within 1e-9; Q^H Q = I within 1e-12; the range
error ||A - Q Q^H A||_2 within 1.0001x the oracle's.
"""
import numpy as np
import pytest
import torch

from oracle import srft
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _device(A, lda_pad=0):
    m, n = A.shape
    dA = torch.zeros(n, m + lda_pad, dtype=torch.float64, device="cuda")
    dA[:, :m] = R.from_numpy_f(A)
    return dA, m + lda_pad


def _complex(planar, l):
    x = R.to_numpy_f(planar)      # m x 2l
    return x[:, :l] + 1j * x[:, l:]


def _range_err(A, Q):
    return np.linalg.norm(A - Q @ (Q.conj().T @ A), 2)


@pytest.mark.parametrize("m,n,l,lda_pad", [
    (300, 256, 16, 0), (777, 512, 40, 3), (1000, 97, 24, 0), (513, 640, 64, 0),
    (2048, 1024, 80, 0), (256, 8192, 72, 0),
])
def test_sketch_and_range_match_oracle(m, n, l, lda_pad):
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n), r=10.0), seed=m + n)
    ref = srft.fast_range_finder(A, l, seed=l)
    dA, lda = _device(A, lda_pad)
    plan = R.Plan(m, n, 2 * l)
    Y = plan.srft_sketch(dA, m, n, l, seed=l, lda=lda)
    Q = plan.range_srft(dA, m, n, l, seed=l, lda=lda)
    assert plan.status() == 0
    y = _complex(Y, l)
    assert np.abs(y - ref.Y).max() <= 1e-12 * np.abs(ref.Y).max()
    q = _complex(Q, l)
    assert np.abs(q.conj().T @ q - np.eye(l)).max() <= 1e-12
    qo = srft.gram_schmidt_phases(ref.Q, ref.Y)
    assert np.abs(q - qo).max() <= 1e-9, np.abs(q - qo).max()
    e_gpu, e_orc = _range_err(A, q), _range_err(A, ref.Q)
    assert e_gpu <= 1.0001 * e_orc + 1e-15, (e_gpu, e_orc)


def test_exact_capture_and_low_rank():
    m, n, k, l = 900, 640, 12, 20
    A = syn.lowrank_matrix(m, n, np.geomspace(1.0, 1e-3, k), seed=3)
    dA, lda = _device(A)
    plan = R.Plan(m, n, 2 * l)
    q = _complex(plan.range_srft(dA, m, n, l, seed=5), l)
    assert plan.status() == 0
    assert _range_err(A, q) <= 1e-13


def test_srft_argument_errors():
    plan = R.Plan(100, 80, 20)
    A = torch.zeros(80, 100, dtype=torch.float64, device="cuda")
    Q = torch.zeros(40, 100, dtype=torch.float64, device="cuda")
    f = R.rsvd_range_srft
    assert f(plan.handle, A, 100, 80, 99, 8, 0, Q, 100) == -5
    assert f(plan.handle, A, 100, 80, 100, 0, 0, Q, 100) == -6
    assert f(plan.handle, A, 100, 80, 100, 81, 0, Q, 100) == -6
    assert f(plan.handle, A, 100, 80, 100, 8, 0, Q, 99) == -9
    assert f(plan.handle, A, 100, 80, 100, 11, 0, Q, 100) == 4   # 2l > plan l_max
    assert f(plan.handle, A, 100, 80, 100, 10, 0, Q, 100) == 0
    assert plan.status() == 0


def test_srft_config_full_size_fp64():
    """The benchmark's FastRandRF: A 16384 x 8192 FP64, Haar factors,
    sigma_i = i^-1.5, l = 80, through the FFT form of the sketch."""
    m, n, l, seed = 16384, 8192, 80, 2
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = np.asfortranarray(dA.cpu().numpy().T)
    Om = srft.srft_matrix(n, l, seed)
    Yo = A @ Om.real + 1j * (A @ Om.imag)
    Qo = srft.gram_schmidt_phases(np.linalg.qr(Yo)[0], Yo)
    plan = R.Plan(m, n, 2 * l)
    Y = plan.srft_sketch(dA, m, n, l, seed)
    Q = plan.range_srft(dA, m, n, l, seed)
    assert plan.status() == 0
    y, q = _complex(Y, l), _complex(Q, l)
    assert np.abs(y - Yo).max() <= 1e-12 * np.abs(Yo).max()
    assert np.abs(q.conj().T @ q - np.eye(l)).max() <= 1e-12
    assert np.abs(q - Qo).max() <= 1e-9, np.abs(q - Qo).max()


@pytest.mark.parametrize("m,n,k,p,lda_pad", [(700, 512, 16, 8, 0), (513, 640, 30, 10, 3),
                                            (1000, 97, 12, 6, 0)])
def test_solve_srft_matches_oracle(m, n, k, p, lda_pad):
    """FastRandRF + Stage B on the complex basis against the oracle's
    srft_rsvd: sigma within 1e-10 relative, U and V^H within 1e-8 after the
    shared phase convention, U S V^H within 1e-10 sigma_1."""
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n), r=8.0), seed=m + 2 * n)
    ref = srft.srft_rsvd(A, k, p, seed=k)
    dA, lda = _device(A, lda_pad)
    plan = R.Plan(m, n, 2 * (k + p))
    U, S, VT = plan.solve_srft(dA, m, n, k, p, seed=k, lda=lda)
    assert plan.status() == 0
    s = S.cpu().numpy()
    assert (np.abs(s - ref.S) / ref.S).max() <= 1e-10
    u = _complex(U, k)
    vt_planar = R.to_numpy_f(VT)          # k x 2n
    vt = vt_planar[:, :n] + 1j * vt_planar[:, n:]
    assert np.abs(u.conj().T @ u - np.eye(k)).max() <= 1e-12
    assert np.abs(vt @ vt.conj().T - np.eye(k)).max() <= 1e-12
    assert np.abs(u - ref.U).max() <= 1e-8, np.abs(u - ref.U).max()
    assert np.abs(vt - ref.Vt).max() <= 1e-8, np.abs(vt - ref.Vt).max()
    rec = (u * s) @ vt
    rec_o = (ref.U * ref.S) @ ref.Vt
    assert np.abs(rec - rec_o).max() <= 1e-10 * ref.S[0]


@pytest.mark.parametrize("k,p", [(12, 8), (6, 10)])
def test_solve_srft_repeated_singular_values(k, p):
    """Stage B when singular values repeat (exactly, up to rounding): A of
    rank 12 with sigma = (3, 2, 2, 1, 1, 1, 0.5, 0.5, 0.25, 0.1, 0.1, 0.1),
    captured exactly by the range.  The complex triplets must stay complex
    orthonormal (U^H U = I, V V^H = I), sigma must match the oracle to 1e-10,
    and U S V^H must reproduce the oracle's rank-k approximation (unique: k
    ends on a gap)."""
    sig = np.array([3.0, 2.0, 2.0, 1.0, 1.0, 1.0, 0.5, 0.5, 0.25, 0.1, 0.1, 0.1])
    m, n = 600, 512
    A = syn.lowrank_matrix(m, n, sig, seed=31)
    ref = srft.srft_rsvd(A, k, p, seed=5)
    dA, lda = _device(A)
    plan = R.Plan(m, n, 2 * (k + p))
    U, S, VT = plan.solve_srft(dA, m, n, k, p, seed=5, lda=lda)
    assert plan.status() == 0
    s = S.cpu().numpy()
    assert (np.abs(s - ref.S) / ref.S).max() <= 1e-10
    assert np.abs(s - sig[:k]).max() <= 1e-12 * sig[0]
    u = _complex(U, k)
    vt_planar = R.to_numpy_f(VT)
    vt = vt_planar[:, :n] + 1j * vt_planar[:, n:]
    assert np.abs(u.conj().T @ u - np.eye(k)).max() <= 1e-12
    assert np.abs(vt @ vt.conj().T - np.eye(k)).max() <= 1e-12
    rec = (u * s) @ vt
    rec_o = (ref.U * ref.S) @ ref.Vt
    assert np.abs(rec - rec_o).max() <= 1e-10 * sig[0]
