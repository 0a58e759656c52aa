"""Python binding of the C ABI (include/rsvd.h), torch tensors as buffers.

The functions carry the C names and only marshal arguments: every step of
the randomized SVD runs in the library's CUDA kernels.  Torch supplies device
memory and the stream.

Layout: a column-major r x c matrix with leading dimension ld is held in a
torch tensor of shape (c, ld) (row j of the tensor is column j of the
matrix); :func:`colmajor` allocates one, :func:`from_numpy_f` converts a
Fortran-ordered numpy array.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

F64, F32, BF16, FP8E4M3 = 0, 1, 2, 3
ERR_NOT_REACHED = 8
PLAIN, MIXED, F64_TENSOR = 0, 1, 2
STATUS = {0: "ok", 1: "cholesky", 2: "jacobi", 3: "timeout", 4: "workspace", 5: "cuda",
          6: "nonfinite", 7: "unsupported"}


class RsvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.load().rsvd_status_string(code).decode()
        super().__init__(f"{where}: status {code} ({msg})")
        self.code = code


def _check(code: int, where: str) -> int:
    if code != 0:
        raise RsvdError(code, where)
    return code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def colmajor(rows: int, cols: int, dtype=torch.float64, ld: int | None = None,
             device="cuda", zero: bool = False):
    ld = ld or rows
    f = torch.zeros if zero else torch.empty
    return f(cols, ld, dtype=dtype, device=device)


def from_numpy_f(a: np.ndarray, device="cuda", dtype=None):
    """Column-major torch copy of a 2-D numpy array (any order)."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def to_numpy_f(t, rows: int | None = None) -> np.ndarray:
    """numpy (rows x cols) Fortran array from a column-major tensor (cols, ld)."""
    a = t.detach().to("cpu", dtype=torch.float64).numpy().T
    if rows is not None:
        a = a[:rows]
    return np.asfortranarray(a)


# ---------------------------------------------------------------------------
# C entry points (same names)
# ---------------------------------------------------------------------------

def rsvd_plan_create(m_max, n_max, l_max, a_dtype=F64, mode=PLAIN, stream=None):
    lib = _lib.load()
    h = ctypes.c_void_p()
    _check(lib.rsvd_plan_create(ctypes.byref(h), m_max, n_max, l_max, a_dtype, mode,
                                _stream_handle(stream)), "rsvd_plan_create")
    return h


def rsvd_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check(_lib.load().rsvd_workspace_size(plan, ctypes.byref(n)), "rsvd_workspace_size")
    return n.value


def rsvd_set_workspace(plan, buf) -> None:
    _check(_lib.load().rsvd_set_workspace(plan, _ptr(buf), buf.numel() * buf.element_size()),
           "rsvd_set_workspace")


def rsvd_plan_status(plan) -> int:
    return _lib.load().rsvd_plan_status(plan)


def rsvd_plan_diagnostics(plan):
    """(jacobi_sweeps, dropped_columns) of the work enqueued so far."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(_lib.load().rsvd_plan_diagnostics(plan, ctypes.byref(a), ctypes.byref(b)),
           "rsvd_plan_diagnostics")
    return a.value, b.value


def rsvd_plan_set_stream(plan, stream=None) -> None:
    _check(_lib.load().rsvd_plan_set_stream(plan, _stream_handle(stream)), "rsvd_plan_set_stream")


def rsvd_plan_set_wait_limit(plan, cycles) -> int:
    return _lib.load().rsvd_plan_set_wait_limit(plan, int(cycles))


def rsvd_plan_prepare_a(plan, A, m, n, lda) -> int:
    return _lib.load().rsvd_plan_prepare_a(plan, _ptr(A), m, n, lda)


def rsvd_plan_release_a(plan) -> int:
    return _lib.load().rsvd_plan_release_a(plan)


def rsvd_set_tile_scales(plan, scales, rows, cols, lds) -> int:
    return _lib.load().rsvd_set_tile_scales(plan, _ptr(scales), rows, cols, lds)


def rsvd_plan_destroy(plan) -> None:
    _lib.load().rsvd_plan_destroy(plan)


def rsvd_status_string(code: int) -> str:
    return _lib.load().rsvd_status_string(code).decode()


def rsvd_kernel_launches() -> int:
    return int(_lib.load().rsvd_kernel_launches())


def rsvd_solve(plan, A, m, n, lda, k, p, q, seed, U, ldu, S, VT, ldvt) -> int:
    return _lib.load().rsvd_solve(plan, _ptr(A), m, n, lda, k, p, q, seed, _ptr(U), ldu, _ptr(S),
                                  _ptr(VT), ldvt)


def rsvd_solve_algorithm(plan, algorithm, A, m, n, lda, k, p, q, seed, U, ldu, S, VT,
                         ldvt) -> int:
    return _lib.load().rsvd_solve_algorithm(plan, algorithm, _ptr(A), m, n, lda, k, p, q, seed,
                                            _ptr(U), ldu, _ptr(S), _ptr(VT), ldvt)


def rsvd_range_adaptive(plan, A, m, n, lda, eps, r, l_cap, seed, Q, ldq):
    """(code, rank); waits on the plan's stream once per block of samples."""
    rank = ctypes.c_int(0)
    code = _lib.load().rsvd_range_adaptive(plan, _ptr(A), m, n, lda, float(eps), r, l_cap, seed,
                                           _ptr(Q), ldq, ctypes.byref(rank))
    return code, rank.value


def rsvd_solve_adaptive(plan, A, m, n, lda, eps, r, l_cap, seed, U, ldu, S, VT, ldvt):
    """(code, rank); waits on the plan's stream once per block of samples."""
    rank = ctypes.c_int(0)
    code = _lib.load().rsvd_solve_adaptive(plan, _ptr(A), m, n, lda, float(eps), r, l_cap, seed,
                                           _ptr(U), ldu, _ptr(S), _ptr(VT), ldvt,
                                           ctypes.byref(rank))
    return code, rank.value


def rsvd_range_srft(plan, A, m, n, lda, l, seed, Q, ldq) -> int:
    return _lib.load().rsvd_range_srft(plan, _ptr(A), m, n, lda, l, seed, _ptr(Q), ldq)


def rsvd_solve_srft(plan, A, m, n, lda, k, p, seed, U, ldu, S, VT, ldvt) -> int:
    return _lib.load().rsvd_solve_srft(plan, _ptr(A), m, n, lda, k, p, seed, _ptr(U), ldu,
                                       _ptr(S), _ptr(VT), ldvt)


def rsvd_srft_sketch(plan, A, m, n, lda, l, seed, Y, ldy) -> int:
    return _lib.load().rsvd_srft_sketch(plan, _ptr(A), m, n, lda, l, seed, _ptr(Y), ldy)


def rsvd_solve_singlepass(plan, A, m, n, lda, k, p, seed, U, ldu, S, VT, ldvt) -> int:
    return _lib.load().rsvd_solve_singlepass(plan, _ptr(A), m, n, lda, k, p, seed, _ptr(U), ldu,
                                             _ptr(S), _ptr(VT), ldvt)


def rsvd_solve_hermitian(plan, A, n, lda, k, p, seed, U, ldu, D) -> int:
    return _lib.load().rsvd_solve_hermitian(plan, _ptr(A), n, lda, k, p, seed, _ptr(U), ldu,
                                            _ptr(D))


def rsvd_gaussian(plan, n, l, seed, stream_id, out_dtype, out, ldo) -> int:
    return _lib.load().rsvd_gaussian(plan, n, l, seed, stream_id, out_dtype, _ptr(out), ldo)


def rsvd_apply_a(plan, A, m, n, lda, X, ldx, l, Y, ldy) -> int:
    return _lib.load().rsvd_apply_a(plan, _ptr(A), m, n, lda, _ptr(X), ldx, l, _ptr(Y), ldy)


def rsvd_apply_at(plan, A, m, n, lda, X, ldx, l, Z, ldz) -> int:
    return _lib.load().rsvd_apply_at(plan, _ptr(A), m, n, lda, _ptr(X), ldx, l, _ptr(Z), ldz)


def rsvd_apply_split(plan, A, m, n, lda, trans, X, ldx, l, slices, out, ldo) -> int:
    return _lib.load().rsvd_apply_split(plan, _ptr(A), m, n, lda, trans, _ptr(X), ldx, l, slices,
                                        _ptr(out), ldo)


def rsvd_orth(plan, Y, rows, l, ldy, Q, ldq, R=None, ldr=0) -> int:
    return _lib.load().rsvd_orth(plan, _ptr(Y), rows, l, ldy, _ptr(Q), ldq, _ptr(R), ldr)


def rsvd_small_svd(plan, M, l, ldm, sig, Um, ldu, Vm, ldv) -> int:
    return _lib.load().rsvd_small_svd(plan, _ptr(M), l, ldm, _ptr(sig), _ptr(Um), ldu, _ptr(Vm),
                                      ldv)


def rsvd_batch_plan_create(max_count, rows_total, cols_total, l_max, a_dtype=F64, stream=None):
    lib = _lib.load()
    h = ctypes.c_void_p()
    _check(lib.rsvd_batch_plan_create(ctypes.byref(h), max_count, rows_total, cols_total, l_max,
                                      a_dtype, _stream_handle(stream)), "rsvd_batch_plan_create")
    return h


def rsvd_solve_batched(plan, problems) -> int:
    """problems: a sequence of _lib.RsvdProblem (or an already built array)."""
    arr = problems if isinstance(problems, ctypes.Array) else (_lib.RsvdProblem * len(problems))(*problems)
    return _lib.load().rsvd_solve_batched(plan, len(arr), arr)


def rsvd_batch_status(plan, count):
    codes = (ctypes.c_int * count)()
    _check(_lib.load().rsvd_batch_status(plan, count, codes), "rsvd_batch_status")
    return list(codes)


BATCH_ENGINE_SIMT, BATCH_ENGINE_TENSOR = 0, 1


def rsvd_batch_set_engine(plan, engine) -> int:
    return _lib.load().rsvd_batch_set_engine(plan, engine)


def rsvd_batch_set_graphs(plan, on) -> int:
    return _lib.load().rsvd_batch_set_graphs(plan, int(on))


def rsvd_batch_set_sm_limit(plan, sms) -> int:
    return _lib.load().rsvd_batch_set_sm_limit(plan, int(sms))


def rsvd_batch_autotune(plan, problems) -> int:
    arr = problems if isinstance(problems, ctypes.Array) else (_lib.RsvdProblem * len(problems))(*problems)
    return _lib.load().rsvd_batch_autotune(plan, len(arr), arr)


def rsvd_grouped_gemm_f32(plan, gemms, trans) -> int:
    """gemms: a sequence of _lib.RsvdGemm (or an already built array)."""
    arr = gemms if isinstance(gemms, ctypes.Array) else (_lib.RsvdGemm * len(gemms))(*gemms)
    return _lib.load().rsvd_grouped_gemm_f32(plan, len(arr), arr, int(trans))


def rsvd_grouped_schedule(shapes, trans, num_sms):
    """The tensor engine's work schedule for product shapes [(M, K, N)]:
    (units as a list of (product, row0, col0, kb0, kb1, slot, t), cta_off,
    info (units, grid, slots, largest t)).  Host computation only."""
    lib = _lib.load()
    flat = (ctypes.c_int64 * (3 * len(shapes)))(*[v for s in shapes for v in s])
    info = (ctypes.c_int * 4)()
    _check(lib.rsvd_grouped_schedule(len(shapes), flat, int(trans), num_sms, None, 0, None, info),
           "rsvd_grouped_schedule")
    units = (ctypes.c_int * (7 * max(1, info[0])))()
    cta = (ctypes.c_int * (num_sms + 1))()
    _check(lib.rsvd_grouped_schedule(len(shapes), flat, int(trans), num_sms, units, info[0], cta,
                                     info), "rsvd_grouped_schedule")
    u = [tuple(units[7 * i: 7 * i + 7]) for i in range(info[0])]
    return u, list(cta)[: info[1] + 1], tuple(info)


def rsvd_apply_a_f64_static(A, m, n, lda, X, ldx, l, Y, ldy, stream=None) -> int:
    return _lib.load().rsvd_apply_a_f64_static(_ptr(A), m, n, lda, _ptr(X), ldx, l, _ptr(Y), ldy,
                                               _stream_handle(stream))


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class BatchPlan:
    """Owns a batch plan (rsvd_batch_plan_create) and its workspace.

    solve(items) takes a list of (A, m, n, k, p, q, seed) with A a
    column-major device tensor (n, lda) of the plan's dtype and returns
    [(U, S, VT)] column-major tensors; enqueued only (status() waits)."""

    def __init__(self, max_count, rows_total, cols_total, l_max, a_dtype=F64, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the randomized SVD library needs a CUDA GPU")
        self.handle = rsvd_batch_plan_create(max_count, rows_total, cols_total, l_max, a_dtype,
                                             stream)
        self.dtype = torch.float64 if a_dtype == F64 else torch.float32
        nbytes = rsvd_workspace_size(self.handle)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        rsvd_set_workspace(self.handle, self.workspace)
        self.count = 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            try:
                rsvd_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def _problems(self, items, outs):
        probs, results = [], []
        for i, (A, m, n, k, p, q, seed) in enumerate(items):
            if outs is None:
                U = torch.empty(k, m, dtype=self.dtype, device=A.device)
                S = torch.empty(k, dtype=torch.float64, device=A.device)
                VT = torch.empty(n, k, dtype=self.dtype, device=A.device)
            else:
                U, S, VT = outs[i]
            probs.append(_lib.RsvdProblem(A.data_ptr(), m, n, A.shape[1], k, p, q, seed,
                                          U.data_ptr(), U.shape[1], S.data_ptr(), VT.data_ptr(),
                                          VT.shape[1]))
            results.append((U, S, VT))
        return probs, results

    def solve(self, items, outs=None):
        probs, results = self._problems(items, outs)
        _check(rsvd_solve_batched(self.handle, probs), "rsvd_solve_batched")
        self.count = len(probs)
        self._keep = (items, results)
        return results

    def set_engine(self, engine):
        _check(rsvd_batch_set_engine(self.handle, engine), "rsvd_batch_set_engine")

    def set_sm_limit(self, sms):
        """SMs of the tensor engine's persistent launches (0: all)."""
        _check(rsvd_batch_set_sm_limit(self.handle, sms), "rsvd_batch_set_sm_limit")

    def set_graphs(self, on=True):
        """Grouped FP32 solves as CUDA graphs (needs a non-default stream)."""
        _check(rsvd_batch_set_graphs(self.handle, on), "rsvd_batch_set_graphs")

    def autotune(self, items, outs=None):
        """Tunes the tensor engine's schedules on these problems (FP32 plans)."""
        probs, results = self._problems(items, outs)
        _check(rsvd_batch_autotune(self.handle, probs), "rsvd_batch_autotune")

    def grouped_gemm(self, gemms, trans):
        """gemms: list of (A, lda, X, ldx, C, ldc, M, K, N, x_upper) with
        device FP32 tensors; C = op(A) X on the tensor engine."""
        arr = (_lib.RsvdGemm * len(gemms))(*[
            _lib.RsvdGemm(_ptr(A), lda, _ptr(X), ldx, _ptr(C), ldc, M, K, N, int(xu))
            for (A, lda, X, ldx, C, ldc, M, K, N, xu) in gemms])
        self._keep_gemm = gemms
        _check(rsvd_grouped_gemm_f32(self.handle, arr, trans), "rsvd_grouped_gemm_f32")

    def status(self):
        return rsvd_batch_status(self.handle, self.count)


class Plan:
    """Owns a C plan and its torch-allocated workspace."""

    def __init__(self, m_max, n_max, l_max, a_dtype=F64, mode=PLAIN, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the randomized SVD library needs a CUDA GPU")
        self.stream = stream
        self.handle = rsvd_plan_create(m_max, n_max, l_max, a_dtype, mode, stream)
        self.mode = mode
        nbytes = rsvd_workspace_size(self.handle)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        rsvd_set_workspace(self.handle, self.workspace)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            try:
                rsvd_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def status(self) -> int:
        return rsvd_plan_status(self.handle)

    def set_tile_scales(self, scales):
        """FP8 plans: scales is the FP32 device tensor (n_tiles, m_tiles) whose
        row J holds column J of the column-major scale matrix."""
        self.scales = scales   # the plan reads it on every later call
        _check(rsvd_set_tile_scales(self.handle, scales, scales.shape[1], scales.shape[0],
                                    scales.shape[1]), "rsvd_set_tile_scales")

    def solve_algorithm(self, algorithm, A, m, n, k, p, q, seed, lda=None):
        """Algorithm 2, 3, 4 or 6 of the thesis: (U, S, VT) as solve(); enqueued only."""
        lda = lda or A.shape[1]
        odt = torch.float64 if self.mode != MIXED else torch.float32
        U = torch.empty(k, m, dtype=odt, device=A.device)
        S = torch.empty(k, dtype=torch.float64, device=A.device)
        VT = torch.empty(n, k, dtype=odt, device=A.device)
        _check(rsvd_solve_algorithm(self.handle, algorithm, A, m, n, lda, k, p, q, seed, U, m, S,
                                    VT, k), "rsvd_solve_algorithm")
        return U, S, VT

    def solve_singlepass(self, A, m, n, k, p, seed, lda=None):
        """Algorithm 6 on a plain plan: (U, S, VT) as solve(); enqueued only."""
        lda = lda or A.shape[1]
        U = torch.empty(k, m, dtype=torch.float64, device=A.device)
        S = torch.empty(k, dtype=torch.float64, device=A.device)
        VT = torch.empty(n, k, dtype=torch.float64, device=A.device)
        _check(rsvd_solve_singlepass(self.handle, A, m, n, lda, k, p, seed, U, m, S, VT, k),
               "rsvd_solve_singlepass")
        return U, S, VT

    def solve_hermitian(self, A, n, k, p, seed, lda=None):
        """Algorithm 5 on a plain plan (A symmetric n x n): (U, D) with U
        (k, n) holding the column-major n x k eigenvectors and D the k
        eigenvalues by decreasing magnitude; enqueued only."""
        lda = lda or A.shape[1]
        U = torch.empty(k, n, dtype=torch.float64, device=A.device)
        D = torch.empty(k, dtype=torch.float64, device=A.device)
        _check(rsvd_solve_hermitian(self.handle, A, n, lda, k, p, seed, U, n, D),
               "rsvd_solve_hermitian")
        return U, D

    def range_adaptive(self, A, m, n, eps, r, l_cap, seed, lda=None):
        """Adaptive range finder on a plain plan: (Q (rank, m) column-major,
        converged).  Waits on the plan's stream once per block of samples."""
        lda = lda or A.shape[1]
        Q = torch.empty(l_cap, m, dtype=torch.float64, device=A.device)
        code, rank = rsvd_range_adaptive(self.handle, A, m, n, lda, eps, r, l_cap, seed, Q, m)
        if code not in (0, ERR_NOT_REACHED):
            _check(code, "rsvd_range_adaptive")
        return Q[:rank], code == 0

    def solve_adaptive(self, A, m, n, eps, r, l_cap, seed, lda=None):
        """Adaptive range finder + small SVD: (U (rank, m), S (rank,),
        VT (n, l_cap)[:, :rank] view, converged); the rank is S.numel()."""
        lda = lda or A.shape[1]
        U = torch.empty(l_cap, m, dtype=torch.float64, device=A.device)
        S = torch.empty(l_cap, dtype=torch.float64, device=A.device)
        VT = torch.empty(n, l_cap, dtype=torch.float64, device=A.device)
        code, rank = rsvd_solve_adaptive(self.handle, A, m, n, lda, eps, r, l_cap, seed, U, m, S,
                                         VT, l_cap)
        if code not in (0, ERR_NOT_REACHED):
            _check(code, "rsvd_solve_adaptive")
        return U[:rank], S[:rank], VT[:, :rank], code == 0

    def range_srft(self, A, m, n, l, seed, lda=None):
        """FastRandRF with the SRFT on a plain plan (l_max >= 2l): Q as a
        column-major planar tensor (2l, m): rows 0..l-1 Re Q, l..2l-1 Im Q.
        Enqueued only."""
        lda = lda or A.shape[1]
        Q = torch.empty(2 * l, m, dtype=torch.float64, device=A.device)
        _check(rsvd_range_srft(self.handle, A, m, n, lda, l, seed, Q, m), "rsvd_range_srft")
        return Q

    def solve_srft(self, A, m, n, k, p, seed, lda=None):
        """FastRandRF + the rank-k SVD on its complex basis (plain plan with
        l_max >= 2(k+p)): U as a planar tensor (2k, m) (rows 0..k-1 Re U),
        S (k,), VT as a planar tensor (2n, k) (rows 0..n-1 Re V^H).
        Enqueued only."""
        lda = lda or A.shape[1]
        U = torch.empty(2 * k, m, dtype=torch.float64, device=A.device)
        S = torch.empty(k, dtype=torch.float64, device=A.device)
        VT = torch.empty(2 * n, k, dtype=torch.float64, device=A.device)
        _check(rsvd_solve_srft(self.handle, A, m, n, lda, k, p, seed, U, m, S, VT, k),
               "rsvd_solve_srft")
        return U, S, VT

    def srft_sketch(self, A, m, n, l, seed, lda=None):
        """Y = A Omega with the SRFT Omega, planar (2l, m).  Enqueued only."""
        lda = lda or A.shape[1]
        Y = torch.empty(2 * l, m, dtype=torch.float64, device=A.device)
        _check(rsvd_srft_sketch(self.handle, A, m, n, lda, l, seed, Y, m), "rsvd_srft_sketch")
        return Y

    def solve(self, A, m, n, k, p, q, seed, lda=None, out=None):
        """A: column-major device tensor (n, lda).  Returns (U, S, VT) as
        column-major tensors U (k, m), S (k,), VT (n, k); enqueued only."""
        lda = lda or A.shape[1]
        odt = torch.float64 if self.mode != MIXED else torch.float32
        if out is None:
            U = torch.empty(k, m, dtype=odt, device=A.device)
            S = torch.empty(k, dtype=torch.float64, device=A.device)
            VT = torch.empty(n, k, dtype=odt, device=A.device)
        else:
            U, S, VT = out
        _check(rsvd_solve(self.handle, A, m, n, lda, k, p, q, seed, U, U.shape[1], S, VT,
                          VT.shape[1]), "rsvd_solve")
        return U, S, VT
