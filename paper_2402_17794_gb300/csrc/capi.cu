// C ABI of the library (include/rsvd.h): plans, workspace, the step-level
// entry points and the host-side orchestration of Algorithm 4 (Section 3.3).
//
// Everything is enqueued on the plan's stream; nothing here waits for the
// GPU except rsvd_plan_status().  The workspace is one caller-owned device
// block carved into fixed regions at plan creation; no call after
// rsvd_plan_create() allocates.
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"
#include "mixed.h"

using namespace rsvd;

namespace {

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int kPartSplits = 16;  // split-K partial slices held in workspace (plain mode)

Layout make_layout(int64_t m, int64_t n, int l, int mode) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t d = sizeof(double);
  const int64_t mn = m > n ? m : n;
  const int lpad = (l + 1) & ~1;
  L.status = take(sizeof(DeviceStatus));
  L.om = take((size_t)n * l * d);
  L.y = take((size_t)m * l * d);
  L.qm = take((size_t)m * l * d);
  L.tmp = take((size_t)mn * l * d);
  L.z = take((size_t)n * l * d);
  L.qb = take((size_t)n * l * d);
  L.part = take((size_t)kPartSplits * mn * l * d);
  L.small_stride = align_up((size_t)l * l * d);
  // G, R1, R1inv, R2, R2inv, Mt, Um, Vm, chol work, jacobi work (2 l x lpad), sig, sign
  L.small = take(L.small_stride * 9 + align_up(2 * (size_t)l * lpad * d) + align_up(2 * (size_t)l * d));
  if (mode == RSVD_MODE_MIXED) {
    MixedLayout ml = mixed_layout(m, n, l);
    L.om16 = take(ml.bytes);
  }
  L.total = off;
  return L;
}

struct Small {
  double *G, *R1, *R1i, *R2, *R2i, *Mt, *Um, *Vm, *cholw, *jw, *sig, *sign;
};

Small small_of(rsvd_plan_t P) {
  char* b = P->ws + P->lay.small;
  size_t s = P->lay.small_stride;
  Small S;
  S.G = (double*)(b + 0 * s);
  S.R1 = (double*)(b + 1 * s);
  S.R1i = (double*)(b + 2 * s);
  S.R2 = (double*)(b + 3 * s);
  S.R2i = (double*)(b + 4 * s);
  S.Mt = (double*)(b + 5 * s);
  S.Um = (double*)(b + 6 * s);
  S.Vm = (double*)(b + 7 * s);
  S.cholw = (double*)(b + 8 * s);
  S.jw = (double*)(b + 9 * s);
  const int l = P->l_max, lpad = (l + 1) & ~1;
  S.sig = (double*)(b + 9 * s + align_up(2 * (size_t)l * lpad * sizeof(double)));
  S.sign = S.sig + l;
  return S;
}

template <typename T>
T* ws_at(rsvd_plan_t P, size_t off) { return (T*)(P->ws + off); }

DeviceStatus* dstatus(rsvd_plan_t P) { return ws_at<DeviceStatus>(P, P->lay.status); }

double* part_of(rsvd_plan_t P, size_t* elems) {
  const int64_t mn = P->m_max > P->n_max ? P->m_max : P->n_max;
  *elems = (size_t)kPartSplits * mn * P->l_max;
  return ws_at<double>(P, P->lay.part);
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;   \
  } while (0)

int gemm(rsvd_plan_t P, const double* A, int64_t lda, bool trans, const double* X, int64_t ldx,
         double* C, int64_t ldc, int64_t M, int64_t K, int N) {
  GemmF64 g{A, lda, trans, X, ldx, C, ldc, M, K, N};
  size_t pe;
  double* part = part_of(P, &pe);
  CK(launch_gemm_f64(g, part, pe, P->num_sms, P->stream));
  return RSVD_OK;
}

// CholeskyQR2: Q = orth(Y) (skipped when Q is NULL); optionally
// Rprod = R2 R1 or its transpose (ld l), the R factor of Y = Q R.
int orth_f64(rsvd_plan_t P, const double* Y, int64_t rows, int l, int64_t ldy, double* Q,
             int64_t ldq, double* T, double* Rprod, bool transpose_R) {
  Small S = small_of(P);
  int rc;
  DeviceStatus* st = dstatus(P);
  // pass 1
  if ((rc = gemm(P, Y, ldy, true, Y, ldy, S.G, l, l, rows, l))) return rc;
  CK(launch_chol_inv(S.G, l, l, S.R1, S.R1i, S.cholw, st, P->stream));
  if ((rc = gemm(P, Y, ldy, false, S.R1i, l, T, rows, rows, l, l))) return rc;
  // pass 2
  if ((rc = gemm(P, T, rows, true, T, rows, S.G, l, l, rows, l))) return rc;
  CK(launch_chol_inv(S.G, l, l, S.R2, S.R2i, S.cholw, st, P->stream));
  if (Q && (rc = gemm(P, T, rows, false, S.R2i, l, Q, ldq, rows, l, l))) return rc;
  if (Rprod) CK(launch_tri_product(S.R2, S.R1, l, Rprod, transpose_R, P->stream));
  return RSVD_OK;
}

int solve_plain(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                int q, uint64_t seed, double* U, int64_t ldu, double* Sout, double* VT,
                int64_t ldvt) {
  const int l = k + p;
  double* om = ws_at<double>(P, P->lay.om);
  double* y = ws_at<double>(P, P->lay.y);
  double* qm = ws_at<double>(P, P->lay.qm);
  double* tmp = ws_at<double>(P, P->lay.tmp);
  double* z = ws_at<double>(P, P->lay.z);
  double* qb = ws_at<double>(P, P->lay.qb);
  Small S = small_of(P);
  int rc;
  // 1. Omega;  2. Y = A Omega;  3. Q = orth(Y)
  CK(launch_gaussian(n, l, seed, 0u, RSVD_F64, om, n, P->stream));
  if ((rc = gemm(P, A, lda, false, om, n, y, m, m, n, l))) return rc;
  if ((rc = orth_f64(P, y, m, l, m, qm, m, tmp, nullptr, false))) return rc;
  // 4-5. power steps with orthonormalisation
  for (int j = 0; j < q; ++j) {
    if ((rc = gemm(P, A, lda, true, qm, m, z, n, n, m, l))) return rc;
    if ((rc = orth_f64(P, z, n, l, n, om, n, tmp, nullptr, false))) return rc;
    if ((rc = gemm(P, A, lda, false, om, n, y, m, m, n, l))) return rc;
    if ((rc = orth_f64(P, y, m, l, m, qm, m, tmp, nullptr, false))) return rc;
  }
  // 6. B^T = A^T Q.  7. B^T = Q_B R_B by CholeskyQR2 (only R_B is formed);
  // one-sided Jacobi on R_B^T = U~ Sigma V_R^T gives sigma and U~ (the left
  // singular vectors of B); the right ones follow as V = B^T U~ Sigma^-1.
  if ((rc = gemm(P, A, lda, true, qm, m, z, n, n, m, l))) return rc;
  if ((rc = orth_f64(P, z, n, l, n, nullptr, n, tmp, S.Mt, true))) return rc;
  double* us_inv = S.Vm;
  CK(launch_jacobi_svd(S.Mt, l, l, S.sig, S.Um, l, nullptr, l, us_inv, S.jw, dstatus(P),
                       P->stream));
  // 8. U = Q U~ (first k columns), V_k = B^T U~_k Sigma_k^-1
  if ((rc = gemm(P, qm, m, false, S.Um, l, U, ldu, m, l, k))) return rc;
  if ((rc = gemm(P, z, n, false, us_inv, l, tmp, n, n, l, k))) return rc;
  // One CholeskyQR pass restores orthonormality of V_k to rounding (the
  // product above carries relative errors ~ eps sigma_1/sigma_i); the
  // triangular factor is I + O(eps sigma_1/sigma_k).
  if ((rc = gemm(P, tmp, n, true, tmp, n, S.G, k, k, n, k))) return rc;
  CK(launch_chol_inv(S.G, k, k, S.R1, S.R1i, S.cholw, dstatus(P), P->stream));
  if ((rc = gemm(P, tmp, n, false, S.R1i, k, qb, n, n, k, k))) return rc;
  CK(launch_finalize_f64(U, m, ldu, k, qb, n, VT, ldvt, S.sig, Sout, S.sign, P->stream));
  return RSVD_OK;
}

bool ready(rsvd_plan_t P) { return P && P->ws && P->ws_bytes >= P->lay.total; }

}  // namespace

extern "C" {

int rsvd_plan_create(rsvd_plan_t* plan, int64_t m_max, int64_t n_max, int l_max, int a_dtype,
                     int mode, void* cuda_stream) {
  if (!plan) return -1;
  *plan = nullptr;
  if (m_max < 1) return -2;
  if (n_max < 1) return -3;
  if (l_max < 1 || l_max > RSVD_L_MAX) return -4;
  if (a_dtype != RSVD_F64 && a_dtype != RSVD_BF16) return -5;
  if (mode != RSVD_MODE_PLAIN && mode != RSVD_MODE_MIXED) return -6;
  if ((mode == RSVD_MODE_PLAIN) != (a_dtype == RSVD_F64)) return -6;
  rsvd_plan_s* P = new (std::nothrow) rsvd_plan_s();
  if (!P) return RSVD_ERR_CUDA;
  P->m_max = m_max;
  P->n_max = n_max;
  P->l_max = l_max;
  P->dtype = a_dtype;
  P->mode = mode;
  P->stream = (cudaStream_t)cuda_stream;
  P->ws = nullptr;
  P->ws_bytes = 0;
  P->lay = make_layout(m_max, n_max, l_max, mode);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost((void**)&P->h_status, sizeof(int) * 4) != cudaSuccess) {
    delete P;
    return RSVD_ERR_CUDA;
  }
  std::memset(P->h_status, 0, sizeof(int) * 4);
  *plan = P;
  return RSVD_OK;
}

int rsvd_workspace_size(rsvd_plan_t plan, size_t* bytes) {
  if (!plan) return -1;
  if (!bytes) return -2;
  *bytes = plan->lay.total;
  return RSVD_OK;
}

int rsvd_set_workspace(rsvd_plan_t plan, void* dev_ptr, size_t bytes) {
  if (!plan) return -1;
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign)) return -2;
  if (bytes < plan->lay.total) return RSVD_ERR_WORKSPACE;
  plan->ws = (char*)dev_ptr;
  plan->ws_bytes = bytes;
  if (cudaMemsetAsync(plan->ws + plan->lay.status, 0, sizeof(DeviceStatus), plan->stream) !=
      cudaSuccess)
    return RSVD_ERR_CUDA;
  return RSVD_OK;
}

int rsvd_plan_set_stream(rsvd_plan_t plan, void* cuda_stream) {
  if (!plan) return -1;
  plan->stream = (cudaStream_t)cuda_stream;
  return RSVD_OK;
}

int rsvd_plan_status(rsvd_plan_t plan) {
  if (!plan) return -1;
  if (!plan->ws) return RSVD_ERR_WORKSPACE;
  DeviceStatus* d = dstatus(plan);
  if (cudaMemcpyAsync(plan->h_status, &d->flags, sizeof(int), cudaMemcpyDeviceToHost,
                      plan->stream) != cudaSuccess)
    return RSVD_ERR_CUDA;
  if (cudaStreamSynchronize(plan->stream) != cudaSuccess) return RSVD_ERR_CUDA;
  int flags = plan->h_status[0];
  if (cudaMemsetAsync(&d->flags, 0, sizeof(int), plan->stream) != cudaSuccess) return RSVD_ERR_CUDA;
  return status_from_flags(flags);
}

int rsvd_plan_diagnostics(rsvd_plan_t plan, int* jacobi_sweeps, int* dropped_columns) {
  if (!plan) return -1;
  if (!plan->ws) return RSVD_ERR_WORKSPACE;
  DeviceStatus* d = dstatus(plan);
  if (cudaMemcpyAsync(plan->h_status, &d->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                      plan->stream) != cudaSuccess)
    return RSVD_ERR_CUDA;
  if (cudaStreamSynchronize(plan->stream) != cudaSuccess) return RSVD_ERR_CUDA;
  if (jacobi_sweeps) *jacobi_sweeps = plan->h_status[1];
  if (dropped_columns) *dropped_columns = plan->h_status[2];
  return RSVD_OK;
}

int rsvd_plan_destroy(rsvd_plan_t plan) {
  if (!plan) return -1;
  if (plan->h_status) cudaFreeHost(plan->h_status);
  delete plan;
  return RSVD_OK;
}

const char* rsvd_status_string(int status) {
  switch (status) {
    case RSVD_OK: return "ok";
    case RSVD_ERR_CHOLESKY: return "Gram Cholesky broke down";
    case RSVD_ERR_JACOBI: return "Jacobi SVD did not converge";
    case RSVD_ERR_TIMEOUT: return "device wait exceeded its iteration limit";
    case RSVD_ERR_WORKSPACE: return "workspace missing or too small for this problem";
    case RSVD_ERR_CUDA: return "CUDA error";
    case RSVD_ERR_NONFINITE: return "non-finite value in the input";
    case RSVD_ERR_UNSUPPORTED: return "unsupported dtype, mode or size";
    default: break;
  }
  if (status < 0) return "invalid argument";
  return "unknown status";
}

int rsvd_solve(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int k, int p,
               int q, uint64_t seed, void* U, int64_t ldu, double* S, void* VT, int64_t ldvt) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (k < 1) return -6;
  if (p < 0) return -7;
  if (q < 0) return -8;
  if (!U) return -10;
  if (ldu < m) return -11;
  if (!S) return -12;
  if (!VT) return -13;
  if (ldvt < k) return -14;
  const int l = k + p;
  if (l > (m < n ? m : n)) return -7;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode == RSVD_MODE_PLAIN)
    return solve_plain(plan, (const double*)A, m, n, lda, k, p, q, seed, (double*)U, ldu, S,
                       (double*)VT, ldvt);
  MixedArgs ma{A, m, n, lda, k, p, q, seed, U, ldu, S, VT, ldvt};
  return solve_mixed(plan, ma);
}

int rsvd_gaussian(rsvd_plan_t plan, int64_t n, int l, uint64_t seed, uint32_t stream, int out_dtype,
                  void* out, int64_t ldo) {
  if (!plan) return -1;
  if (n < 1) return -2;
  if (l < 1) return -3;
  if (out_dtype != RSVD_F64 && out_dtype != RSVD_BF16) return -6;
  if (!out) return -7;
  if (ldo < n) return -8;
  CK(launch_gaussian(n, l, seed, stream, out_dtype, out, ldo, plan->stream));
  return RSVD_OK;
}

int rsvd_apply_a(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, const void* X,
                 int64_t ldx, int l, void* Y, int64_t ldy) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (!X) return -6;
  if (ldx < n) return -7;
  if (l < 1) return -8;
  if (!Y) return -9;
  if (ldy < m) return -10;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode == RSVD_MODE_PLAIN)
    return gemm(plan, (const double*)A, lda, false, (const double*)X, ldx, (double*)Y, ldy, m, n, l);
  return mixed_apply(plan, A, m, n, lda, X, ldx, l, Y, ldy, false);
}

int rsvd_apply_at(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                  const void* X, int64_t ldx, int l, void* Z, int64_t ldz) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (!X) return -6;
  if (ldx < m) return -7;
  if (l < 1) return -8;
  if (!Z) return -9;
  if (ldz < n) return -10;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode == RSVD_MODE_PLAIN)
    return gemm(plan, (const double*)A, lda, true, (const double*)X, ldx, (double*)Z, ldz, n, m, l);
  return mixed_apply(plan, A, m, n, lda, X, ldx, l, Z, ldz, true);
}

int rsvd_orth(rsvd_plan_t plan, const double* Y, int64_t rows, int l, int64_t ldy, double* Q,
              int64_t ldq, double* R, int64_t ldr) {
  if (!plan) return -1;
  if (!Y) return -2;
  if (rows < 1) return -3;
  if (l < 1 || l > rows) return -4;
  if (ldy < rows) return -5;
  if (!Q) return -6;
  if (ldq < rows) return -7;
  if (R && ldr < l) return -9;
  const int64_t mn = plan->m_max > plan->n_max ? plan->m_max : plan->n_max;
  if (!ready(plan) || rows > mn || l > plan->l_max) return RSVD_ERR_WORKSPACE;
  Small S = small_of(plan);
  double* tmp = ws_at<double>(plan, plan->lay.tmp);
  int rc = orth_f64(plan, Y, rows, l, ldy, Q, ldq, tmp, R ? S.Mt : nullptr, false);
  if (rc) return rc;
  if (R)
    CK(cudaMemcpy2DAsync(R, ldr * sizeof(double), S.Mt, l * sizeof(double), l * sizeof(double), l,
                         cudaMemcpyDeviceToDevice, plan->stream));
  return RSVD_OK;
}

int rsvd_small_svd(rsvd_plan_t plan, const double* M, int l, int64_t ldm, double* sig, double* Um,
                   int64_t ldu, double* Vm, int64_t ldv) {
  if (!plan) return -1;
  if (!M) return -2;
  if (l < 1 || l > plan->l_max) return -3;
  if (ldm < l) return -4;
  if (!sig) return -5;
  if (!Um) return -6;
  if (ldu < l) return -7;
  if (!Vm) return -8;
  if (ldv < l) return -9;
  if (!ready(plan)) return RSVD_ERR_WORKSPACE;
  Small S = small_of(plan);
  CK(launch_jacobi_svd(M, l, ldm, sig, Um, ldu, Vm, ldv, nullptr, S.jw, dstatus(plan),
                       plan->stream));
  return RSVD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch accounting
// ---------------------------------------------------------------------------
#include <atomic>

namespace {
std::atomic<uint64_t> g_launches{0};
}

void rsvd::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" uint64_t rsvd_kernel_launches(void) {
  return g_launches.load(std::memory_order_relaxed);
}
