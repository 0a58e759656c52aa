// C ABI of the library (include/rsvd.h): plans, workspace, the step-level
// entry points and the host-side orchestration of Algorithm 4 (Section 3.3).
//
// Everything is enqueued on the plan's stream; nothing here waits for the
// GPU except rsvd_plan_status().  The workspace is one caller-owned device
// block carved into fixed regions at plan creation; no call after
// rsvd_plan_create() allocates.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "batched.h"
#include "grouped_tc.h"
#include "pipeline.h"
#include "umma.h"

using namespace rsvd;

namespace {

#define CK RSVD_CK

bool ready(rsvd_plan_t P) { return plan_ready(P); }

// FP8 A: scales set and covering m x n, rows 16-byte aligned for TMA.
bool fp8_ready(rsvd_plan_t P, int64_t m, int64_t n, int64_t lda) {
  return P->scales && (m + 127) / 128 <= P->scale_rows && (n + 127) / 128 <= P->scale_cols &&
         lda % 16 == 0;
}

// x > 0, finite, and a power of two (no mantissa bits).
bool power_of_two(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  const uint32_t e = (b >> 23) & 0xFF, mant = b & 0x7FFFFF;
  return (b >> 31) == 0 && e != 0 && e != 0xFF && mant == 0;
}

// RSVD_MODE_F64_TENSOR plans: A's digit slices are built at the start of a
// call that reads A, and its passes run on the tensor cores until the call
// returns.  Plain plans: nothing.
// A matrix prepared by rsvd_plan_prepare_a is reused as long as the call
// names the same (A, m, n, lda).
struct TcScope {
  rsvd_plan_t P;
  int rc = RSVD_OK;
  bool keep = false;
  TcScope(rsvd_plan_t p, const void* A, int64_t m, int64_t n, int64_t lda) : P(p) {
    if (!P->f64tc) return;
    if (P->tc_pinned && P->tc_A == A && P->tc_m == m && P->tc_n == n && P->tc_lda == lda) {
      keep = true;
      return;
    }
    P->tc_pinned = 0;   // another matrix: its slices replace the prepared ones
    rc = f64tc_begin(P, (const double*)A, m, n, lda);
  }
  ~TcScope() {
    if (P->f64tc && !keep) f64tc_end(P);
  }
};

}  // namespace

extern "C" {

int rsvd_plan_create(rsvd_plan_t* plan, int64_t m_max, int64_t n_max, int l_max, int a_dtype,
                     int mode, void* cuda_stream) {
  if (!plan) return -1;
  *plan = nullptr;
  if (m_max < 1) return -2;
  if (n_max < 1) return -3;
  if (l_max < 1 || l_max > RSVD_L_MAX) return -4;
  if (a_dtype != RSVD_F64 && a_dtype != RSVD_BF16 && a_dtype != RSVD_FP8E4M3) return -5;
  if (mode != RSVD_MODE_PLAIN && mode != RSVD_MODE_MIXED && mode != RSVD_MODE_F64_TENSOR)
    return -6;
  const bool f64tc = mode == RSVD_MODE_F64_TENSOR;
  if (f64tc) mode = RSVD_MODE_PLAIN;   // plain in everything but the passes over A
  if ((mode == RSVD_MODE_PLAIN) != (a_dtype == RSVD_F64)) return -6;
  if (mode == RSVD_MODE_MIXED && l_max > 256) return -4;
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
  P->batched = 0;
  P->scales = nullptr;
  P->lds = P->scale_rows = P->scale_cols = 0;
  P->batch_lay = nullptr;
  P->h_ctx = nullptr;
  P->ctx_event = nullptr;
  P->batch_engine = kBatchSimt;
  P->batch_graphs = 0;
  P->batch_sms = 0;
  P->batch_tc = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost((void**)&P->h_status, sizeof(int) * 8) != cudaSuccess) {
    delete P;
    return RSVD_ERR_CUDA;
  }
  P->f64tc = f64tc ? 1 : 0;
  P->lay = make_layout(m_max, n_max, l_max, mode, P->num_sms, f64tc);
  std::memset(P->h_status, 0, sizeof(int) * 8);
  *plan = P;
  return RSVD_OK;
}

int rsvd_workspace_size(rsvd_plan_t plan, size_t* bytes) {
  if (!plan) return -1;
  if (!bytes) return -2;
  *bytes = plan->batched ? plan->batch_lay->total : plan->lay.total;
  return RSVD_OK;
}

int rsvd_batch_plan_create(rsvd_plan_t* plan, int max_count, int64_t rows_total,
                           int64_t cols_total, int l_max, int a_dtype, void* cuda_stream) {
  if (!plan) return -1;
  *plan = nullptr;
  if (max_count < 1) return -2;
  if (rows_total < 1) return -3;
  if (cols_total < 1) return -4;
  if (l_max < 1 || l_max > RSVD_L_MAX) return -5;
  if (a_dtype != RSVD_F64 && a_dtype != RSVD_F32) return -6;
  rsvd_plan_s* P = new (std::nothrow) rsvd_plan_s();
  if (!P) return RSVD_ERR_CUDA;
  P->m_max = rows_total;
  P->n_max = cols_total;
  P->l_max = l_max;
  P->dtype = a_dtype;
  P->mode = RSVD_MODE_PLAIN;
  P->stream = (cudaStream_t)cuda_stream;
  P->ws = nullptr;
  P->ws_bytes = 0;
  P->batched = 1;
  P->max_count = max_count;
  P->rows_total = rows_total;
  P->cols_total = cols_total;
  P->h_ctx = nullptr;
  P->ctx_event = nullptr;
  P->h_status = nullptr;
  P->batch_engine = a_dtype == RSVD_F32 ? kBatchTensor : kBatchSimt;
  P->batch_graphs = 0;
  P->batch_sms = 0;
  P->batch_tc = nullptr;
  P->batch_lay = new (std::nothrow) BatchLayout(
      make_batch_layout(max_count, rows_total, cols_total, l_max, a_dtype));
  int dev = 0;
  if (!P->batch_lay || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost(&P->h_ctx, batch_ctx_bytes(max_count) + 4 * sizeof(int) * max_count) !=
          cudaSuccess ||
      cudaMallocHost((void**)&P->h_status, sizeof(int) * 8) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ctx_event, cudaEventDisableTiming) != cudaSuccess) {
    if (P->h_ctx) cudaFreeHost(P->h_ctx);
    if (P->h_status) cudaFreeHost(P->h_status);
    delete P->batch_lay;
    delete P;
    return RSVD_ERR_CUDA;
  }
  *plan = P;
  return RSVD_OK;
}

int rsvd_solve_batched(rsvd_plan_t plan, int count, const rsvd_problem_t* problems) {
  if (!plan || !plan->batched) return -1;
  if (count < 1 || count > plan->max_count) return -2;
  if (!problems) return -3;
  if (!plan->ws || plan->ws_bytes < plan->batch_lay->total) return RSVD_ERR_WORKSPACE;
  int64_t rows = 0, cols = 0;
  for (int i = 0; i < count; ++i) {
    const rsvd_problem_t& q = problems[i];
    const int l = q.k + q.p;
    if (!q.A || q.m < 1 || q.n < 1 || q.lda < q.m || q.k < 1 || q.p < 0 || q.q < 0 ||
        l > (q.m < q.n ? q.m : q.n) || !q.U || q.ldu < q.m || !q.S || !q.VT || q.ldvt < q.k)
      return -(100 + i);
    if (l > plan->l_max) return RSVD_ERR_WORKSPACE;
    rows += q.m;
    cols += q.n;
  }
  if (rows > plan->rows_total || cols > plan->cols_total) return RSVD_ERR_WORKSPACE;
  return solve_batched(plan, count, problems);
}

int rsvd_batch_set_engine(rsvd_plan_t plan, int engine) {
  if (!plan || !plan->batched) return -1;
  if (engine != RSVD_BATCH_ENGINE_SIMT && engine != RSVD_BATCH_ENGINE_TENSOR) return -2;
  if (engine == RSVD_BATCH_ENGINE_TENSOR && plan->dtype != RSVD_F32) return RSVD_ERR_UNSUPPORTED;
  plan->batch_engine = engine == RSVD_BATCH_ENGINE_TENSOR ? kBatchTensor : kBatchSimt;
  return RSVD_OK;
}

int rsvd_batch_set_graphs(rsvd_plan_t plan, int on) {
  if (!plan || !plan->batched) return -1;
  if (on && (plan->dtype != RSVD_F32 || plan->batch_engine != kBatchTensor))
    return RSVD_ERR_UNSUPPORTED;
  if (on && plan->stream == nullptr) return -2;
  plan->batch_graphs = on ? 1 : 0;
  return RSVD_OK;
}

int rsvd_batch_set_sm_limit(rsvd_plan_t plan, int sms) {
  if (!plan || !plan->batched) return -1;
  if (sms < 0) return -2;
  plan->batch_sms = sms;
  return RSVD_OK;
}

int rsvd_batch_autotune(rsvd_plan_t plan, int count, const rsvd_problem_t* problems) {
  if (!plan || !plan->batched) return -1;
  if (count < 1 || count > plan->max_count) return -2;
  if (!problems) return -3;
  if (plan->dtype != RSVD_F32 || plan->batch_engine != kBatchTensor) return RSVD_ERR_UNSUPPORTED;
  if (!plan->ws || plan->ws_bytes < plan->batch_lay->total) return RSVD_ERR_WORKSPACE;
  int64_t rows = 0, cols = 0;
  for (int i = 0; i < count; ++i) {
    const rsvd_problem_t& q = problems[i];
    const int l = q.k + q.p;
    if (!q.A || q.m < 1 || q.n < 1 || q.lda < q.m || q.k < 1 || q.p < 0 || q.q < 0 ||
        l > (q.m < q.n ? q.m : q.n) || !q.U || q.ldu < q.m || !q.S || !q.VT || q.ldvt < q.k)
      return -(100 + i);
    if (l > plan->l_max) return RSVD_ERR_WORKSPACE;
    rows += q.m;
    cols += q.n;
  }
  if (rows > plan->rows_total || cols > plan->cols_total) return RSVD_ERR_WORKSPACE;
  return batch_autotune(plan, count, problems);
}

int rsvd_grouped_gemm_f32(rsvd_plan_t plan, int count, const rsvd_gemm_t* gemms, int trans) {
  if (!plan || !plan->batched || plan->dtype != RSVD_F32 || plan->batch_engine != kBatchTensor)
    return -1;
  if (count < 1 || count > plan->max_count) return -2;
  if (!gemms) return -3;
  if (!plan->ws || plan->ws_bytes < plan->batch_lay->total) return RSVD_ERR_WORKSPACE;
  for (int i = 0; i < count; ++i) {
    const rsvd_gemm_t& g = gemms[i];
    const bool bad = g.M < 0 || g.M > (1 << 30) || g.K < 1 || g.K > (1 << 30) || g.N < 1 ||
                     g.N > RSVD_L_MAX ||
                     (g.M > 0 && (!g.A || !g.X || !g.C || g.ldc < g.M || g.ldx < g.K ||
                                  g.lda < (trans ? g.K : g.M)));
    if (bad) return -(100 + i);
  }
  return grouped_gemm_f32(plan, count, gemms, trans);
}

int rsvd_grouped_schedule(int count, const int64_t* shapes, int trans, int num_sms, int* units,
                          int max_units, int* cta_off, int* info) {
  if (count < 1) return -1;
  if (!shapes || !info) return -2;
  if (num_sms < 1) return -3;
  std::vector<GtcShape> sh(count);
  for (int i = 0; i < count; ++i) {
    const int64_t M = shapes[3 * i], K = shapes[3 * i + 1], N = shapes[3 * i + 2];
    if (M < 0 || M > (1 << 30) || K < 1 || K > (1 << 30) || N < 1 || N > RSVD_L_MAX)
      return -(100 + i);
    sh[i] = {(int)M, (int)K, (int)N};
  }
  GtcSchedule sc;
  gtc_schedule(sh.data(), count, !trans, num_sms, sc);
  info[0] = (int)sc.units.size();
  info[1] = sc.grid;
  info[2] = sc.slots;
  info[3] = sc.tmax;
  if ((units && max_units < (int)sc.units.size())) return RSVD_ERR_WORKSPACE;
  if (units)
    for (size_t u = 0; u < sc.units.size(); ++u) {
      const GtcUnit& x = sc.units[u];
      const int v[7] = {x.prob, x.row0, x.col0, x.kb0, x.kb1, x.slot, x.t};
      for (int j = 0; j < 7; ++j) units[7 * u + j] = v[j];
    }
  if (cta_off) {
    if (num_sms < sc.grid) return RSVD_ERR_WORKSPACE;
    for (int c = 0; c <= sc.grid; ++c) cta_off[c] = sc.cta_off[c];
    for (int c = sc.grid + 1; c <= num_sms; ++c) cta_off[c] = sc.cta_off[sc.grid];
  }
  return RSVD_OK;
}

int rsvd_batch_status(rsvd_plan_t plan, int count, int* codes) {
  if (!plan || !plan->batched) return -1;
  if (count < 1 || count > plan->max_count) return -2;
  if (!codes) return -3;
  if (!plan->ws) return RSVD_ERR_WORKSPACE;
  return batch_status(plan, count, codes);
}

int rsvd_set_workspace(rsvd_plan_t plan, void* dev_ptr, size_t bytes) {
  if (!plan) return -1;
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign)) return -2;
  if (plan->batched) {
    if (bytes < plan->batch_lay->total) return RSVD_ERR_WORKSPACE;
    plan->ws = (char*)dev_ptr;
    plan->ws_bytes = bytes;
    return RSVD_OK;
  }
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

int rsvd_plan_set_wait_limit(rsvd_plan_t plan, int64_t cycles) {
  if (!plan) return -1;
  if (cycles < 0) return -2;
  plan->wait_cycles = (long long)cycles;
  return RSVD_OK;
}

int rsvd_plan_prepare_a(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max) return RSVD_ERR_WORKSPACE;
  if (!plan->f64tc) return RSVD_OK;
  plan->tc_pinned = 0;
  const int rc = f64tc_begin(plan, (const double*)A, m, n, lda);
  if (rc == RSVD_OK) plan->tc_pinned = 1;
  return rc;
}

int rsvd_plan_release_a(rsvd_plan_t plan) {
  if (!plan) return -1;
  plan->tc_pinned = 0;
  if (plan->f64tc) f64tc_end(plan);
  return RSVD_OK;
}

int rsvd_set_tile_scales(rsvd_plan_t plan, const float* scales, int64_t rows, int64_t cols,
                         int64_t lds) {
  if (!plan) return -1;
  if (plan->dtype != RSVD_FP8E4M3) return RSVD_ERR_UNSUPPORTED;
  if (!scales) return -2;
  if (rows < 1) return -3;
  if (cols < 1) return -4;
  if (lds < rows) return -5;
  // the scales are read once here and checked: every one must be a positive
  // power of two (the tensor-core path folds it into BF16 exactly)
  std::vector<float> h((size_t)lds * cols);
  if (cudaMemcpy(h.data(), scales, h.size() * sizeof(float), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return RSVD_ERR_CUDA;
  for (int64_t J = 0; J < cols; ++J)
    for (int64_t I = 0; I < rows; ++I)
      if (!power_of_two(h[I + J * lds])) return -2;
  plan->scales = scales;
  plan->lds = lds;
  plan->scale_rows = rows;
  plan->scale_cols = cols;
  return RSVD_OK;
}

int rsvd_plan_status(rsvd_plan_t plan) {
  if (!plan) return -1;
  if (!plan->ws) return RSVD_ERR_WORKSPACE;
  if (plan->batched) {
    // per-problem codes: rsvd_batch_status; here only the plan-wide word of
    // the tensor engine (a timeout of a grouped launch), read and cleared
    if (plan->batch_lay->xs_ncols == 0)
      return cudaStreamSynchronize(plan->stream) == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
    int* g = (int*)(plan->ws + plan->batch_lay->gflags);
    if (cudaMemcpyAsync(plan->h_status, g, sizeof(int), cudaMemcpyDeviceToHost, plan->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(plan->stream) != cudaSuccess)
      return RSVD_ERR_CUDA;
    const int flags = plan->h_status[0];
    if (cudaMemsetAsync(g, 0, sizeof(int), plan->stream) != cudaSuccess) return RSVD_ERR_CUDA;
    return status_from_flags(flags);
  }
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
  if (plan->h_ctx) cudaFreeHost(plan->h_ctx);
  if (plan->ctx_event) cudaEventDestroy(plan->ctx_event);
  batch_tc_free(plan);
  delete plan->batch_lay;
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
    case RSVD_ERR_NOT_REACHED: return "tolerance not reached within l_cap columns";
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
  if (plan->mode == RSVD_MODE_MIXED && (lda % 8 || ((uintptr_t)A % 16)))
    return RSVD_ERR_UNSUPPORTED;
  if (plan->dtype == RSVD_FP8E4M3 && !fp8_ready(plan, m, n, lda)) return RSVD_ERR_UNSUPPORTED;
  if (plan->mode == RSVD_MODE_PLAIN) {
    TcScope tc(plan, A, m, n, lda);
    if (tc.rc) return tc.rc;
    return solve_plain(plan, (const double*)A, m, n, lda, k, p, q, seed, (double*)U, ldu, S,
                       (double*)VT, ldvt);
  }
  return solve_mixed(plan, A, m, n, lda, k, p, q, seed, (float*)U, ldu, S, (float*)VT, ldvt);
}

int rsvd_solve_algorithm(rsvd_plan_t plan, int algorithm, const void* A, int64_t m, int64_t n,
                         int64_t lda, int k, int p, int q, uint64_t seed, void* U, int64_t ldu,
                         double* S, void* VT, int64_t ldvt) {
  if (!plan) return -1;
  if (algorithm != 2 && algorithm != 3 && algorithm != 4 && algorithm != 6) return -2;
  if (!A) return -3;
  if (m < 1) return -4;
  if (n < 1) return -5;
  if (lda < m) return -6;
  if (k < 1) return -7;
  if (p < 0) return -8;
  if (q < 0) return -9;
  if (!U) return -11;
  if (ldu < m) return -12;
  if (!S) return -13;
  if (!VT) return -14;
  if (ldvt < k) return -15;
  const int l = k + p;
  if (l > (m < n ? m : n)) return -8;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->batched) return RSVD_ERR_UNSUPPORTED;
  if (algorithm == 2) q = 0;   // Algorithm 2 is Algorithm 4 without power steps
  if (algorithm == 2 || algorithm == 4)
    return rsvd_solve(plan, A, m, n, lda, k, p, q, seed, U, ldu, S, VT, ldvt);
  if (plan->mode != RSVD_MODE_PLAIN) return RSVD_ERR_UNSUPPORTED;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  if (algorithm == 3)
    return solve_plain_alg3(plan, (const double*)A, m, n, lda, k, p, q, seed, (double*)U, ldu, S,
                            (double*)VT, ldvt);
  return solve_singlepass(plan, (const double*)A, m, n, lda, k, p, seed, (double*)U, ldu, S,
                          (double*)VT, ldvt);
}

int rsvd_solve_singlepass(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                          int k, int p, uint64_t seed, void* U, int64_t ldu, double* S, void* VT,
                          int64_t ldvt) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (k < 1) return -6;
  if (p < 0) return -7;
  if (!U) return -9;
  if (ldu < m) return -10;
  if (!S) return -11;
  if (!VT) return -12;
  if (ldvt < k) return -13;
  const int l = k + p;
  if (l > (m < n ? m : n)) return -7;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode != RSVD_MODE_PLAIN || plan->batched) return RSVD_ERR_UNSUPPORTED;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  return solve_singlepass(plan, (const double*)A, m, n, lda, k, p, seed, (double*)U, ldu, S,
                          (double*)VT, ldvt);
}

int rsvd_solve_hermitian(rsvd_plan_t plan, const void* A, int64_t n, int64_t lda, int k, int p,
                         uint64_t seed, void* U, int64_t ldu, double* D) {
  if (!plan) return -1;
  if (!A) return -2;
  if (n < 1) return -3;
  if (lda < n) return -4;
  if (k < 1) return -5;
  if (p < 0) return -6;
  if (k + p > n) return -6;
  if (!U) return -8;
  if (ldu < n) return -9;
  if (!D) return -10;
  if (!ready(plan) || n > plan->m_max || n > plan->n_max || k + p > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode != RSVD_MODE_PLAIN || plan->batched) return RSVD_ERR_UNSUPPORTED;
  TcScope tc(plan, A, n, n, lda);
  if (tc.rc) return tc.rc;
  return solve_hermitian(plan, (const double*)A, n, lda, k, p, seed, (double*)U, ldu, D);
}

namespace {

// Shared argument checks of the two adaptive entry points (positions of
// A .. seed are the same in both); returns 0 or the error code.
int adaptive_args(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, double eps,
                  int r, int l_cap, const int* rank) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (!(eps > 0.0) || !std::isfinite(eps)) return -6;
  if (r < 1) return -7;
  if (l_cap < 1 || l_cap > (m < n ? m : n)) return -8;
  if (!rank) return -20;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l_cap > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (r >= (plan->l_max < 64 ? plan->l_max : 64)) return -7;
  if (plan->mode != RSVD_MODE_PLAIN || plan->batched) return RSVD_ERR_UNSUPPORTED;
  return 0;
}

}  // namespace

int rsvd_range_adaptive(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                        double eps, int r, int l_cap, uint64_t seed, void* Q, int64_t ldq,
                        int* rank) {
  int rc = adaptive_args(plan, A, m, n, lda, eps, r, l_cap, rank);
  if (rc == -20) return -12;
  if (rc) return rc;
  if (!Q) return -10;
  if (ldq < m) return -11;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  return range_adaptive(plan, (const double*)A, m, n, lda, eps, r, l_cap, seed, (double*)Q, ldq,
                        rank);
}

int rsvd_solve_adaptive(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                        double eps, int r, int l_cap, uint64_t seed, void* U, int64_t ldu,
                        double* S, void* VT, int64_t ldvt, int* rank) {
  int rc = adaptive_args(plan, A, m, n, lda, eps, r, l_cap, rank);
  if (rc == -20) return -15;
  if (rc) return rc;
  if (!U) return -10;
  if (ldu < m) return -11;
  if (!S) return -12;
  if (!VT) return -13;
  if (ldvt < l_cap) return -14;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  return solve_adaptive(plan, (const double*)A, m, n, lda, eps, r, l_cap, seed, (double*)U, ldu,
                        S, (double*)VT, ldvt, rank);
}

namespace {

int srft_args(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int l,
              const void* out, int64_t ldo) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1 || n > INT32_MAX) return -4;
  if (lda < m) return -5;
  if (l < 1 || l > (m < n ? m : n) || 2 * l > RSVD_L_MAX) return -6;
  if (!out) return -8;
  if (ldo < m) return -9;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || 2 * l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode != RSVD_MODE_PLAIN || plan->batched) return RSVD_ERR_UNSUPPORTED;
  return 0;
}

}  // namespace

int rsvd_range_srft(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int l,
                    uint64_t seed, void* Q, int64_t ldq) {
  const int rc = srft_args(plan, A, m, n, lda, l, Q, ldq);
  if (rc) return rc;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  return range_srft(plan, (const double*)A, m, n, lda, l, seed, (double*)Q, ldq);
}

int rsvd_solve_srft(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int k,
                    int p, uint64_t seed, void* U, int64_t ldu, double* S, void* VT,
                    int64_t ldvt) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1 || n > INT32_MAX) return -4;
  if (lda < m) return -5;
  if (k < 1) return -6;
  if (p < 0 || k + p > (m < n ? m : n) || 2 * (k + p) > RSVD_L_MAX) return -7;
  if (!U) return -9;
  if (ldu < m) return -10;
  if (!S) return -11;
  if (!VT) return -12;
  if (ldvt < k) return -13;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || 2 * (k + p) > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->mode != RSVD_MODE_PLAIN || plan->batched) return RSVD_ERR_UNSUPPORTED;
  TcScope tc(plan, A, m, n, lda);
  if (tc.rc) return tc.rc;
  return solve_srft(plan, (const double*)A, m, n, lda, k, p, seed, (double*)U, ldu, S,
                    (double*)VT, ldvt);
}

int rsvd_srft_sketch(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int l,
                     uint64_t seed, void* Y, int64_t ldy) {
  const int rc = srft_args(plan, A, m, n, lda, l, Y, ldy);
  if (rc) return rc;
  return sketch_srft(plan, (const double*)A, m, n, lda, l, seed, (double*)Y, ldy);
}

int rsvd_gaussian(rsvd_plan_t plan, int64_t n, int l, uint64_t seed, uint32_t stream, int out_dtype,
                  void* out, int64_t ldo) {
  if (!plan) return -1;
  if (n < 1) return -2;
  if (l < 1) return -3;
  if (out_dtype != RSVD_F64 && out_dtype != RSVD_F32 && out_dtype != RSVD_BF16) return -6;
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
  if (plan->dtype == RSVD_FP8E4M3 && !fp8_ready(plan, m, n, lda)) return RSVD_ERR_UNSUPPORTED;
  if (plan->mode == RSVD_MODE_PLAIN) {
    TcScope tc(plan, A, m, n, lda);
    if (tc.rc) return tc.rc;
    return gemm<double>(plan, (const double*)A, lda, false, (const double*)X, ldx, (double*)Y, ldy,
                        m, n, l);
  }
  return mixed_apply(plan, A, m, n, lda, X, ldx, l, (float*)Y, ldy, false);
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
  if (plan->dtype == RSVD_FP8E4M3 && !fp8_ready(plan, m, n, lda)) return RSVD_ERR_UNSUPPORTED;
  if (plan->mode == RSVD_MODE_PLAIN) {
    TcScope tc(plan, A, m, n, lda);
    if (tc.rc) return tc.rc;
    return gemm<double>(plan, (const double*)A, lda, true, (const double*)X, ldx, (double*)Z, ldz,
                        n, m, l);
  }
  return mixed_apply(plan, A, m, n, lda, X, ldx, l, (float*)Z, ldz, true);
}

int rsvd_apply_split(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                     int trans, const float* X, int64_t ldx, int l, int slices, float* out,
                     int64_t ldo) {
  if (!plan) return -1;
  if (!A) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (lda < m) return -5;
  if (trans != 0 && trans != 1) return -6;
  const int64_t rows = trans ? m : n, rows_out = trans ? n : m;
  if (!X) return -7;
  if (ldx < rows) return -8;
  if (l < 1) return -9;
  if (slices < 1 || slices > 3) return -10;
  if (!out) return -11;
  if (ldo < rows_out) return -12;
  if (plan->mode != RSVD_MODE_MIXED) return RSVD_ERR_UNSUPPORTED;
  if (!ready(plan) || m > plan->m_max || n > plan->n_max || l > plan->l_max)
    return RSVD_ERR_WORKSPACE;
  if (plan->dtype == RSVD_FP8E4M3 && !fp8_ready(plan, m, n, lda)) return RSVD_ERR_UNSUPPORTED;
  return mixed_apply_split(plan, A, m, n, lda, X, ldx, l, slices, out, ldo, trans != 0);
}

int rsvd_orth(rsvd_plan_t plan, const void* Y, int64_t rows, int l, int64_t ldy, void* Q,
              int64_t ldq, void* R, int64_t ldr) {
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
  int rc;
  size_t es;
  void* Rtmp;
  if (plan->mode == RSVD_MODE_PLAIN) {
    Work<double> W = work_of<double>(plan);
    Rtmp = W.Mt;
    es = sizeof(double);
    rc = orth<double>(plan, (const double*)Y, rows, l, ldy, (double*)Q, ldq, R ? W.Mt : nullptr,
                      false);
  } else {
    Work<float> W = work_of<float>(plan);
    Rtmp = W.Mt;
    es = sizeof(float);
    rc = orth<float>(plan, (const float*)Y, rows, l, ldy, (float*)Q, ldq, R ? W.Mt : nullptr,
                     false);
  }
  if (rc) return rc;
  if (R)
    CK(cudaMemcpy2DAsync(R, ldr * es, Rtmp, l * es, l * es, l, cudaMemcpyDeviceToDevice,
                         plan->stream));
  return RSVD_OK;
}

int rsvd_small_svd(rsvd_plan_t plan, const void* M, int l, int64_t ldm, void* sig, void* Um,
                   int64_t ldu, void* Vm, int64_t ldv) {
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
  if (plan->mode == RSVD_MODE_PLAIN) {
    Work<double> W = work_of<double>(plan);
    CK(launch_jacobi_svd<double>((const double*)M, l, ldm, (double*)sig, (double*)Um, ldu,
                                 (double*)Vm, ldv, nullptr, W.jw, dstatus(plan), plan->stream));
  } else {
    Work<float> W = work_of<float>(plan);
    CK(launch_jacobi_svd<float>((const float*)M, l, ldm, (float*)sig, (float*)Um, ldu,
                                (float*)Vm, ldv, nullptr, W.jw, dstatus(plan), plan->stream));
  }
  return RSVD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch accounting
// ---------------------------------------------------------------------------
#include <atomic>
#include <mutex>

namespace {
std::atomic<uint64_t> g_launches{0};
}

void rsvd::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

size_t rsvd::dynamic_smem_cap(const void* func) {
  struct Entry {
    const void* func;
    int device;
    size_t cap;
  };
  static Entry cache[64];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (cache[i].func == func && cache[i].device == dev) return cache[i].cap;
  int optin = 0;
  cudaFuncAttributes fa{};
  size_t cap = 48 * 1024;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, func) == cudaSuccess && (size_t)optin > fa.sharedSizeBytes) {
    const size_t c = (size_t)optin - fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c) ==
        cudaSuccess)
      cap = c;
  }
  cudaGetLastError();  // a refused attribute leaves the 48 KB default, not a sticky error
  if (used < 64) cache[used++] = Entry{func, dev, cap};
  return cap;
}

extern "C" uint64_t rsvd_kernel_launches(void) {
  return g_launches.load(std::memory_order_relaxed);
}
