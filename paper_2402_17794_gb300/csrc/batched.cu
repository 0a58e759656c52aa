// Many independent randomized SVDs (Algorithm 4, Section 3.3) in grouped
// launches: every step of the path runs once for the whole batch.
//
//  * One table of per-problem contexts (operand pointers, sizes, workspace
//    slices) is copied to the device per batched solve; every grouped kernel
//    reads its problem's entry with blockIdx.y (GEMMs, elementwise steps) or
//    blockIdx.x (the l x l steps), so uneven sizes share one launch and no
//    launch depends on another problem's size beyond the grid bounds.
//  * GEMMs: 2-D grid (row tiles of the largest problem, problems[, column
//    tiles]); CTAs past a problem's extent exit at once.  No split-K, so a
//    problem's result does not depend on what else is in the batch.
//  * l x l steps (Cholesky + inverse, Jacobi SVD, signs): one CTA per problem.
//  * Power steps: problem i takes part in iteration j only while j < q_i.
// Arithmetic is FP64 (RSVD_F64 plans) or FP32 (RSVD_F32 plans) throughout.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batched.h"
#include "gemm_body.cuh"
#include "grouped_tc.h"
#include "omega_body.cuh"
#include "pipeline.h"
#include "small_body.cuh"

namespace rsvd {
namespace {

using dense::SMALL_THREADS;
using simt::BM;
using simt::THREADS;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

template <typename T>
struct Ctx {
  const T* A;
  int64_t m, n, lda;
  int k, p, q, l;
  uint64_t seed;
  T* U;
  int64_t ldu;
  double* S;
  T* VT;
  int64_t ldvt;
  T *om, *y, *qm, *tmp, *z, *qb;
  T *G, *R1, *R1i, *R2, *R2i, *Mt, *Um, *UsInv, *jw, *sig, *sign, *cholw;
  DeviceStatus* status;
  void* xs;   // tensor engine: this problem's slab of BF16 operand slices
};

// GEMM operands of each grouped step for one problem.
enum GOp {
  OP_A_OM_Y = 0,    // Y = A Omega (or A W)
  OP_AT_QM_Z,       // Z = A^T Q
  OP_GRAM_Y,        // G = Y^T Y
  OP_GRAM_Z,        // G = Z^T Z
  OP_GRAM_TM,       // G = T^T T, T m x l
  OP_GRAM_TN,       // G = T^T T, T n x l
  OP_TRSM_Y,        // T = Y R1^-1 (m x l)
  OP_TRSM_Z,        // T = Z R1^-1 (n x l)
  OP_TRSM_TM_QM,    // Q = T R2^-1 (m x l)
  OP_TRSM_TN_OM,    // W = T R2^-1 (n x l)
  OP_LIFT_U,        // U = Q U~_k
  OP_LIFT_V,        // T = Z (U~ Sigma^-1)_k   (n x k)
  OP_GRAM_V,        // G = T^T T (k x k)
  OP_TRSM_V,        // Qb = T R1^-1 (n x k)
  OP_COUNT
};

template <typename T>
__device__ __forceinline__ GemmArgs<T> op_args(const Ctx<T>& P, int op) {
  const int l = P.l, k = P.k;
  switch (op) {
    case OP_A_OM_Y: return {P.A, P.lda, false, P.om, P.n, P.y, P.m, P.m, P.n, l};
    case OP_AT_QM_Z: return {P.A, P.lda, true, P.qm, P.m, P.z, P.n, P.n, P.m, l};
    case OP_GRAM_Y: return {P.y, P.m, true, P.y, P.m, P.G, l, l, P.m, l};
    case OP_GRAM_Z: return {P.z, P.n, true, P.z, P.n, P.G, l, l, P.n, l};
    case OP_GRAM_TM: return {P.tmp, P.m, true, P.tmp, P.m, P.G, l, l, P.m, l};
    case OP_GRAM_TN: return {P.tmp, P.n, true, P.tmp, P.n, P.G, l, l, P.n, l};
    case OP_TRSM_Y: return {P.y, P.m, false, P.R1i, l, P.tmp, P.m, P.m, l, l};
    case OP_TRSM_Z: return {P.z, P.n, false, P.R1i, l, P.tmp, P.n, P.n, l, l};
    case OP_TRSM_TM_QM: return {P.tmp, P.m, false, P.R2i, l, P.qm, P.m, P.m, l, l};
    case OP_TRSM_TN_OM: return {P.tmp, P.n, false, P.R2i, l, P.om, P.n, P.n, l, l};
    case OP_LIFT_U: return {P.qm, P.m, false, P.Um, l, P.U, P.ldu, P.m, l, k};
    case OP_LIFT_V: return {P.z, P.n, false, P.UsInv, l, P.tmp, P.n, P.n, l, k};
    case OP_GRAM_V: return {P.tmp, P.n, true, P.tmp, P.n, P.G, k, k, P.n, k};
    default: return {P.tmp, P.n, false, P.R1i, k, P.qb, P.n, P.n, k, k};
  }
}

// iter >= 0: only problems with q > iter take part (power steps).
__device__ __forceinline__ bool active(int q, int iter) { return iter < 0 || iter < q; }

template <typename T, int TN, bool TRANS>
__global__ void __launch_bounds__(THREADS)
grouped_gemm_kernel(const Ctx<T>* __restrict__ ctx, int op, int iter) {
  const Ctx<T>& P = ctx[blockIdx.y];
  if (!active(P.q, iter)) return;
  const GemmArgs<T> g = op_args(P, op);
  const int64_t r0 = (int64_t)blockIdx.x * BM;
  const int c0 = blockIdx.z * 16 * TN;
  if (r0 >= g.M || c0 >= g.N) return;
  simt::gemm_tile<T, TN, TRANS>(g.A, g.lda, g.X, g.ldx, g.C, g.ldc, g.M, g.N, r0, c0, 0, g.K);
}

// Tensor engine: the grouped step's product table, one entry per problem
// (M = 0 for problems outside this power iteration).  The column tile follows
// the same rule as the host schedule, from the tile limits in `caps`.
__global__ void gtc_table_kernel(const Ctx<float>* __restrict__ ctx, int count, int op, int iter,
                                 int x_upper, GtcCaps caps, GtcGemm* __restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const Ctx<float>& P = ctx[i];
  const GemmArgs<float> a = op_args(P, op);
  GtcGemm g;
  g.A = a.A;
  g.X = a.X;
  g.C = a.C;
  g.xs = reinterpret_cast<uint16_t*>(P.xs);
  g.lda = a.lda;
  g.ldx = a.ldx;
  g.ldc = a.ldc;
  g.M = active(P.q, iter) ? (int)a.M : 0;
  g.K = (int)a.K;
  g.N = a.N;
  g.x_upper = x_upper;
  g.kpad = (g.K + kGtcBlockK - 1) / kGtcBlockK * kGtcBlockK;
  const int t = gtc_tile_rule(g.N, caps.cap[gtc_bucket(g.N)]);
  g.ncols = (g.N + t - 1) / t * t;
  g.t = t;
  g.pad_ = 0;
  tab[i] = g;
}

// Cholesky + inverse: which 0 -> (G, l) into R1/R1i, 1 -> into R2/R2i,
// 2 -> (G, k) into R1/R1i (re-orthonormalisation of V_k).  The register
// variant serves FP32 problems with l <= 160, the shared-memory one the rest.
template <typename T>
__global__ void __launch_bounds__(dense::CHOL_THREADS)
grouped_chol_kernel(const Ctx<T>* __restrict__ ctx, int which, int iter, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Ctx<T>& P = ctx[blockIdx.x];
  if (!active(P.q, iter)) return;
  const int l = which == 2 ? P.k : P.l;
  T* R = which == 1 ? P.R2 : P.R1;
  T* Ri = which == 1 ? P.R2i : P.R1i;
  T* W = use_smem ? reinterpret_cast<T*>(smem_raw) : P.cholw;
  dense::chol_inv_blocked<T, dense::CholPanel<T>::value>(P.G, l, l, R, Ri, W, P.status);
}

template <int E>
__global__ void __launch_bounds__(dense::CHOL_REG_THREADS)
grouped_chol_regs_kernel(const Ctx<float>* __restrict__ ctx, int which, int iter) {
  const Ctx<float>& P = ctx[blockIdx.x];
  if (!active(P.q, iter)) return;
  const int l = which == 2 ? P.k : P.l;
  float* R = which == 1 ? P.R2 : P.R1;
  float* Ri = which == 1 ? P.R2i : P.R1i;
  dense::chol_inv_regs<E>(P.G, l, l, R, Ri, P.status);
}

// Mt = (R2 R1)^T, the transposed R factor of B^T.
template <typename T>
__global__ void grouped_tri_kernel(const Ctx<T>* __restrict__ ctx) {
  const Ctx<T>& P = ctx[blockIdx.y];
  const int l = P.l;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < l * l; t += gridDim.x * blockDim.x) {
    const int i = t % l, j = t / l;
    T s = T(0);
    if (i <= j)
      for (int u = i; u <= j; ++u) s = fma(P.R2[i + u * l], P.R1[u + j * l], s);
    P.Mt[j + i * l] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(dense::JACOBI_THREADS)
grouped_jacobi_kernel(const Ctx<T>* __restrict__ ctx, int use_smem) {
  extern __shared__ __align__(16) unsigned char jsm_raw[];
  const Ctx<T>& P = ctx[blockIdx.x];
  T* Wm = use_smem ? reinterpret_cast<T*>(jsm_raw) : P.jw;
  dense::jacobi_body<T, dense::JACOBI_REGS_SMALL>(P.Mt, P.l, P.l, P.sig, P.Um, P.l, nullptr, P.l,
                                                  P.UsInv, Wm,
                        dense::jacobi_ld<T>(P.l, use_smem != 0), P.status);
}

template <typename T>
__global__ void grouped_gaussian_kernel(const Ctx<T>* __restrict__ ctx);

template <>
__global__ void grouped_gaussian_kernel<double>(const Ctx<double>* __restrict__ ctx) {
  const Ctx<double>& P = ctx[blockIdx.y];
  const uint64_t total = (uint64_t)P.n * (uint64_t)P.l;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x)
    P.om[t] = omega::gaussian_value_f64(t, 0u, P.seed);   // om is n x l, ld n: index t = j*n + i
}

// FP32 batches draw Omega with the FP32 generator (24-bit uniforms, FP32
// Box-Muller): the FP64 transcendentals run at the GPU's FP64 rate, and the
// FP32 solve cannot resolve the difference.
template <>
__global__ void grouped_gaussian_kernel<float>(const Ctx<float>* __restrict__ ctx) {
  const Ctx<float>& P = ctx[blockIdx.y];
  const uint64_t total = (uint64_t)P.n * (uint64_t)P.l;
  const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x)
    P.om[t] = omega::gaussian_at_f32(t, 0u, k0, k1);
}

template <typename T>
__global__ void grouped_sign_kernel(const Ctx<T>* __restrict__ ctx) {
  const Ctx<T>& P = ctx[blockIdx.y];
  const int col = blockIdx.x;
  if (col >= P.k) return;
  dense::sign_body<T>(P.U + (int64_t)col * P.ldu, P.m, P.sign + col);
}

template <typename T>
__global__ void grouped_vt_kernel(const Ctx<T>* __restrict__ ctx) {
  const Ctx<T>& P = ctx[blockIdx.y];
  const int64_t total = P.n * (int64_t)P.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / P.k;
    const int i = (int)(t - j * P.k);
    P.VT[i + j * P.ldvt] = P.sign[i] * P.qb[j + (int64_t)i * P.n];
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < P.k; i += blockDim.x) P.S[i] = (double)P.sig[i];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct BatchShape {
  int count;
  int64_t max_m, max_n;
  int max_l, max_k, max_q;
};

template <typename T>
size_t small_elems(int l) {
  const int lpad = (l + 1) & ~1;
  return 8 * (size_t)l * l + 2 * (size_t)l * lpad + 2 * (size_t)l + (size_t)l * l +
         33 * (size_t)(l + 64);
}

// ---- tensor engine (FP32 batches) ----
// The grouped products of a solve come in ten shapes (M, K, N per problem);
// each has one work schedule, built on the host when the batch's shapes
// change and kept on the device.
constexpr int kGeo = 10;
int geo_of(int op) {
  switch (op) {
    case OP_A_OM_Y: return 0;
    case OP_AT_QM_Z: return 1;
    case OP_GRAM_Y: case OP_GRAM_TM: return 2;
    case OP_GRAM_Z: case OP_GRAM_TN: return 3;
    case OP_TRSM_Y: case OP_TRSM_TM_QM: return 4;
    case OP_TRSM_Z: case OP_TRSM_TN_OM: return 5;
    case OP_LIFT_U: return 6;
    case OP_LIFT_V: return 7;
    case OP_GRAM_V: return 8;
    default: return 9;   // OP_TRSM_V
  }
}
bool geo_ax(int g) { return !(g == 1 || g == 2 || g == 3 || g == 8); }
bool op_upper(int op) {
  return op == OP_TRSM_Y || op == OP_TRSM_Z || op == OP_TRSM_TM_QM || op == OP_TRSM_TN_OM ||
         op == OP_TRSM_V;
}
GtcShape geo_shape(int g, int64_t m64, int64_t n64, int l, int k) {
  const int m = (int)m64, n = (int)n64;
  switch (g) {
    case 0: return {m, n, l};
    case 1: return {n, m, l};
    case 2: return {l, m, l};
    case 3: return {l, n, l};
    case 4: return {m, l, l};
    case 5: return {n, l, l};
    case 6: return {m, l, k};
    case 7: return {n, l, k};
    case 8: return {k, n, k};
    default: return {n, k, k};
  }
}
// a representative op of each shape (tuning runs)
int geo_op(int g) {
  const int ops[kGeo] = {OP_A_OM_Y, OP_AT_QM_Z, OP_GRAM_Y, OP_GRAM_Z, OP_TRSM_Y,
                         OP_TRSM_Z, OP_LIFT_U, OP_LIFT_V, OP_GRAM_V, OP_TRSM_V};
  return ops[g];
}

struct BatchTc {
  std::vector<int64_t> sig;    // shapes and tuning generation the solve's schedules were built for
  std::vector<int64_t> gsig;   // the same for the schedule of rsvd_grouped_gemm_f32
  GtcSchedule s[kGeo];
  size_t uoff[kGeo], coff[kGeo], foff[kGeo];
  std::vector<char> blob;
  // CUDA graph of a whole grouped solve (rsvd_batch_set_graphs), valid for
  // the launch signature xsig
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> xsig;
  ~BatchTc() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Lays out schedules (units, CTA offsets, fix entries) in one blob at the
// start of the plan's schedule region and copies it there (stream-ordered).
int tc_upload(rsvd_plan_t P, BatchTc& S, int first, int last) {
  const BatchLayout& L = *P->batch_lay;
  S.blob.clear();
  size_t off = 0;
  for (int g = first; g < last; ++g) {
    const GtcSchedule& sc = S.s[g];
    S.uoff[g] = off;
    off = align16(off + sc.units.size() * sizeof(GtcUnit));
    S.coff[g] = off;
    off = align16(off + sc.cta_off.size() * sizeof(int));
    S.foff[g] = off;
    off = align16(off + sc.fix.size() * sizeof(GtcFix));
  }
  if (off > L.sched_bytes) return RSVD_ERR_WORKSPACE;
  S.blob.assign(off, 0);
  for (int g = first; g < last; ++g) {
    const GtcSchedule& sc = S.s[g];
    if (!sc.units.empty())
      std::memcpy(S.blob.data() + S.uoff[g], sc.units.data(), sc.units.size() * sizeof(GtcUnit));
    std::memcpy(S.blob.data() + S.coff[g], sc.cta_off.data(), sc.cta_off.size() * sizeof(int));
    if (!sc.fix.empty())
      std::memcpy(S.blob.data() + S.foff[g], sc.fix.data(), sc.fix.size() * sizeof(GtcFix));
  }
  if (off) RSVD_CK(cudaMemcpyAsync(P->ws + L.sched, S.blob.data(), off, cudaMemcpyHostToDevice,
                                   P->stream));
  return RSVD_OK;
}

// A schedule whose partial slots do not fit is rebuilt without splits.
void tc_build(rsvd_plan_t P, const GtcShape* sh, int count, bool ax, GtcSchedule& out,
              int force_chunk = 0, const GtcCaps* caps = nullptr) {
  const BatchLayout& L = *P->batch_lay;
  const int sms = P->batch_sms > 0 ? std::min(P->batch_sms, P->num_sms) : P->num_sms;
  gtc_schedule(sh, count, ax, sms, out, force_chunk, caps);
  if ((size_t)out.slots * 128 * out.tmax > L.part_floats)
    gtc_schedule(sh, count, ax, sms, out, 1 << 30, caps);
}

// Schedules of the ten shapes for the batch in the host context table.
int tc_prepare(rsvd_plan_t P, int count) {
  BatchTc* S = reinterpret_cast<BatchTc*>(P->batch_tc);
  if (!S) {
    S = new (std::nothrow) BatchTc();
    if (!S) return RSVD_ERR_CUDA;
    P->batch_tc = S;
  }
  const Ctx<float>* h = reinterpret_cast<const Ctx<float>*>(P->h_ctx);
  std::vector<int64_t> sig;
  sig.reserve(4 * (size_t)count + 2);
  sig.push_back(count);
  sig.push_back(gtc_generation());
  sig.push_back(P->batch_sms);
  for (int i = 0; i < count; ++i) {
    sig.push_back(h[i].m);
    sig.push_back(h[i].n);
    sig.push_back(h[i].l);
    sig.push_back(h[i].k);
  }
  if (sig == S->sig) return RSVD_OK;
  S->sig.clear();
  S->gsig.clear();   // the schedule region is rewritten below
  std::vector<GtcShape> sh(count);
  for (int g = 0; g < kGeo; ++g) {
    for (int i = 0; i < count; ++i) sh[i] = geo_shape(g, h[i].m, h[i].n, h[i].l, h[i].k);
    tc_build(P, sh.data(), count, geo_ax(g), S->s[g]);
  }
  int rc = tc_upload(P, *S, 0, kGeo);
  if (rc) return rc;
  S->sig.swap(sig);
  return RSVD_OK;
}

// One grouped product on the tensor engine: table, X slices, pass.
int gtc_run(rsvd_plan_t P, const Ctx<float>* d, int count, int op, int iter,
            const GtcSchedule& sc, size_t uoff, size_t coff, size_t foff, const GtcCaps& caps) {
  const BatchLayout& L = *P->batch_lay;
  GtcGemm* tab = reinterpret_cast<GtcGemm*>(P->ws + L.gtab);
  gtc_table_kernel<<<(count + 127) / 128, 128, 0, P->stream>>>(d, count, op, iter,
                                                              op_upper(op) ? 1 : 0, caps, tab);
  note_launch();
  RSVD_CK(cudaGetLastError());
  int rc = launch_gtc_split(tab, count, (int)std::min<int64_t>(P->rows_total, 1 << 20),
                            sc.tmax, P->stream);
  if (rc) return rc;
  GtcLaunch g;
  g.ax = geo_ax(geo_of(op));
  g.gemm = tab;
  g.count = count;
  g.tmax = sc.tmax;
  g.units = reinterpret_cast<const GtcUnit*>(P->ws + L.sched + uoff);
  g.cta_off = reinterpret_cast<const int*>(P->ws + L.sched + coff);
  g.grid = sc.grid;
  g.fix = reinterpret_cast<const GtcFix*>(P->ws + L.sched + foff);
  g.nfix = (int)sc.fix.size();
  g.part = reinterpret_cast<float*>(P->ws + L.part);
  g.status = reinterpret_cast<int*>(P->ws + L.gflags);
  g.wait_cycles = P->wait_cycles;
  return launch_gtc(g, P->stream);
}

int gtc_op(rsvd_plan_t P, const Ctx<float>* d, const BatchShape& b, int op, int iter) {
  BatchTc* S = reinterpret_cast<BatchTc*>(P->batch_tc);
  const int g = geo_of(op);
  GtcCaps caps;
  gtc_caps(caps);
  return gtc_run(P, d, b.count, op, iter, S->s[g], S->uoff[g], S->coff[g], S->foff[g], caps);
}

template <typename T, bool TRANS>
int launch_grouped_gemm(rsvd_plan_t P, const Ctx<T>* dctx, const BatchShape& b, int op, int iter,
                        int64_t max_rows, int max_cols) {
  const int per = std::min(max_cols, 96);
  const int tn = (per + 15) / 16;
  const int col_tiles = (max_cols + 16 * tn - 1) / (16 * tn);
  dim3 grid((unsigned)((max_rows + BM - 1) / BM), (unsigned)b.count, (unsigned)col_tiles);
  switch (tn) {
#define RSVD_G(TNV) \
  case TNV: grouped_gemm_kernel<T, TNV, TRANS><<<grid, THREADS, 0, P->stream>>>(dctx, op, iter); break;
    RSVD_G(1) RSVD_G(2) RSVD_G(3) RSVD_G(4) RSVD_G(5) RSVD_G(6)
#undef RSVD_G
    default: return RSVD_ERR_UNSUPPORTED;
  }
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

template <typename T>
int gop(rsvd_plan_t P, const Ctx<T>* d, const BatchShape& b, int op, int iter) {
  if constexpr (sizeof(T) == 4) {
    if (P->batch_engine == kBatchTensor)
      return gtc_op(P, reinterpret_cast<const Ctx<float>*>(d), b, op, iter);
  }
  const int64_t mm = b.max_m, nn = b.max_n;
  const int L = b.max_l, K = b.max_k;
  switch (op) {
    case OP_A_OM_Y: return launch_grouped_gemm<T, false>(P, d, b, op, iter, mm, L);
    case OP_AT_QM_Z: return launch_grouped_gemm<T, true>(P, d, b, op, iter, nn, L);
    case OP_GRAM_Y: case OP_GRAM_Z: case OP_GRAM_TM: case OP_GRAM_TN:
      return launch_grouped_gemm<T, true>(P, d, b, op, iter, L, L);
    case OP_TRSM_Y: case OP_TRSM_TM_QM: return launch_grouped_gemm<T, false>(P, d, b, op, iter, mm, L);
    case OP_TRSM_Z: case OP_TRSM_TN_OM: return launch_grouped_gemm<T, false>(P, d, b, op, iter, nn, L);
    case OP_LIFT_U: return launch_grouped_gemm<T, false>(P, d, b, op, iter, mm, K);
    case OP_LIFT_V: return launch_grouped_gemm<T, false>(P, d, b, op, iter, nn, K);
    case OP_GRAM_V: return launch_grouped_gemm<T, true>(P, d, b, op, iter, K, K);
    default: return launch_grouped_gemm<T, false>(P, d, b, op, iter, nn, K);
  }
}

template <typename T>
int gchol(rsvd_plan_t P, const Ctx<T>* d, const BatchShape& b, int which, int iter) {
  const int l = which == 2 ? b.max_k : b.max_l;
  const size_t smem = dense::chol_work_elems(l) * sizeof(T);
  const bool sm = smem <= dynamic_smem_cap((const void*)grouped_chol_kernel<T>);
  if constexpr (sizeof(T) == 4) {
    if (dense::chol_in_regs<T>(l)) {
      // the block edge covers the batch's largest l; smaller problems leave
      // their extra rows and columns at zero
      const int nt = dense::CHOL_REG_THREADS;
      switch (dense::chol_reg_edge(l)) {
        case 1: grouped_chol_regs_kernel<1><<<b.count, nt, 0, P->stream>>>(d, which, iter); break;
        case 2: grouped_chol_regs_kernel<2><<<b.count, nt, 0, P->stream>>>(d, which, iter); break;
        case 3: grouped_chol_regs_kernel<3><<<b.count, nt, 0, P->stream>>>(d, which, iter); break;
        case 4: grouped_chol_regs_kernel<4><<<b.count, nt, 0, P->stream>>>(d, which, iter); break;
        default: grouped_chol_regs_kernel<5><<<b.count, nt, 0, P->stream>>>(d, which, iter);
      }
      note_launch();
      RSVD_CK(cudaGetLastError());
      return RSVD_OK;
    }
  }
  grouped_chol_kernel<T><<<b.count, dense::CHOL_THREADS, sm ? smem : 0, P->stream>>>(d, which, iter,
                                                                               sm ? 1 : 0);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

// CholeskyQR2 over the batch: src -> dst (dst_op < 0: only the R factor Mt).
template <typename T>
int gorth(rsvd_plan_t P, const Ctx<T>* d, const BatchShape& b, bool on_m, int iter, bool want_q,
          bool want_r) {
  int rc;
  if ((rc = gop<T>(P, d, b, on_m ? OP_GRAM_Y : OP_GRAM_Z, iter))) return rc;
  if ((rc = gchol<T>(P, d, b, 0, iter))) return rc;
  if ((rc = gop<T>(P, d, b, on_m ? OP_TRSM_Y : OP_TRSM_Z, iter))) return rc;
  if ((rc = gop<T>(P, d, b, on_m ? OP_GRAM_TM : OP_GRAM_TN, iter))) return rc;
  if ((rc = gchol<T>(P, d, b, 1, iter))) return rc;
  if (want_q && (rc = gop<T>(P, d, b, on_m ? OP_TRSM_TM_QM : OP_TRSM_TN_OM, iter))) return rc;
  if (want_r) {
    dim3 grid((unsigned)std::max(1, (b.max_l * b.max_l + 255) / 256), (unsigned)b.count);
    grouped_tri_kernel<T><<<grid, 256, 0, P->stream>>>(d);
    note_launch();
    RSVD_CK(cudaGetLastError());
  }
  return RSVD_OK;
}

// Y = A W or Y = A Omega for every problem; orth(Y) -> Q.  (Z, W likewise.)
template <typename T>
int solve_batched_t(rsvd_plan_t P, const Ctx<T>* d, const BatchShape& b) {
  int rc;
  {
    dim3 grid(64, (unsigned)b.count);
    grouped_gaussian_kernel<T><<<grid, 256, 0, P->stream>>>(d);
    note_launch();
    RSVD_CK(cudaGetLastError());
  }
  if ((rc = gop<T>(P, d, b, OP_A_OM_Y, -1))) return rc;
  if ((rc = gorth<T>(P, d, b, true, -1, true, false))) return rc;
  for (int j = 0; j < b.max_q; ++j) {
    if ((rc = gop<T>(P, d, b, OP_AT_QM_Z, j))) return rc;
    if ((rc = gorth<T>(P, d, b, false, j, true, false))) return rc;
    if ((rc = gop<T>(P, d, b, OP_A_OM_Y, j))) return rc;
    if ((rc = gorth<T>(P, d, b, true, j, true, false))) return rc;
  }
  if ((rc = gop<T>(P, d, b, OP_AT_QM_Z, -1))) return rc;
  if ((rc = gorth<T>(P, d, b, false, -1, false, true))) return rc;
  {
    // every problem's l <= max_l: the padded stride is not monotone in l
    size_t need = 0;
    for (int ll = 1; ll <= b.max_l; ++ll)
      need = std::max(need, (size_t)dense::jacobi_ld<T>(ll, true) * ((ll + 1) & ~1) * sizeof(T));
    const bool sm = need <= dynamic_smem_cap((const void*)grouped_jacobi_kernel<T>);
    grouped_jacobi_kernel<T><<<b.count, dense::JACOBI_THREADS, sm ? need : 0, P->stream>>>(
        d, sm ? 1 : 0);
    note_launch();
    RSVD_CK(cudaGetLastError());
  }
  if ((rc = gop<T>(P, d, b, OP_LIFT_U, -1))) return rc;
  if ((rc = gop<T>(P, d, b, OP_LIFT_V, -1))) return rc;
  if ((rc = gop<T>(P, d, b, OP_GRAM_V, -1))) return rc;
  if ((rc = gchol<T>(P, d, b, 2, -1))) return rc;
  if ((rc = gop<T>(P, d, b, OP_TRSM_V, -1))) return rc;
  {
    dim3 grid((unsigned)b.max_k, (unsigned)b.count);
    grouped_sign_kernel<T><<<grid, 1024, 0, P->stream>>>(d);
    note_launch();
    dim3 g2(64, (unsigned)b.count);
    grouped_vt_kernel<T><<<g2, 256, 0, P->stream>>>(d);
    note_launch();
    RSVD_CK(cudaGetLastError());
  }
  return RSVD_OK;
}

template <typename T>
int fill_ctx(rsvd_plan_t P, int count, const rsvd_problem_t* pr, BatchShape* b) {
  const BatchLayout& L = *P->batch_lay;
  Ctx<T>* h = reinterpret_cast<Ctx<T>*>(P->h_ctx);
  char* ws = P->ws;
  int64_t moff = 0, noff = 0, xoff = 0;
  b->count = count;
  b->max_m = b->max_n = 0;
  b->max_l = b->max_k = 1;
  b->max_q = 0;
  const size_t per_small = align_up(small_elems<T>(P->l_max) * sizeof(T)) +
                           align_up(sizeof(DeviceStatus));
  for (int i = 0; i < count; ++i) {
    const rsvd_problem_t& q = pr[i];
    Ctx<T>& c = h[i];
    const int l = q.k + q.p;
    c.A = (const T*)q.A;
    c.m = q.m;
    c.n = q.n;
    c.lda = q.lda;
    c.k = q.k;
    c.p = q.p;
    c.q = q.q;
    c.l = l;
    c.seed = q.seed;
    c.U = (T*)q.U;
    c.ldu = q.ldu;
    c.S = q.S;
    c.VT = (T*)q.VT;
    c.ldvt = q.ldvt;
    const int lm = P->l_max;
    c.om = (T*)(ws + L.om) + noff * lm;
    c.z = (T*)(ws + L.z) + noff * lm;
    c.qb = (T*)(ws + L.qb) + noff * lm;
    c.y = (T*)(ws + L.y) + moff * lm;
    c.qm = (T*)(ws + L.qm) + moff * lm;
    c.tmp = (T*)(ws + L.tmp) + (moff + noff) * lm;
    char* sb = ws + L.small + (size_t)i * per_small;
    T* s = (T*)sb;
    const size_t ll = (size_t)lm * lm;
    c.G = s;
    c.R1 = s + ll;
    c.R1i = s + 2 * ll;
    c.R2 = s + 3 * ll;
    c.R2i = s + 4 * ll;
    c.Mt = s + 5 * ll;
    c.Um = s + 6 * ll;
    c.UsInv = s + 7 * ll;
    c.jw = s + 8 * ll;
    const int lpad = (lm + 1) & ~1;
    c.sig = c.jw + 2 * (size_t)lm * lpad;
    c.sign = c.sig + lm;
    c.cholw = c.sign + lm;
    c.status = (DeviceStatus*)(sb + align_up(small_elems<T>(lm) * sizeof(T)));
    c.xs = nullptr;
    if (L.xs_ncols > 0) {
      c.xs = ws + L.xs + (size_t)3 * 2 * L.xs_ncols * xoff;
      xoff += std::max(q.m, q.n) + kGtcBlockK;
    }
    moff += q.m;
    noff += q.n;
    b->max_m = std::max(b->max_m, q.m);
    b->max_n = std::max(b->max_n, q.n);
    b->max_l = std::max(b->max_l, l);
    b->max_k = std::max(b->max_k, q.k);
    b->max_q = std::max(b->max_q, q.q);
  }
  return RSVD_OK;
}

}  // namespace

BatchLayout make_batch_layout(int max_count, int64_t rows_total, int64_t cols_total, int l,
                              int dtype) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t e = dtype == RSVD_F64 ? sizeof(double) : sizeof(float);
  const size_t small = dtype == RSVD_F64 ? small_elems<double>(l) : small_elems<float>(l);
  L.om = take((size_t)cols_total * l * e);
  L.z = take((size_t)cols_total * l * e);
  L.qb = take((size_t)cols_total * l * e);
  L.y = take((size_t)rows_total * l * e);
  L.qm = take((size_t)rows_total * l * e);
  L.tmp = take((size_t)(rows_total + cols_total) * l * e);
  L.small = take((size_t)max_count * (align_up(small * e) + align_up(sizeof(DeviceStatus))));
  L.ctx = take((size_t)max_count * sizeof(Ctx<double>));
  L.xs_ncols = 0;
  L.sched_bytes = L.part_floats = 0;
  L.gtab = L.xs = L.sched = L.part = L.gflags = off;
  if (dtype == RSVD_F32) {
    // slabs: 3 slices x (max(m, n) + 64) rows x (l rounded to 16 + 80) columns
    // of BF16 per problem; schedules: ten shapes of at most
    // 4 (rows + cols) / 128 + count row tiles x ceil(l / 48) column tiles each
    L.xs_ncols = (l + 15) / 16 * 16 + kGtcMaxTile;
    L.gtab = take((size_t)max_count * sizeof(GtcGemm));
    L.xs = take((size_t)3 * 2 * L.xs_ncols * (size_t)(rows_total + cols_total +
                                                      (int64_t)kGtcBlockK * max_count));
    const size_t tiles = (size_t)4 * ((size_t)(rows_total + cols_total) / 128 + 2 * max_count) *
                         (size_t)((l + 47) / 48);
    L.sched_bytes = (size_t)kGeo * (tiles * (sizeof(GtcUnit) + sizeof(GtcFix)) + 4096 + 64);
    L.sched = take(L.sched_bytes);
    // partial slots of split tiles: up to eight per problem
    L.part_floats = (size_t)std::max(1024, 8 * max_count) * 128 * kGtcMaxTile;
    L.part = take(L.part_floats * sizeof(float));
    L.gflags = take(256);
  }
  L.total = off;
  return L;
}

size_t batch_ctx_bytes(int max_count) { return (size_t)max_count * sizeof(Ctx<double>); }

namespace {

// Everything a grouped FP32 solve enqueues after its context table is
// filled on the host (the part a CUDA graph captures): the table copy, the
// status words, and the steps of Algorithm 4.
int enqueue_f32(rsvd_plan_t P, int count, const BatchShape& b, bool capturing) {
  const size_t bytes = (size_t)count * sizeof(Ctx<double>);
  void* dctx = P->ws + P->batch_lay->ctx;
  RSVD_CK(cudaMemcpyAsync(dctx, P->h_ctx, bytes, cudaMemcpyHostToDevice, P->stream));
  // in a graph, an external record node: the event is recorded at every
  // replay, so the next solve's host side waits for this copy
  RSVD_CK(capturing ? cudaEventRecordWithFlags(P->ctx_event, P->stream, cudaEventRecordExternal)
                    : cudaEventRecord(P->ctx_event, P->stream));
  const size_t per_small = align_up(small_elems<float>(P->l_max) * sizeof(float)) +
                           align_up(sizeof(DeviceStatus));
  const size_t st_off = per_small - align_up(sizeof(DeviceStatus));
  RSVD_CK(cudaMemset2DAsync(P->ws + P->batch_lay->small + st_off, per_small, 0,
                            sizeof(DeviceStatus), count, P->stream));
  if (P->batch_engine == kBatchTensor)
    RSVD_CK(cudaMemsetAsync(P->ws + P->batch_lay->gflags, 0, sizeof(int), P->stream));
  return solve_batched_t<float>(P, reinterpret_cast<const Ctx<float>*>(dctx), b);
}

// The same as one CUDA graph: captured when the launch signature (shapes,
// power steps, tuning generation, wait limit) differs from the last capture,
// replayed otherwise.  The graph's table copy reads the pinned staging
// buffer at replay time, so new operands of the same shapes need no new
// capture.
int solve_f32_graph(rsvd_plan_t P, int count, const BatchShape& b) {
  int rc;
  if ((rc = tc_prepare(P, count))) return rc;   // schedule upload: outside the capture
  BatchTc* S = reinterpret_cast<BatchTc*>(P->batch_tc);
  const Ctx<float>* h = reinterpret_cast<const Ctx<float>*>(P->h_ctx);
  std::vector<int64_t> sig = S->sig;
  sig.push_back(P->wait_cycles);
  for (int i = 0; i < count; ++i) sig.push_back(h[i].q);
  if (!S->exec || sig != S->xsig) {
    if (S->exec) cudaGraphExecDestroy(S->exec);
    S->exec = nullptr;
    S->xsig.clear();
    RSVD_CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    const int rc2 = enqueue_f32(P, count, b, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(P->stream, &graph);
    if (rc2 || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc2 ? rc2 : RSVD_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&S->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      S->exec = nullptr;
      return RSVD_ERR_CUDA;
    }
    S->xsig.swap(sig);
  }
  RSVD_CK(cudaGraphLaunch(S->exec, P->stream));
  return RSVD_OK;
}

}  // namespace

int solve_batched(rsvd_plan_t P, int count, const rsvd_problem_t* pr) {
  // the previous solve's table copy must have left the staging buffer
  if (cudaEventSynchronize(P->ctx_event) != cudaSuccess) return RSVD_ERR_CUDA;
  BatchShape b;
  int rc;
  const size_t bytes = (size_t)count * sizeof(Ctx<double>);
  void* dctx = P->ws + P->batch_lay->ctx;
  if (P->dtype == RSVD_F64) {
    if ((rc = fill_ctx<double>(P, count, pr, &b))) return rc;
  } else {
    if ((rc = fill_ctx<float>(P, count, pr, &b))) return rc;
    if (P->batch_graphs && P->batch_engine == kBatchTensor && P->stream != nullptr)
      return solve_f32_graph(P, count, b);
  }
  RSVD_CK(cudaMemcpyAsync(dctx, P->h_ctx, bytes, cudaMemcpyHostToDevice, P->stream));
  RSVD_CK(cudaEventRecord(P->ctx_event, P->stream));
  // per-problem status words start clear
  {
    const size_t per_small =
        (P->dtype == RSVD_F64 ? align_up(small_elems<double>(P->l_max) * sizeof(double))
                              : align_up(small_elems<float>(P->l_max) * sizeof(float))) +
        align_up(sizeof(DeviceStatus));
    const size_t st_off = per_small - align_up(sizeof(DeviceStatus));
    RSVD_CK(cudaMemset2DAsync(P->ws + P->batch_lay->small + st_off, per_small, 0, sizeof(DeviceStatus),
                              count, P->stream));
  }
  if (P->dtype == RSVD_F64)
    return solve_batched_t<double>(P, (const Ctx<double>*)dctx, b);
  if (P->batch_engine == kBatchTensor) {
    if ((rc = tc_prepare(P, count))) return rc;
    RSVD_CK(cudaMemsetAsync(P->ws + P->batch_lay->gflags, 0, sizeof(int), P->stream));
  }
  return solve_batched_t<float>(P, (const Ctx<float>*)dctx, b);
}

namespace {

BatchTc* tc_state(rsvd_plan_t P) {
  if (!P->batch_tc) P->batch_tc = new (std::nothrow) BatchTc();
  return reinterpret_cast<BatchTc*>(P->batch_tc);
}

// Mean time of `reps` runs of one grouped product under schedule g of S.
int time_run(rsvd_plan_t P, const Ctx<float>* d, int count, int g, BatchTc& S, const GtcCaps& caps,
             cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int rc;
  if ((rc = gtc_run(P, d, count, geo_op(g), -1, S.s[g], S.uoff[g], S.coff[g], S.foff[g], caps)))
    return rc;
  RSVD_CK(cudaEventRecord(e0, P->stream));
  const int reps = 3;
  for (int r = 0; r < reps; ++r)
    if ((rc = gtc_run(P, d, count, geo_op(g), -1, S.s[g], S.uoff[g], S.coff[g], S.foff[g], caps)))
      return rc;
  RSVD_CK(cudaEventRecord(e1, P->stream));
  RSVD_CK(cudaEventSynchronize(e1));
  RSVD_CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  return RSVD_OK;
}

int autotune_body(rsvd_plan_t P, int count, const Ctx<float>* d, BatchTc& S, cudaEvent_t e0,
                  cudaEvent_t e1) {
  const Ctx<float>* h = reinterpret_cast<const Ctx<float>*>(P->h_ctx);
  std::vector<GtcShape> sh(count);
  int rc;
  // 1. column tile limits for N above 80, on the passes over A (shapes 0, 1)
  for (int g = 0; g < 2; ++g) {
    std::vector<int> seen;
    for (int i = 0; i < count; ++i) {
      const int N = h[i].l;
      const int B = gtc_bucket(N);
      if (N <= kGtcMaxTile || gtc_tile_tuned(N) ||
          std::find(seen.begin(), seen.end(), B) != seen.end())
        continue;
      seen.push_back(B);
      int best = kGtcMaxTile;
      float best_ms = 1e30f;
      for (int cap : {48, 64, 80}) {
        GtcCaps c2;
        gtc_caps(c2);
        c2.cap[B] = cap;
        for (int j = 0; j < count; ++j) {
          sh[j] = geo_shape(g, h[j].m, h[j].n, h[j].l, h[j].k);
          if (gtc_bucket(sh[j].N) != B) sh[j].M = 0;
        }
        tc_build(P, sh.data(), count, geo_ax(g), S.s[g], 0, &c2);
        if ((rc = tc_upload(P, S, g, g + 1))) return rc;
        float ms = 0.f;
        if ((rc = time_run(P, d, count, g, S, c2, e0, e1, &ms))) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best = cap;
        }
      }
      gtc_set_tile_cap(N, best);
    }
  }
  // 2. contraction chunk per (form, K bucket) on the passes and the Grams
  GtcCaps caps;
  gtc_caps(caps);
  for (int g = 0; g < 4; ++g) {
    const bool ax = geo_ax(g);
    std::vector<int> seen;
    for (int i = 0; i < count; ++i) {
      const GtcShape si = geo_shape(g, h[i].m, h[i].n, h[i].l, h[i].k);
      const int K = si.K, M = si.M;
      const int B = gtc_bucket(K) + 32 * (M <= 128 ? 1 : 0);
      if (gtc_chunk_tuned(ax, K, M) || std::find(seen.begin(), seen.end(), B) != seen.end())
        continue;
      seen.push_back(B);
      int kbmax = 1;
      for (int j = 0; j < count; ++j) {
        sh[j] = geo_shape(g, h[j].m, h[j].n, h[j].l, h[j].k);
        if (gtc_bucket(sh[j].K) + 32 * (sh[j].M <= 128 ? 1 : 0) != B) sh[j].M = 0;
        else kbmax = std::max(kbmax, (sh[j].K + kGtcBlockK - 1) / kGtcBlockK);
      }
      int best = kGtcDefaultChunk;
      float best_ms = 1e30f;
      bool whole_done = false;
      for (int chunk : {4, 8, 16, 32, 64, 128, 256}) {
        if (chunk >= kbmax) {
          if (whole_done) continue;   // every candidate from here on splits nothing
          whole_done = true;
        }
        tc_build(P, sh.data(), count, ax, S.s[g], chunk, &caps);
        if ((rc = tc_upload(P, S, g, g + 1))) return rc;
        float ms = 0.f;
        if ((rc = time_run(P, d, count, g, S, caps, e0, e1, &ms))) return rc;
        if (ms < best_ms * 0.97f) {   // a split has to win clearly
          best_ms = ms;
          best = chunk;
        }
      }
      gtc_set_chunk(ax, K, M, best);
    }
  }
  return RSVD_OK;
}

}  // namespace

int batch_autotune(rsvd_plan_t P, int count, const rsvd_problem_t* pr) {
  if (P->dtype != RSVD_F32 || P->batch_engine != kBatchTensor) return RSVD_ERR_UNSUPPORTED;
  if (cudaEventSynchronize(P->ctx_event) != cudaSuccess) return RSVD_ERR_CUDA;
  BatchShape b;
  int rc;
  if ((rc = fill_ctx<float>(P, count, pr, &b))) return rc;
  void* dctx = P->ws + P->batch_lay->ctx;
  RSVD_CK(cudaMemcpyAsync(dctx, P->h_ctx, (size_t)count * sizeof(Ctx<double>),
                          cudaMemcpyHostToDevice, P->stream));
  BatchTc* S = tc_state(P);
  if (!S) return RSVD_ERR_CUDA;
  S->sig.clear();   // the schedule region is reused by the trial runs
  S->gsig.clear();
  cudaEvent_t e0, e1;
  RSVD_CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RSVD_ERR_CUDA;
  }
  rc = autotune_body(P, count, reinterpret_cast<const Ctx<float>*>(dctx), *S, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RSVD_CK(cudaEventRecord(P->ctx_event, P->stream));
  S->sig.clear();
  return rc;
}

int grouped_gemm_f32(rsvd_plan_t P, int count, const rsvd_gemm_t* gm, int trans) {
  const BatchLayout& L = *P->batch_lay;
  std::vector<GtcGemm> tab(count);
  std::vector<GtcShape> sh(count);
  const size_t xs_cap = (size_t)3 * 2 * L.xs_ncols *
                        (size_t)(P->rows_total + P->cols_total + (int64_t)kGtcBlockK * P->max_count);
  size_t xoff = 0;
  for (int i = 0; i < count; ++i) {
    const rsvd_gemm_t& q = gm[i];
    GtcGemm& g = tab[i];
    g.A = q.A;
    g.X = q.X;
    g.C = q.C;
    g.lda = q.lda;
    g.ldx = q.ldx;
    g.ldc = q.ldc;
    g.M = (int)q.M;
    g.K = (int)q.K;
    g.N = q.N;
    g.x_upper = q.x_upper ? 1 : 0;
    g.kpad = (g.K + kGtcBlockK - 1) / kGtcBlockK * kGtcBlockK;
    const int t = gtc_tile(g.N);
    g.ncols = (g.N + t - 1) / t * t;
    g.t = t;
    g.pad_ = 0;
    const size_t bytes = (size_t)3 * 2 * g.kpad * g.ncols;
    g.xs = reinterpret_cast<uint16_t*>(P->ws + L.xs + xoff);
    xoff += (bytes + 255) / 256 * 256;
    if (xoff > xs_cap) return RSVD_ERR_WORKSPACE;
    sh[i] = {g.M, g.K, g.N};
  }
  BatchTc* S = tc_state(P);
  if (!S) return RSVD_ERR_CUDA;
  const int g = trans ? 1 : 0;
  int rc;
  // the schedule depends only on the shapes: kept across calls with the same ones
  std::vector<int64_t> sig;
  sig.reserve(3 * (size_t)count + 3);
  sig.push_back(trans);
  sig.push_back(count);
  sig.push_back(gtc_generation());
  sig.push_back(P->batch_sms);
  for (const GtcShape& x : sh) {
    sig.push_back(x.M);
    sig.push_back(x.K);
    sig.push_back(x.N);
  }
  if (sig != S->gsig) {
    S->sig.clear();   // the schedule region is overwritten
    S->gsig.clear();
    tc_build(P, sh.data(), count, !trans, S->s[g]);
    if ((rc = tc_upload(P, *S, g, g + 1))) return rc;
    S->gsig.swap(sig);
  }
  GtcGemm* dtab = reinterpret_cast<GtcGemm*>(P->ws + L.gtab);
  RSVD_CK(cudaMemcpyAsync(dtab, tab.data(), (size_t)count * sizeof(GtcGemm),
                          cudaMemcpyHostToDevice, P->stream));
  int max_kpad = 64;
  for (const GtcGemm& t : tab) max_kpad = std::max(max_kpad, t.kpad);
  if ((rc = launch_gtc_split(dtab, count, max_kpad, S->s[g].tmax, P->stream))) return rc;
  GtcLaunch l;
  l.ax = !trans;
  l.gemm = dtab;
  l.count = count;
  l.tmax = S->s[g].tmax;
  l.units = reinterpret_cast<const GtcUnit*>(P->ws + L.sched + S->uoff[g]);
  l.cta_off = reinterpret_cast<const int*>(P->ws + L.sched + S->coff[g]);
  l.grid = S->s[g].grid;
  l.fix = reinterpret_cast<const GtcFix*>(P->ws + L.sched + S->foff[g]);
  l.nfix = (int)S->s[g].fix.size();
  l.part = reinterpret_cast<float*>(P->ws + L.part);
  l.status = reinterpret_cast<int*>(P->ws + L.gflags);
  l.wait_cycles = P->wait_cycles;
  RSVD_CK(cudaMemsetAsync(P->ws + L.gflags, 0, sizeof(int), P->stream));
  return launch_gtc(l, P->stream);
}

void batch_tc_free(rsvd_plan_t P) {
  delete reinterpret_cast<BatchTc*>(P->batch_tc);
  P->batch_tc = nullptr;
}

int batch_status(rsvd_plan_t P, int count, int* codes) {
  const size_t per_small =
      (P->dtype == RSVD_F64 ? align_up(small_elems<double>(P->l_max) * sizeof(double))
                            : align_up(small_elems<float>(P->l_max) * sizeof(float))) +
      align_up(sizeof(DeviceStatus));
  const size_t st_off = per_small - align_up(sizeof(DeviceStatus));
  // gather the first word (flags) of each problem's status into the pinned buffer
  RSVD_CK(cudaMemcpy2DAsync(P->h_ctx, sizeof(int), P->ws + P->batch_lay->small + st_off, per_small,
                            sizeof(int), count, cudaMemcpyDeviceToHost, P->stream));
  int* f = (int*)P->h_ctx;
  f[count] = 0;
  if (P->batch_lay->xs_ncols > 0)   // a timeout in a tensor-engine launch concerns every problem
    RSVD_CK(cudaMemcpyAsync(f + count, P->ws + P->batch_lay->gflags, sizeof(int),
                            cudaMemcpyDeviceToHost, P->stream));
  RSVD_CK(cudaStreamSynchronize(P->stream));
  for (int i = 0; i < count; ++i) codes[i] = status_from_flags(f[i] | f[count]);
  return RSVD_OK;
}

}  // namespace rsvd
