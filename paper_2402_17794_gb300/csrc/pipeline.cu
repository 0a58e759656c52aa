// Host-side orchestration of Algorithm 4 (Section 3.3) for both paths.
//
// Plain path (FP64 A):   every step in FP64; passes over A on the CUDA cores,
//                        or (RSVD_MODE_F64_TENSOR plans) on the tensor cores
//                        as exact products of BF16 digit slices.
// Mixed path (BF16 A):   passes over A on the tcgen05 tensor cores with BF16
//                        operands and FP32 accumulation; everything else in
//                        FP32.  The q power steps use a single BF16 copy of
//                        the operand; one extra power step follows with the
//                        operand split in two BF16 slices (bf16x2, ~16 bits),
//                        and the final B^T = A^T Q uses three slices
//                        (bf16x3, ~24 bits, i.e. FP32-accurate since A is
//                        exact in BF16).
//
// Steps shared by both paths (templated on the element type):
//   orth       CholeskyQR2 (Gram on the CUDA cores, one-CTA Cholesky + inverse)
//   finish     B^T = Q_B R_B (R only), one-sided Jacobi of R_B^T, U = Q U~,
//              V = B^T U~ Sigma^-1 re-orthonormalised, signs and output layout.
#include <algorithm>

#include "pipeline.h"
#include "umma.h"

namespace rsvd {

namespace {

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }
int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

// x = x_1 + x_2 + ... : slice s of column c (blockIdx.y = s * stride + c)
// holds the BF16 rounding of what the earlier slices left over.
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t rows, int l, int64_t ldx,
                                  int stride, __nv_bfloat16* __restrict__ out, int64_t ldo) {
  const int cc = blockIdx.y;
  const int s = cc / stride, c = cc - s * stride;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    float v = (c < l) ? X[r + (int64_t)c * ldx] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    for (int j = 0; j < s; ++j) {  // peel the leading slices off
      v -= __bfloat162float(h);
      h = __float2bfloat16_rn(v);
    }
    out[r + (int64_t)cc * ldo] = h;
  }
}

int split_operand(rsvd_plan_t P, const float* X, int64_t rows, int l, int64_t ldx, int slices,
                  int stride, __nv_bfloat16* out, int64_t ldo) {
  const int bx = (int)std::min<int64_t>((rows + 255) / 256, 16);
  dim3 grid(bx, slices * stride);
  split_bf16_kernel<<<grid, 256, 0, P->stream>>>(X, rows, l, ldx, stride, out, ldo);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

// FP8 A: the same pass with block-scaled E4M3 MMAs, the operand in
// 2 x `slices` E4M3 slices (4 significant bits each, so the same precision
// as `slices` BF16 slices).
int mx8_pass(rsvd_plan_t P, bool ax, const void* A, int64_t m, int64_t n, int64_t lda,
             const float* X, int64_t ldxf, int l, int slices, float* out, int64_t ldo,
             bool accumulate) {
  MixedWork MW = mixed_work_of(P);
  const int64_t rows = ax ? n : m;
  const int64_t ldx = round16(rows);
  const int l16 = (l + 15) / 16 * 16;
  const int S = 2 * slices;
  if ((size_t)ldx * S * l16 > MW.xcat_elems * sizeof(__nv_bfloat16)) return RSVD_ERR_WORKSPACE;
  uint8_t* x8 = reinterpret_cast<uint8_t*>(MW.xcat);
  const int chunk = mx8_chunk_rows(ax, m, n, l, S);
  if (!chunk) return RSVD_ERR_UNSUPPORTED;
  int rc = launch_split_e4m3(X, rows, l, ldxf, S, chunk, x8, ldx, MW.xexp, MW.colscale,
                             MW.colbits, P->stream);
  if (rc) return rc;
  Mx8Call c;
  c.ax = ax;
  c.A = A;
  c.m = m;
  c.n = n;
  c.lda = lda;
  c.scales = P->scales;
  c.lds = P->lds;
  c.X = x8;
  c.ldx = ldx;
  c.xexp = MW.xexp;
  c.colscale = MW.colscale;
  c.chunk = chunk;
  c.slices = S;
  c.l = l;
  c.out = out;
  c.ldo = ldo;
  c.part = MW.apart;
  c.part_floats = MW.apart_floats;
  c.accumulate = accumulate;
  c.wait_cycles = P->wait_cycles;
  return launch_apass_mx8(c, P->num_sms, &dstatus(P)->flags, P->stream);
}

// One tcgen05 pass: out = A X (ax) or A^T X with X = `slices`-way BF16 split of
// the FP32 operand (rows x l, ld rows).
int mixed_pass_ld(rsvd_plan_t P, bool ax, const void* A, int64_t m, int64_t n, int64_t lda,
                  const float* X, int64_t ldxf, int l, int slices, float* out, int64_t ldo) {
  if (P->dtype == RSVD_FP8E4M3)
    return mx8_pass(P, ax, A, m, n, lda, X, ldxf, l, slices, out, ldo, false);
  MixedWork MW = mixed_work_of(P);
  const int64_t rows = ax ? n : m;
  const int64_t ldx = round8(rows);
  const int l16 = (l + 15) / 16 * 16;
  if ((size_t)ldx * slices * l16 > MW.xcat_elems) return RSVD_ERR_WORKSPACE;
  int rc = split_operand(P, X, rows, l, ldxf, slices, l16, MW.xcat, ldx);
  if (rc) return rc;
  ApassCall c;
  c.ax = ax;
  c.A = A;
  c.m = m;
  c.n = n;
  c.lda = lda;
  c.X = MW.xcat;
  c.ldx = ldx;
  c.x_cols = slices * l16;
  c.l = l;
  c.slices = slices;
  c.slice_stride = l16;
  c.out = out;
  c.ldo = ldo;
  c.part = MW.apart;
  c.part_floats = MW.apart_floats;
  c.fp8 = P->dtype == RSVD_FP8E4M3;
  c.scales = P->scales;
  c.lds = P->lds;
  c.wait_cycles = P->wait_cycles;
  rc = launch_apass_bf16(c, P->num_sms, &dstatus(P)->flags, P->stream);
  if (rc != RSVD_ERR_UNSUPPORTED || slices == 1) return rc;
  // the slices do not fit two shared-memory stages at this l: run the leading
  // slices, then add the last slice's product in a second pass
  c.slices = slices - 1;
  c.x_cols = (slices - 1) * l16;
  if ((rc = launch_apass_bf16(c, P->num_sms, &dstatus(P)->flags, P->stream))) return rc;
  c.slices = 1;
  c.X = MW.xcat + (size_t)(slices - 1) * l16 * ldx;
  c.x_cols = l16;
  c.accumulate = true;
  return launch_apass_bf16(c, P->num_sms, &dstatus(P)->flags, P->stream);
}

int mixed_pass(rsvd_plan_t P, bool ax, const void* A, int64_t m, int64_t n, int64_t lda,
               const float* X, int l, int slices, float* out, int64_t ldo) {
  return mixed_pass_ld(P, ax, A, m, n, lda, X, ax ? n : m, l, slices, out, ldo);
}

}  // namespace

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------

Layout make_layout(int64_t m, int64_t n, int l, int mode, int num_sms, bool f64tc) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t e = mode == RSVD_MODE_PLAIN ? sizeof(double) : sizeof(float);
  const int64_t mn = m > n ? m : n;
  const int lpad = (l + 1) & ~1;
  L.status = take(sizeof(DeviceStatus));
  L.om = take((size_t)n * l * e);
  L.y = take((size_t)m * l * e);
  L.qm = take((size_t)m * l * e);
  L.tmp = take((size_t)mn * l * e);
  L.z = take((size_t)n * l * e);
  L.qb = take((size_t)n * l * e);
  L.part = take((size_t)kPartSplits * mn * l * e);
  L.small_stride = align_up((size_t)l * l * e);
  // G, R1, R1inv, R2, R2inv, Mt, Um, Vm, jacobi work (2 l x lpad), sig, sign, chol work
  L.small = take(L.small_stride * 8 + align_up(2 * (size_t)l * lpad * e) +
                 align_up(2 * (size_t)l * e) +
                 align_up(((size_t)l * l + 33 * (size_t)(l + 64)) * e));
  L.sp = take(L.small_stride * kSinglePassSlots + align_up(kSinglePassVecs * (size_t)l * e));
  L.ad = take((size_t)m * l * e);
  L.refine = take(((size_t)20 * l * l + 8 * (size_t)l) * sizeof(double));
  L.chol64 = take(chol64_work_bytes(l));
  if (mode == RSVD_MODE_MIXED) {
    const int l16 = (l + 15) / 16 * 16;
    // BF16 operand slices (up to three), or up to six E4M3 slices and the
    // chunk exponents of an FP8 plan's operand
    L.om16 = take((size_t)round16(mn) * 3 * l16 * sizeof(__nv_bfloat16) +
                  (size_t)mx8_xexp_count(mn) * sizeof(int) + (size_t)2 * 256 * sizeof(float));
    L.y32 = take(apass_partial_floats(num_sms, l) * sizeof(float));
  }
  if (f64tc) {
    const int64_t lw = (int64_t)kF64tcMaxL;
    L.tc_ncol = (n + 127) / 128 * 128;
    L.tc_ldsl = round8(m);
    L.tc_ldxs = round8(mn);
    L.tc_slices = take((size_t)6 * L.tc_ncol * L.tc_ldsl * 2);
    L.tc_rmax = take(sizeof(int) * (size_t)m);
    L.tc_xs = take((size_t)6 * lw * L.tc_ldxs * 2);
    L.tc_fexp = take(sizeof(int) * (size_t)lw);
    L.tc_rawt = take((size_t)mn * lw * 8);
    L.tc_rawr = take((size_t)mn * lw * 4);
    L.tc_partt = take((size_t)num_sms * 2 * 128 * lw * 8);
    L.tc_partr = take((size_t)num_sms * 2 * 128 * lw * 4);
    L.tc_yncol = ((int64_t)l + 127) / 128 * 128;
    L.tc_ys = take((size_t)6 * L.tc_yncol * L.tc_ldxs * 2);
    L.tc_yrmax = take(sizeof(int) * (size_t)L.tc_ldxs);
  }
  L.total = off;
  return L;
}

template <typename T>
Work<T> work_of(rsvd_plan_t P) {
  Work<T> W;
  char* b = P->ws;
  const Layout& L = P->lay;
  W.om = (T*)(b + L.om);
  W.y = (T*)(b + L.y);
  W.qm = (T*)(b + L.qm);
  W.tmp = (T*)(b + L.tmp);
  W.z = (T*)(b + L.z);
  W.qb = (T*)(b + L.qb);
  W.part = (T*)(b + L.part);
  const int64_t mn = P->m_max > P->n_max ? P->m_max : P->n_max;
  W.part_elems = (size_t)kPartSplits * mn * P->l_max;
  char* s = b + L.small;
  const size_t st = L.small_stride;
  W.G = (T*)(s + 0 * st);
  W.R1 = (T*)(s + 1 * st);
  W.R1i = (T*)(s + 2 * st);
  W.R2 = (T*)(s + 3 * st);
  W.R2i = (T*)(s + 4 * st);
  W.Mt = (T*)(s + 5 * st);
  W.Um = (T*)(s + 6 * st);
  W.Vm = (T*)(s + 7 * st);
  W.jw = (T*)(s + 8 * st);
  const int l = P->l_max, lpad = (l + 1) & ~1;
  const size_t jw_bytes = align_up(2 * (size_t)l * lpad * sizeof(T));
  W.sig = (T*)(s + 8 * st + jw_bytes);
  W.sign = W.sig + l;
  W.cholw = (T*)(s + 8 * st + jw_bytes + align_up(2 * (size_t)l * sizeof(T)));
  return W;
}
template Work<double> work_of<double>(rsvd_plan_t);
template Work<float> work_of<float>(rsvd_plan_t);

MixedWork mixed_work_of(rsvd_plan_t P) {
  MixedWork M;
  const int64_t mn = P->m_max > P->n_max ? P->m_max : P->n_max;
  const int l16 = (P->l_max + 15) / 16 * 16;
  M.xcat = (__nv_bfloat16*)(P->ws + P->lay.om16);
  M.xcat_elems = (size_t)round16(mn) * 3 * l16;
  M.xexp = (int*)(M.xcat + M.xcat_elems);
  M.colscale = (float*)(M.xexp + mx8_xexp_count(mn));
  M.colbits = (unsigned*)(M.colscale + 256);
  M.apart = (float*)(P->ws + P->lay.y32);
  M.apart_floats = apass_partial_floats(P->num_sms, P->l_max);
  return M;
}

DeviceStatus* dstatus(rsvd_plan_t P) { return (DeviceStatus*)(P->ws + P->lay.status); }

bool plan_ready(rsvd_plan_t P) { return P && P->ws && P->ws_bytes >= P->lay.total; }

// ---------------------------------------------------------------------------
// Shared steps
// ---------------------------------------------------------------------------

int f64tc_begin(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda) {
  const Layout& L = P->lay;
  int rc = f64tc_prepare_a(A, m, n, lda, P->ws + L.tc_slices, L.tc_ldsl, L.tc_ncol,
                           (int*)(P->ws + L.tc_rmax), &dstatus(P)->flags, P->num_sms, P->stream);
  if (rc) return rc;
  P->tc_A = A;
  P->tc_m = m;
  P->tc_n = n;
  P->tc_lda = lda;
  return RSVD_OK;
}

namespace {

// C (ldc) = A X (ax) or A^T X for the prepared A, X (ldx) with N columns, on
// the tensor cores.
int f64tc_pass(rsvd_plan_t P, bool ax, const double* X, int64_t ldx, double* C, int64_t ldc,
               int N) {
  const Layout& L = P->lay;
  F64tcCall c;
  c.ax = ax;
  c.slices = P->ws + L.tc_slices;
  c.m = P->tc_m;
  c.n = P->tc_n;
  c.ldsl = L.tc_ldsl;
  c.ncol = L.tc_ncol;
  c.rmax = (const int*)(P->ws + L.tc_rmax);
  c.X = X;
  c.ldx = ldx;
  c.l = N;
  c.out = C;
  c.ldo = ldc;
  c.xslices = P->ws + L.tc_xs;
  c.ldxs = L.tc_ldxs;
  c.fexp = (int*)(P->ws + L.tc_fexp);
  c.raw_t = (int64_t*)(P->ws + L.tc_rawt);
  c.raw_r = (float*)(P->ws + L.tc_rawr);
  c.part_t = (int64_t*)(P->ws + L.tc_partt);
  c.part_r = (float*)(P->ws + L.tc_partr);
  c.wait_cycles = P->wait_cycles;
  return launch_apass_f64tc(c, P->num_sms, &dstatus(P)->flags, P->stream);
}

// The same tensor-core FP64 products with a sample Y (rows x cols, ldy) in
// the role of A, for the CholeskyQR pass inside the power steps: Y's digit
// slices are cut once (f64tc_slice_y), then G = Y^T Y and Q = Y R^-1 are
// passes over them (f64tc_y_pass).  The plan's prepared A is left alone.
int f64tc_slice_y(rsvd_plan_t P, const double* Y, int64_t rows, int cols, int64_t ldy) {
  const Layout& L = P->lay;
  if (rows > L.tc_ldxs || cols > L.tc_yncol) return RSVD_ERR_UNSUPPORTED;
  return f64tc_prepare_a(Y, rows, cols, ldy, P->ws + L.tc_ys, L.tc_ldxs, L.tc_yncol,
                         (int*)(P->ws + L.tc_yrmax), &dstatus(P)->flags, P->num_sms, P->stream);
}
int f64tc_y_pass(rsvd_plan_t P, int64_t rows, int cols, bool ax, const double* X, int64_t ldx,
                 double* C, int64_t ldc, int N) {
  const Layout& L = P->lay;
  F64tcCall c;
  c.ax = ax;
  c.slices = P->ws + L.tc_ys;
  c.m = rows;
  c.n = cols;
  c.ldsl = L.tc_ldxs;
  c.ncol = L.tc_yncol;
  c.rmax = (const int*)(P->ws + L.tc_yrmax);
  c.X = X;
  c.ldx = ldx;
  c.l = N;
  c.out = C;
  c.ldo = ldc;
  c.xslices = P->ws + L.tc_xs;
  c.ldxs = L.tc_ldxs;
  c.fexp = (int*)(P->ws + L.tc_fexp);
  c.raw_t = (int64_t*)(P->ws + L.tc_rawt);
  c.raw_r = (float*)(P->ws + L.tc_rawr);
  c.part_t = (int64_t*)(P->ws + L.tc_partt);
  c.part_r = (float*)(P->ws + L.tc_partr);
  c.wait_cycles = P->wait_cycles;
  return launch_apass_f64tc(c, P->num_sms, &dstatus(P)->flags, P->stream);
}

}  // namespace

template <typename T>
int gemm(rsvd_plan_t P, const T* A, int64_t lda, bool trans, const T* X, int64_t ldx, T* C,
         int64_t ldc, int64_t M, int64_t K, int N, bool x_upper) {
  if constexpr (sizeof(T) == 8) {
    // a pass over the prepared A of an RSVD_MODE_F64_TENSOR plan
    if (P->tc_A && (const void*)A == P->tc_A && lda == P->tc_lda && !x_upper &&
        (trans ? (M == P->tc_n && K == P->tc_m) : (M == P->tc_m && K == P->tc_n)))
      return f64tc_pass(P, !trans, X, ldx, C, ldc, N);
  }
  GemmArgs<T> g{A, lda, trans, X, ldx, C, ldc, M, K, N, x_upper};
  Work<T> W = work_of<T>(P);
  RSVD_CK(launch_gemm<T>(g, W.part, W.part_elems, P->num_sms, P->stream));
  return RSVD_OK;
}

// G (ld l) = Y^T Y for Y rows x l (ldy): upper-triangle Gram kernel, or the
// general product when the kernel does not cover l.
template <typename T>
int gram(rsvd_plan_t P, const T* Y, int64_t ldy, int64_t rows, int l, T* G) {
  if (!gram_supported<T>(l)) return gemm<T>(P, Y, ldy, true, Y, ldy, G, l, l, rows, l);
  Work<T> W = work_of<T>(P);
  RSVD_CK(launch_gram<T>(Y, ldy, rows, l, G, l, W.part, W.part_elems, P->num_sms, P->stream));
  return RSVD_OK;
}
template int gemm<double>(rsvd_plan_t, const double*, int64_t, bool, const double*, int64_t,
                          double*, int64_t, int64_t, int64_t, int, bool);
template int gemm<float>(rsvd_plan_t, const float*, int64_t, bool, const float*, int64_t, float*,
                         int64_t, int64_t, int64_t, int, bool);
template int gram<double>(rsvd_plan_t, const double*, int64_t, int64_t, int, double*);
template int gram<float>(rsvd_plan_t, const float*, int64_t, int64_t, int, float*);

// R and R^-1 of the Gram G (ld l): the FP64 multi-kernel Cholesky for
// l >= 32 on both paths (FP64 arithmetic whatever T is), the one-CTA
// kernels below that or where `fp64` is false (the single CholeskyQR pass
// inside the mixed power steps, whose Q only carries its range forward).
template <typename T>
int chol(rsvd_plan_t P, const T* G, int l, T* R, T* Rinv, bool fp64 = true) {
  const Work<T> W = work_of<T>(P);
  if (l >= 32 && fp64)
    RSVD_CK(launch_chol64<T>(G, l, l, R, Rinv, P->ws + P->lay.chol64, dstatus(P), P->stream));
  else
    RSVD_CK(launch_chol_inv<T>(G, l, l, R, Rinv, W.cholw, dstatus(P), P->stream));
  return RSVD_OK;
}

template <typename T>
int orth(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq, T* Rprod,
         bool transpose_R) {
  Work<T> W = work_of<T>(P);
  DeviceStatus* st = dstatus(P);
  int rc;
  // pass 1: G = Y^T Y = R1^T R1, T1 = Y R1^-1
  if ((rc = gram<T>(P, Y, ldy, rows, l, W.G))) return rc;
  if ((rc = chol<T>(P, W.G, l, W.R1, W.R1i))) return rc;
  if ((rc = gemm<T>(P, Y, ldy, false, W.R1i, l, W.tmp, rows, rows, l, l, true))) return rc;
  // pass 2: G = T1^T T1 = R2^T R2, Q = T1 R2^-1
  if ((rc = gram<T>(P, W.tmp, rows, rows, l, W.G))) return rc;
  if ((rc = chol<T>(P, W.G, l, W.R2, W.R2i))) return rc;
  if (Q && (rc = gemm<T>(P, W.tmp, rows, false, W.R2i, l, Q, ldq, rows, l, l, true))) return rc;
  if (Rprod) RSVD_CK(launch_tri_product<T>(W.R2, W.R1, l, Rprod, transpose_R, P->stream));
  return RSVD_OK;
}
template int orth<double>(rsvd_plan_t, const double*, int64_t, int, int64_t, double*, int64_t,
                          double*, bool);
template int orth<float>(rsvd_plan_t, const float*, int64_t, int, int64_t, float*, int64_t, float*,
                         bool);

// One CholeskyQR pass: Q = Y R^-1 with R the Cholesky factor of Y^T Y.  Q
// spans range(Y) exactly; its columns are orthonormal to about u kappa(Y)^2.
template <typename T>
int orth1(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq) {
  Work<T> W = work_of<T>(P);
  int rc;
  if constexpr (sizeof(T) == 8) {
    // tensor-core FP64 plans: the Gram and Y R^-1 as exact digit-slice
    // products (about 2^-43 relative to the row and column scales; only
    // range(Q) carries forward from this pass)
    if (P->f64tc && l <= kF64tcMaxL) {
      if ((rc = f64tc_slice_y(P, Y, rows, l, ldy))) return rc;
      if ((rc = f64tc_y_pass(P, rows, l, false, Y, ldy, W.G, l, l))) return rc;
      if ((rc = chol<T>(P, W.G, l, W.R1, W.R1i))) return rc;
      return f64tc_y_pass(P, rows, l, true, W.R1i, l, Q, ldq, l);
    }
  }
  if ((rc = gram<T>(P, Y, ldy, rows, l, W.G))) return rc;
  if ((rc = chol<T>(P, W.G, l, W.R1, W.R1i, sizeof(T) == 8))) return rc;
  return gemm<T>(P, Y, ldy, false, W.R1i, l, Q, ldq, rows, l, l, true);
}
template int orth1<float>(rsvd_plan_t, const float*, int64_t, int, int64_t, float*, int64_t);
template int orth1<double>(rsvd_plan_t, const double*, int64_t, int, int64_t, double*, int64_t);

// Shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
// SIAM J. Sci. Comput. 2020): one Cholesky QR of Y with the Gram shifted by
// s = 11 (rows l + l (l+1)) u ||Y||_F^2, which keeps the factorisation defined
// for condition numbers up to about 1/u, then CholeskyQR2 of the result.  Q
// may not alias Y.  Used where the sample is far worse conditioned than the
// power steps of Algorithm 4 leave it (Algorithm 3).
template <typename T>
int orth_shifted(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq) {
  Work<T> W = work_of<T>(P);
  DeviceStatus* st = dstatus(P);
  int rc;
  if ((rc = gram<T>(P, Y, ldy, rows, l, W.G))) return rc;
  const double u = (sizeof(T) == 8) ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
  RSVD_CK(launch_shift_diag<T>(W.G, l, l, 11.0 * ((double)rows * l + (double)l * (l + 1)) * u,
                               P->stream));
  if ((rc = chol<T>(P, W.G, l, W.R1, W.R1i))) return rc;
  if ((rc = gemm<T>(P, Y, ldy, false, W.R1i, l, Q, ldq, rows, l, l, true))) return rc;
  return orth<T>(P, Q, rows, l, ldq, Q, ldq, nullptr, false);
}
template int orth_shifted<double>(rsvd_plan_t, const double*, int64_t, int, int64_t, double*,
                                  int64_t);

// Step 7: the SVD of the l x l factor Mt = R_B^T: W.sig, W.Um (its left
// singular vectors, B's) and Us = Um diag(1 / sig) (ld l), computed to FP64
// accuracy on both paths.
//  * FP64 (plain): a one-sided Jacobi in FP32 with its rotations V32
//    accumulated, V32 made orthogonal in FP64 (Newton-Schulz), then the FP64
//    one-sided Jacobi of Mt V (same left singular vectors and values; its
//    columns are already orthogonal to about 1e-6, so it converges in a few
//    sweeps instead of seven).
//  * FP32 (mixed): the FP32 one-sided Jacobi, then two FP64 refinement steps
//    of (U, sig, V = Mt^T U diag(1/sig)) against the FP64 copy of Mt; sig64
//    receives the FP64 singular values for the output.
// FP64-accurate M = U diag(sig) W^T of an l x l FP64 matrix M (ld l), U (ld
// l) and sig only.  An FP32 one-sided Jacobi, three FP64 Ogita-Aishima
// refinement steps on copies, and the convergence check; when the check
// fails, the FP64 one-sided Jacobi of M V (V the FP32 rotations made
// orthogonal in FP64 by two Newton-Schulz steps) recomputes U and sig (the
// kernel reads the check's flag, so no host round trip).  Scratch: the plan's
// refinement region.
int svd64_u(rsvd_plan_t P, const double* M, int l, double* sig, double* U) {
  const Work<double> W = work_of<double>(P);
  const size_t ll = (size_t)l * l;
  double* d = (double*)(P->ws + P->lay.refine);
  double *M64 = d, *V64 = d + 2 * ll, *work = d + 4 * ll;
  double* s64 = d + 12 * ll;
  float* f = (float*)(d + 12 * ll + l);
  float *M32 = f, *U32 = f + ll, *V32 = f + 2 * ll, *s32 = f + 3 * ll;
  double *Ur = d + 16 * ll, *Vr = d + 17 * ll;
  int* accept = (int*)(d + 18 * ll);
  cudaStream_t st = P->stream;
  DeviceStatus* status = dstatus(P);
  RSVD_CK((launch_convert<double, float>(M, (int64_t)ll, M32, st)));
  RSVD_CK(launch_jacobi_svd<float>(M32, l, l, s32, U32, l, V32, l, nullptr, (float*)W.jw,
                                   status, st));
  RSVD_CK((launch_convert<float, double>(V32, (int64_t)ll, V64, st)));
  // V32 is orthogonal to about 1e-6, which would move sigma(M V) by as much:
  // two Newton-Schulz steps make it orthogonal to FP64 rounding
  RSVD_CK(launch_orthonormalize(V64, l, 2, work, st));
  RSVD_CK(launch_small_product(M, V64, l, M64, st));          // M V
  RSVD_CK((launch_convert<float, double>(U32, (int64_t)ll, Ur, st)));
  RSVD_CK((launch_convert<double, double>(V64, (int64_t)ll, Vr, st)));
  RSVD_CK((launch_convert<float, double>(s32, (int64_t)l, s64, st)));
  RSVD_CK(launch_svd_refine(M, l, Ur, Vr, s64, 3, 1e-6, work, st));
  RSVD_CK(launch_svd_accept(M, l, Ur, Vr, s64, work, accept, st));
  RSVD_CK((launch_convert<double, double>(s64, (int64_t)l, sig, st)));
  RSVD_CK((launch_convert<double, double>(Ur, (int64_t)ll, U, st)));
  RSVD_CK(launch_jacobi_svd<double>(M64, l, l, sig, U, l, nullptr, l, nullptr, W.jw, status, st,
                                    accept));
  return RSVD_OK;
}

template <typename T>
int small_svd_fp64(rsvd_plan_t P, const Work<T>& W, int l, T* us_inv, double* sig64) {
  const size_t ll = (size_t)l * l;
  double* d = (double*)(P->ws + P->lay.refine);
  double *M64 = d, *U64 = d + ll, *V64 = d + 2 * ll, *Us64 = d + 3 * ll, *work = d + 4 * ll;
  double* s64 = d + 12 * ll;
  float* f = (float*)(d + 12 * ll + l);
  float *M32 = f, *U32 = f + ll, *V32 = f + 2 * ll, *s32 = f + 3 * ll;
  cudaStream_t st = P->stream;
  DeviceStatus* status = dstatus(P);
  if constexpr (sizeof(T) == 8) {
    if (int rc = svd64_u(P, W.Mt, l, W.sig, W.Um)) return rc;
    RSVD_CK(launch_scale_cols(W.Um, W.sig, l, us_inv, st));
    (void)M64;
    (void)U64;
    (void)V64;
    (void)Us64;
    (void)work;
    (void)sig64;
    (void)M32;
    (void)U32;
    (void)V32;
    (void)s32;
    (void)status;
  } else {
    RSVD_CK(launch_jacobi_svd<float>(W.Mt, l, l, W.sig, W.Um, l, nullptr, l, nullptr, W.jw,
                                     status, st));
    RSVD_CK((launch_convert<float, double>(W.Mt, (int64_t)ll, M64, st)));
    RSVD_CK((launch_convert<float, double>(W.Um, (int64_t)ll, U64, st)));
    RSVD_CK((launch_convert<float, double>(W.sig, (int64_t)l, s64, st)));
    RSVD_CK(launch_scale_cols(U64, s64, l, Us64, st));
    RSVD_CK(launch_right_vectors(M64, Us64, l, V64, st));
    RSVD_CK(launch_svd_refine(M64, l, U64, V64, s64, 2, 1e-6, work, st));
    RSVD_CK(launch_scale_cols(U64, s64, l, Us64, st));
    RSVD_CK((launch_convert<double, float>(U64, (int64_t)ll, W.Um, st)));
    RSVD_CK((launch_convert<double, float>(Us64, (int64_t)ll, us_inv, st)));
    RSVD_CK((launch_convert<double, float>(s64, (int64_t)l, W.sig, st)));
    if (sig64) RSVD_CK((launch_convert<double, double>(s64, (int64_t)l, sig64, st)));
    (void)M32;
    (void)U32;
    (void)V32;
    (void)s32;
  }
  return RSVD_OK;
}

template <typename T>
int finish(rsvd_plan_t P, const Work<T>& W, int64_t m, int64_t n, int l, int k, T* U, int64_t ldu,
           double* S, T* VT, int64_t ldvt) {
  int rc;
  // B^T (in W.z) = Q_B R_B: only R_B is formed; Mt = R_B^T
  if ((rc = orth<T>(P, W.z, n, l, n, nullptr, n, W.Mt, true))) return rc;
  // R_B^T = U~ Sigma V_R^T; U~ are B's left singular vectors
  T* us_inv = W.Vm;
  double* s_fp64 = (double*)(P->ws + P->lay.refine) + 15 * (size_t)l * l;   // past the scratch
  if ((rc = small_svd_fp64<T>(P, W, l, us_inv, sizeof(T) == 4 ? s_fp64 : nullptr))) return rc;
  // step 8: U = Q U~ (first k columns)
  if ((rc = gemm<T>(P, W.qm, m, false, W.Um, l, U, ldu, m, l, k))) return rc;
  // V_k = B^T U~_k Sigma_k^-1, then one CholeskyQR pass restores orthonormality
  // to rounding (the product carries relative errors ~ eps sigma_1/sigma_i)
  if ((rc = gemm<T>(P, W.z, n, false, us_inv, l, W.tmp, n, n, l, k))) return rc;
  if ((rc = gram<T>(P, W.tmp, n, n, k, W.G))) return rc;
  if ((rc = chol<T>(P, W.G, k, W.R1, W.R1i))) return rc;
  if ((rc = gemm<T>(P, W.tmp, n, false, W.R1i, k, W.qb, n, n, k, k, true))) return rc;
  RSVD_CK(launch_finalize<T>(U, m, ldu, k, W.qb, n, VT, ldvt, W.sig, S, W.sign, P->stream));
  // the mixed path reports the FP64 singular values of the refined small SVD
  if (sizeof(T) == 4) RSVD_CK((launch_convert<double, double>(s_fp64, (int64_t)k, S, P->stream)));
  return RSVD_OK;
}

template int finish<double>(rsvd_plan_t, const Work<double>&, int64_t, int64_t, int, int,
                           double*, int64_t, double*, double*, int64_t);

// ---------------------------------------------------------------------------
// Full solves
// ---------------------------------------------------------------------------

int solve_plain_alg3(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k,
                     int p, int q, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                     int64_t ldvt) {
  const int l = k + p;
  Work<double> W = work_of<double>(P);
  int rc;
  // Algorithm 3 (Section 3.2): 1. Omega;  2. Y = A Omega;  3-4. q times
  // Z = A^T Y, Y = A Z, with no orthonormalisation in between;  5. Q = orth(Y)
  RSVD_CK(launch_gaussian(n, l, seed, 0u, RSVD_F64, W.om, n, P->stream));
  if ((rc = gemm<double>(P, A, lda, false, W.om, n, W.y, m, m, n, l))) return rc;
  for (int j = 0; j < q; ++j) {
    if ((rc = gemm<double>(P, A, lda, true, W.y, m, W.z, n, n, m, l))) return rc;
    if ((rc = gemm<double>(P, A, lda, false, W.z, n, W.y, m, m, n, l))) return rc;
  }
  if ((rc = orth_shifted<double>(P, W.y, m, l, m, W.qm, m))) return rc;
  // 6. B^T = A^T Q;  7-8. small SVD and lift
  if ((rc = gemm<double>(P, A, lda, true, W.qm, m, W.z, n, n, m, l))) return rc;
  return finish<double>(P, W, m, n, l, k, U, ldu, S, VT, ldvt);
}

int solve_plain(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                int q, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                int64_t ldvt) {
  const int l = k + p;
  Work<double> W = work_of<double>(P);
  int rc;
  // 1. Omega;  2. Y = A Omega;  3. Q = orth(Y)
  // Only range(Q) carries into the next product, so inside the power steps
  // one CholeskyQR pass is enough (columns orthonormal to u kappa(Y)^2, the
  // range exact; it breaks down only past kappa ~ 1e8); the Q that B is
  // formed from (after the last power step) takes CholeskyQR2.
  RSVD_CK(launch_gaussian(n, l, seed, 0u, RSVD_F64, W.om, n, P->stream));
  if ((rc = gemm<double>(P, A, lda, false, W.om, n, W.y, m, m, n, l))) return rc;
  if (q == 0) {
    if ((rc = orth<double>(P, W.y, m, l, m, W.qm, m, nullptr, false))) return rc;
  } else if ((rc = orth1<double>(P, W.y, m, l, m, W.qm, m))) {
    return rc;
  }
  // 4-5. power steps with orthonormalisation: W = orth(A^T Q), Q = orth(A W)
  for (int j = 0; j < q; ++j) {
    if ((rc = gemm<double>(P, A, lda, true, W.qm, m, W.z, n, n, m, l))) return rc;
    if ((rc = orth1<double>(P, W.z, n, l, n, W.om, n))) return rc;
    if ((rc = gemm<double>(P, A, lda, false, W.om, n, W.y, m, m, n, l))) return rc;
    if (j == q - 1) {
      if ((rc = orth<double>(P, W.y, m, l, m, W.qm, m, nullptr, false))) return rc;
    } else if ((rc = orth1<double>(P, W.y, m, l, m, W.qm, m))) {
      return rc;
    }
  }
  // 6. B^T = A^T Q;  7-8. small SVD and lift
  if ((rc = gemm<double>(P, A, lda, true, W.qm, m, W.z, n, n, m, l))) return rc;
  return finish<double>(P, W, m, n, l, k, U, ldu, S, VT, ldvt);
}

int solve_mixed(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                int q, uint64_t seed, float* U, int64_t ldu, double* S, float* VT,
                int64_t ldvt) {
  const int l = k + p;
  Work<float> W = work_of<float>(P);
  int rc;
  // 1. Omega (FP32, rounded to BF16 for the pass);  2. Y = A Omega;  3. Q = orth(Y)
  // Inside the power steps only range(Q) matters to the next product, and the
  // product rounds Q to BF16 (relative 2^-9) before using it, so one
  // CholeskyQR pass (orthonormal to u kappa^2) is enough there; the Q that B
  // and U are formed from takes two passes.
  RSVD_CK(launch_gaussian(n, l, seed, 0u, kOutF32Fast, W.om, n, P->stream));
  if ((rc = mixed_pass(P, true, A, m, n, lda, W.om, l, 1, W.y, m))) return rc;
  if ((rc = orth1<float>(P, W.y, m, l, m, W.qm, m))) return rc;
  // 4-5. q power steps on a BF16 operand, then one refinement step on bf16x2
  for (int j = 0; j <= q; ++j) {
    const int slices = (j == q) ? 2 : 1;
    if ((rc = mixed_pass(P, false, A, m, n, lda, W.qm, l, slices, W.z, n))) return rc;
    if ((rc = orth1<float>(P, W.z, n, l, n, W.om, n))) return rc;
    if ((rc = mixed_pass(P, true, A, m, n, lda, W.om, l, slices, W.y, m))) return rc;
    if (j < q) {
      if ((rc = orth1<float>(P, W.y, m, l, m, W.qm, m))) return rc;
    } else if ((rc = orth<float>(P, W.y, m, l, m, W.qm, m, nullptr, false))) {
      return rc;
    }
  }
  // 6. B^T = A^T Q with Q split in three BF16 slices;  7-8. small SVD and lift
  if ((rc = mixed_pass(P, false, A, m, n, lda, W.qm, l, 3, W.z, n))) return rc;
  return finish<float>(P, W, m, n, l, k, U, ldu, S, VT, ldvt);
}

int mixed_apply(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda, const void* X,
                int64_t ldx, int l, float* out, int64_t ldo, bool trans) {
  MixedWork MW = mixed_work_of(P);
  const int l16 = (l + 15) / 16 * 16;
  ApassCall c;
  c.ax = !trans;
  c.A = A;
  c.m = m;
  c.n = n;
  c.lda = lda;
  c.X = X;
  c.ldx = ldx;
  c.x_cols = l;
  c.l = l;
  c.slices = 1;
  c.slice_stride = l16;
  c.out = out;
  c.ldo = ldo;
  c.part = MW.apart;
  c.part_floats = MW.apart_floats;
  c.fp8 = P->dtype == RSVD_FP8E4M3;
  c.scales = P->scales;
  c.lds = P->lds;
  c.wait_cycles = P->wait_cycles;
  return launch_apass_bf16(c, P->num_sms, &dstatus(P)->flags, P->stream);
}

int mixed_apply_split(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda,
                      const float* X, int64_t ldx, int l, int slices, float* out, int64_t ldo,
                      bool trans) {
  return mixed_pass_ld(P, !trans, A, m, n, lda, X, ldx, l, slices, out, ldo);
}

}  // namespace rsvd
