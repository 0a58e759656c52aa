// Internal declarations shared by the library's translation units.
// Not part of the public C ABI (see include/rsvd.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rsvd.h"

namespace rsvd {

// Host-side count of kernel launches made by this library (all launchers
// call note_launch() once per <<<...>>>).
void note_launch();

// Largest dynamic shared memory a launch of kernel `func` may request on the
// current device: the opt-in limit minus the kernel's static shared memory.
// The kernel's attribute is raised to it on first use (cached per device).
size_t dynamic_smem_cap(const void* func);

constexpr int kMaxSplits = 32;      // split-K partial slices kept in workspace
constexpr size_t kAlign = 256;

// Device status word bits live in one int; codes are ORed as (1 << code).
struct DeviceStatus {
  int flags;        // bit (1 << RSVD_ERR_*) set by kernels
  int jacobi_sweeps;
  int deficient;    // number of dropped (deficient) columns in the last orth
  int ad_stop;      // adaptive range finder: accepted columns at the stop, or -1
  int ad_dropped;   // adaptive range finder: first dropped column of the block
  int pad[59];
};

inline int status_from_flags(int flags) {
  // report the most severe code first
  const int order[] = {RSVD_ERR_NONFINITE, RSVD_ERR_TIMEOUT, RSVD_ERR_CHOLESKY, RSVD_ERR_JACOBI};
  for (int c : order)
    if (flags & (1 << c)) return c;
  return RSVD_OK;
}

// Workspace carve-up (offsets in bytes from the workspace base).
struct Layout {
  size_t status, om, y, qm, tmp, z, qb, part, small, total;
  size_t sp;            // l x l slots of the single-pass solve (Algorithm 6)
  size_t ad;            // second m x l sample buffer of the adaptive range finder
  // mixed-mode extras: BF16 operand slices (om16), tcgen05 partial slots (y32)
  size_t om16, y32;
  size_t small_stride;  // bytes of one l x l FP64 matrix (padded)
  size_t refine;        // FP64 / FP32 l x l scratch of the small SVD (step 7)
  size_t chol64;        // scratch of the FP64 multi-kernel Cholesky
  // RSVD_MODE_F64_TENSOR: A's digit slices, row exponents, the operand's
  // slices and exponents, raw outputs and partial slots of the passes
  size_t tc_slices, tc_rmax, tc_xs, tc_fexp, tc_rawt, tc_rawr, tc_partt, tc_partr;
  size_t tc_ys, tc_yrmax;          // digit slices and row exponents of a sample Y (orth)
  int64_t tc_yncol;
  int64_t tc_ncol, tc_ldsl, tc_ldxs;
};

}  // namespace rsvd

namespace rsvd {
struct BatchLayout;
}

struct rsvd_plan_s {
  int64_t m_max, n_max;
  int l_max;
  int dtype, mode;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  rsvd::Layout lay;
  int* h_status;     // pinned host copy of DeviceStatus.flags
  int num_sms;
  // FP8 A (rsvd_set_tile_scales): per-tile scales, tile (I, J) at scales[I + J * lds]
  const float* scales;
  int64_t lds, scale_rows, scale_cols;
  // batch plans (rsvd_batch_plan_create)
  int batched;
  int max_count;
  int64_t rows_total, cols_total;
  rsvd::BatchLayout* batch_lay;   // owned
  void* h_ctx;                    // pinned staging for the context table
  cudaEvent_t ctx_event;          // marks the table copy of the last batched solve
  int batch_engine;               // kBatchSimt or kBatchTensor (FP32 batch plans)
  int batch_graphs;               // rsvd_batch_set_graphs: grouped solves as CUDA graphs
  int batch_sms;                  // rsvd_batch_set_sm_limit: SMs of a grouped tensor launch (0: all)
  void* batch_tc;                 // tensor-engine host state (schedules), owned
  long long wait_cycles;          // rsvd_plan_set_wait_limit (0: the default bound)
  int f64tc;                      // RSVD_MODE_F64_TENSOR (mode holds RSVD_MODE_PLAIN)
  const void* tc_A;               // the A whose slices are current (during a call)
  int64_t tc_m, tc_n, tc_lda;
  int tc_pinned;                  // rsvd_plan_prepare_a: slices kept across calls
};

namespace rsvd {

// ---- kernels' host launchers (all enqueue on `st`) ----

// Omega (n x l) for (seed, stream): FP64, FP32 or BF16 output, each rounded
// from the FP64 value; columns col0 .. col0+l-1 of the generator's matrix.  kOutF32Fast (internal, mixed path): FP32 Box-Muller on
// 24-bit uniforms from the same Philox words (the FP64 transcendental
// functions run at the FP64 rate, 1/64 of FP32 on this GPU).
constexpr int kOutF32 = RSVD_F32;
constexpr int kOutF32Fast = 101;
cudaError_t launch_gaussian(int64_t n, int l, uint64_t seed, uint32_t stream_id,
                            int out_dtype, void* out, int64_t ldo, cudaStream_t st,
                            int64_t col0 = 0);

// Tall-skinny GEMM on the CUDA cores:  C (M x N) = op(A) X,  op(A) = A (M x K,
// lda) or A^T (A stored K x M, lda).  X is K x N (ldx).  Split-K partials go
// to `part` (up to part_elems elements) when more than one split is used.
// x_upper: X is upper triangular (K == N, op(A) = A); column c of the product
// then only contracts over k <= c, so each column tile stops at its last column.
template <typename T>
struct GemmArgs {
  const T* A; int64_t lda; bool trans;
  const T* X; int64_t ldx;
  T* C; int64_t ldc;
  int64_t M, K; int N;
  bool x_upper = false;
};
template <typename T>
cudaError_t launch_gemm(const GemmArgs<T>& g, T* part, size_t part_elems, int num_sms,
                        cudaStream_t st);

// Gram product G = Y^T Y (Y rows x l, ldy) on the CUDA cores, both triangles of
// G (ldg) written; per-CTA partials (l*l elements each, at most num_sms of
// them, bounded by part_elems) go to `part`.  gram_supported(l) tells whether
// this kernel covers l (else use launch_gemm).
template <typename T>
bool gram_supported(int l);
template <typename T>
cudaError_t launch_gram(const T* Y, int64_t ldy, int64_t rows, int l, T* G, int64_t ldg, T* part,
                        size_t part_elems, int num_sms, cudaStream_t st);

// One-CTA Cholesky of the l x l Gram G (ldg) -> upper R (l x l, ld l) and
// its inverse Rinv (ld l); deficient pivots zero the row of R and the row and
// column of Rinv.  Sets status bits on non-finite input.  work: at least
// l*(l+2) elements (used when that does not fit in shared memory).
template <typename T>
cudaError_t launch_chol_inv(const T* G, int64_t ldg, int l, T* R, T* Rinv, T* work,
                            DeviceStatus* status, cudaStream_t st);

// G_ii += coeff * trace(G) for i < l: the diagonal shift of shifted
// CholeskyQR (one block; the trace is summed in FP64).
template <typename T>
cudaError_t launch_shift_diag(T* G, int l, int64_t ldg, double coeff, cudaStream_t st);

// out (l x l, ld l) = R2 * R1 for upper triangular R1, R2 (ld l); if
// transpose_out, out = (R2 R1)^T.
template <typename T>
cudaError_t launch_tri_product(const T* R2, const T* R1, int l, T* out, bool transpose_out,
                               cudaStream_t st);

// One-CTA one-sided Jacobi SVD of the l x l matrix M (ldm): M = Um diag(sig) Vm^T.
// Vm may be NULL (rotations not accumulated); UsInv (ld l), if non-NULL,
// receives Um diag(1/sig).  work holds 2 * l_even * l elements.  skip (device,
// may be NULL): when *skip is nonzero at launch time the kernel returns at
// once and writes nothing (FP64 only).
template <typename T>
cudaError_t launch_jacobi_svd(const T* M, int l, int64_t ldm, T* sig, T* Um, int64_t ldu, T* Vm,
                              int64_t ldv, T* UsInv, T* work, DeviceStatus* status,
                              cudaStream_t st, const int* skip = nullptr);

// Sign convention + outputs of the lift: flips columns of U (m x k, ldu) so
// each column's largest-|.| entry is positive, writes S[i] = sig[i] and
// VT (k x n, ldvt) = diag(sign) Vk^T with Vk n x k (ld n).
template <typename T>
cudaError_t launch_finalize(T* U, int64_t m, int64_t ldu, int k, const T* Vk, int64_t n, T* VT,
                            int64_t ldvt, const T* sig, double* S, T* sign_work, cudaStream_t st);

// Cholesky factor R (upper, G = R^T R) and R^-1 (both l x l, ld l) of the
// Gram G (ldg) in FP64 arithmetic over many SMs (see chol64.cu); work:
// chol64_work_bytes(l).  Dropped pivots and non-finite input as
// launch_chol_inv.
size_t chol64_work_bytes(int l);
template <typename T>
cudaError_t launch_chol64(const T* G, int64_t ldg, int l, T* R, T* Rinv, void* work,
                          DeviceStatus* status, cudaStream_t st);

// FP64 refinement of an approximate SVD M = U diag(s) V^T (all l x l, ld l),
// `steps` steps in place (see svd_refine.cu); work: 8 l^2 doubles.
cudaError_t launch_svd_refine(const double* M, int l, double* U, double* V, double* s, int steps,
                              double cluster_tol, double* work, cudaStream_t st);
// Us = U diag(1/s) (0 where s_i <= 0); V = M^T Us; C = A B (all l x l, ld l, FP64).
// accept = 1 when the refined SVD (U, V, s) of M passes the convergence check
// of svd_refine.cu (U, V orthogonal to 1e-13, U^T M V diagonal to 1e-12 of
// each pair's larger sigma), else 0.  work: 4 l^2 doubles.
cudaError_t launch_svd_accept(const double* M, int l, const double* U, const double* V,
                              const double* s, double* work, int* accept, cudaStream_t st);
cudaError_t launch_scale_cols(const double* U, const double* s, int l, double* Us,
                              cudaStream_t st);
cudaError_t launch_right_vectors(const double* M, const double* Us, int l, double* V,
                                 cudaStream_t st);
cudaError_t launch_small_product(const double* A, const double* B, int l, double* C,
                                 cudaStream_t st);
// V <- V (3 I - V^T V) / 2, `steps` times (work: 2 l^2 doubles).
cudaError_t launch_orthonormalize(double* V, int l, int steps, double* work, cudaStream_t st);
template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* in, int64_t count, Tout* out, cudaStream_t st);

// Flips columns of U (m x k, ldu) so each column's largest-|.| entry is
// positive (lowest index on ties).
template <typename T>
cudaError_t launch_sign_columns(T* U, int64_t m, int64_t ldu, int k, T* sign_work,
                                cudaStream_t st);

}  // namespace rsvd
