// Host-side orchestration of Algorithm 4 (Section 3.3): workspace views and
// the steps shared by the plain (FP64) and mixed (BF16 A, FP32 elsewhere)
// paths.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace rsvd {

#define RSVD_CK(expr)                               \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;    \
  } while (0)

constexpr int kPartSplits = 16;  // SIMT split-K partial slices held in workspace
constexpr int kSinglePassSlots = 24;  // l x l matrices of the single-pass solve
constexpr int kSinglePassVecs = 8;    // l-vectors of the single-pass solve

// Views of the workspace for the element type T of the path (double for the
// plain path, float for the mixed path).
template <typename T>
struct Work {
  T *om, *y, *qm, *tmp, *z, *qb;  // n x l, m x l, m x l, max(m,n) x l, n x l, n x l
  T* part;                        // SIMT split-K partials
  size_t part_elems;
  T *G, *R1, *R1i, *R2, *R2i, *Mt, *Um, *Vm, *cholw, *jw, *sig, *sign;
};

// Mixed-path extras: the BF16 operand (up to three slices side by side) and
// the partial slots of the tcgen05 passes.
struct MixedWork {
  __nv_bfloat16* xcat;      // also the E4M3 slices of an FP8 plan's operand
  size_t xcat_elems;
  int* xexp;                // FP8: exponent of each 64-row chunk of the operand
  float* colscale;          // FP8: power-of-two column scales of the operand (256)
  unsigned* colbits;        // FP8: column maxima scratch (256)
  float* apart;
  size_t apart_floats;
};

Layout make_layout(int64_t m, int64_t n, int l, int mode, int num_sms, bool f64tc = false);
// RSVD_MODE_F64_TENSOR: builds A's digit slices and marks A as the matrix
// whose passes run on the tensor cores until f64tc_end().
int f64tc_begin(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda);
inline void f64tc_end(rsvd_plan_t P) { P->tc_A = nullptr; }
template <typename T>
Work<T> work_of(rsvd_plan_t P);
MixedWork mixed_work_of(rsvd_plan_t P);
// FP64-accurate SVD M = U diag(sig) W^T of an l x l FP64 matrix (ld l): U (ld
// l) and sig, from an FP32 Jacobi refined in FP64 and checked, with the FP64
// Jacobi as the fallback (pipeline.cu).  Uses the plan's refinement scratch.
int svd64_u(rsvd_plan_t P, const double* M, int l, double* sig, double* U);
DeviceStatus* dstatus(rsvd_plan_t P);
bool plan_ready(rsvd_plan_t P);

// C = op(A) X on the CUDA cores (see GemmArgs); x_upper: X is upper triangular.
template <typename T>
int gemm(rsvd_plan_t P, const T* A, int64_t lda, bool trans, const T* X, int64_t ldx, T* C,
         int64_t ldc, int64_t M, int64_t K, int N, bool x_upper = false);

// G (l x l, ld l) = Y^T Y, both triangles.
template <typename T>
int gram(rsvd_plan_t P, const T* Y, int64_t ldy, int64_t rows, int l, T* G);

// CholeskyQR2: Q = orth(Y) (Q may be NULL: only R is formed); Rprod, if
// non-NULL, receives R2 R1 (or its transpose), the R factor of Y = Q R.
template <typename T>
int orth(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq,
         T* Rprod, bool transpose_R);

// One CholeskyQR pass: Q = Y R^-1 (range(Q) = range(Y); columns orthonormal
// to about u kappa(Y)^2).
template <typename T>
int orth1(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq);

// Steps 6-8 after B^T = A^T Q is in W.z and Q in W.qm (m x l): small SVD of
// B, U = Q U~ and V, truncated to k columns, signs and output layout.
template <typename T>
int finish(rsvd_plan_t P, const Work<T>& W, int64_t m, int64_t n, int l, int k, T* U, int64_t ldu,
           double* S, T* VT, int64_t ldvt);

int solve_plain(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                int q, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                int64_t ldvt);
int solve_mixed(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                int q, uint64_t seed, float* U, int64_t ldu, double* S, float* VT, int64_t ldvt);

// Algorithm 3 (power steps without re-orthonormalisation), FP64; the sample
// is orthonormalised once by shifted CholeskyQR3.
int solve_plain_alg3(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k,
                     int p, int q, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                     int64_t ldvt);

// Shifted CholeskyQR3: Q = orth(Y) for ill-conditioned Y (Q must not alias Y).
template <typename T>
int orth_shifted(rsvd_plan_t P, const T* Y, int64_t rows, int l, int64_t ldy, T* Q, int64_t ldq);

// Algorithm 6 (single-pass randomized SVD of a general matrix), FP64.
int solve_singlepass(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k,
                     int p, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                     int64_t ldvt);

// Algorithm 5 (single-pass randomized EVD of a symmetric matrix), FP64:
// U (n x k, ldu) and the eigenvalues D (k, by decreasing magnitude).
int solve_hermitian(rsvd_plan_t P, const double* A, int64_t n, int64_t lda, int k, int p,
                    uint64_t seed, double* U, int64_t ldu, double* D);

// Adaptive randomized range finder (Halko, Martinsson, Tropp 2011, Algorithm
// 4.2), FP64, blocked: Q (ldq) gets rank <= l_cap orthonormal columns.
// Synchronous.  RSVD_OK when the tolerance test passed, RSVD_ERR_NOT_REACHED
// when l_cap columns were reached first.
int range_adaptive(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, double eps,
                   int r, int l_cap, uint64_t seed, double* Q, int64_t ldq, int* rank);
// The adaptive range followed by B = Q^T A, its SVD and U = Q U~ (all columns).
int solve_adaptive(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, double eps,
                   int r, int l_cap, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                   int64_t ldvt, int* rank);

// SRFT test matrix and FastRandRF (Halko, Martinsson, Tropp 2011, Algorithm
// 4.5), FP64.  Complex matrices are planar: m x l complex = real m x 2l
// [Re | Im].  The plan needs l_max >= 2l.
// srft_setup: D's diagonal (d_re, d_im, n each) and R's l coordinates r.
int srft_setup(rsvd_plan_t P, int64_t n, int l, uint64_t seed, double* d_re, double* d_im, int* r);
// Y (m x 2l planar, ldy) = A Omega: by explicit Omega and one real product.
int srft_sketch_dense(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                      const double* d_re, const double* d_im, const int* r, double* Y,
                      int64_t ldy);
// The same product through length-64 FFTs (n a multiple of 64); see srft_fft.cu.
bool srft_fft_supported(int64_t n, int l);
int srft_sketch_fft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                    const double* d_re, const double* d_im, const int* r, double* Y, int64_t ldy);
// The FFT form when n allows it, else the dense form.
int srft_sketch(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                const double* d_re, const double* d_im, const int* r, double* Y, int64_t ldy);
// Complex CholeskyQR2 of planar Y (rows x l complex) through real kernels;
// Q (planar, ldq) may alias Y.
int orth_complex(rsvd_plan_t P, const double* Y, int64_t rows, int l, int64_t ldy, double* Q,
                 int64_t ldq);
int range_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
               uint64_t seed, double* Q, int64_t ldq);
int sketch_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                uint64_t seed, double* Y, int64_t ldy);
// FastRandRF, then the rank-k SVD on the complex basis (Stage B): U (m x 2k
// planar, ldu), S (k), VT (k x 2n planar [Re V^H | Im V^H], ldvt).
int solve_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k, int p,
               uint64_t seed, double* U, int64_t ldu, double* S, double* VT, int64_t ldvt);

// One pass exactly as the mixed solve runs it: the FP32 operand X (ld ldx)
// split into `slices` BF16 slices (BF16 A) or 2 x `slices` E4M3 slices with
// block-scaled MMAs (FP8 A).
int mixed_apply_split(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda,
                      const float* X, int64_t ldx, int l, int slices, float* out, int64_t ldo,
                      bool trans);
// Step entry: one tcgen05 pass with a BF16 operand X (ldx) of `l` columns.
int mixed_apply(rsvd_plan_t P, const void* A, int64_t m, int64_t n, int64_t lda, const void* X,
                int64_t ldx, int l, float* out, int64_t ldo, bool trans);

}  // namespace rsvd
