// Single-pass randomized SVD of a general matrix (Algorithm 6, Section 3.4.2),
// FP64 (plain mode), l = k + p:
//
//   1. Omega_c (n x l, Philox stream 0), Omega_r (m x l, stream 1)
//   2. Y_c = A Omega_c, Y_r = A^T Omega_r        (the only two passes over A)
//   3. Q_c, Q_r: the k dominant left singular vectors of Y_c, Y_r
//   4. C (k x k): least squares of the joint system
//        (Omega_r^T Q_c) C = Y_r^T Q_r,   C (Q_r^T Omega_c) = Q_c^T Y_c
//   5. C = U^ Sigma V^T
//   6. U = Q_c U^, V = Q_r V^
//
// GPU form of the steps:
//  * step 3: Y = Q1 R by CholeskyQR2 (Q1 overwrites Y), R = Ur diag(s) Wr^T by
//    one-sided Jacobi, so the dominant left singular vectors are Q1 Ur_k.
//    Q_c is never formed: every product with it is taken through Q1 and Ur_k.
//  * step 4: with Y = Q1 R and orthonormal Q1,  Y_r^T Q_r = R_r^T Ur_k and
//    (Q_c^T Y_c)^T = R_c^T Uc_k, so only the two (Omega^T Q1) products touch
//    m or n rows.  The least-squares solution of the joint system solves its
//    normal equations  (M^T M) C + C (N N^T) = M^T P + R N^T  (M = Omega_r^T
//    Q_c, P = Y_r^T Q_r, N = Q_r^T Omega_c, R = Q_c^T Y_c), a Sylvester
//    equation with SPD coefficients: with M^T M = Va diag(la) Va^T and
//    N N^T = Vb diag(lb) Vb^T (one-sided Jacobi on each),
//        C = Va [ (Va^T F Vb)_ij / (la_i + lb_j) ] Vb^T.
//  * steps 5-6: one-sided Jacobi on C with the rotations accumulated, then
//    U = Q1c (Uc_k U^) and V = Q1r (Ur_k V^), signs as in Algorithm 4.
#include "pipeline.h"

namespace rsvd {
namespace {

// C (M x N, ldc) = beta C + op(A) op(B), op(A) M x K, op(B) K x N: the small
// dense products of steps 4-6 (dimensions <= RSVD_L_MAX).  32 x 32 output
// tiles, 256 threads, each thread four entries of one row.
template <typename T>
__global__ void small_gemm_kernel(const T* __restrict__ A, int64_t lda, int ta,
                                  const T* __restrict__ B, int64_t ldb, int tb,
                                  T* __restrict__ C, int64_t ldc, int M, int N, int K, int beta) {
  __shared__ T As[32][33];
  __shared__ T Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e & 31, c = e >> 5;
      {   // As[i][t] = op(A)(i0 + i, k0 + t): consecutive threads along A's rows
        const int i = ta ? c : r, t = ta ? r : c;
        const int gi = i0 + i, gt = k0 + t;
        As[i][t] = (gi < M && gt < K) ? (ta ? A[gt + (int64_t)gi * lda] : A[gi + (int64_t)gt * lda])
                                      : T(0);
      }
      {   // Bs[t][j] = op(B)(k0 + t, j0 + j)
        const int t = tb ? c : r, j = tb ? r : c;
        const int gt = k0 + t, gj = j0 + j;
        Bs[t][j] = (gt < K && gj < N) ? (tb ? B[gj + (int64_t)gt * ldb] : B[gt + (int64_t)gj * ldb])
                                      : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const T a = As[tx][t];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(a, Bs[t][ty + 8 * r], acc[r]);
    }
    __syncthreads();
  }
  const int gi = i0 + tx;
  if (gi >= M) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gj = j0 + ty + 8 * r;
    if (gj < N) {
      T* c = C + gi + (int64_t)gj * ldc;
      *c = beta ? *c + acc[r] : acc[r];
    }
  }
}

// G_ij /= (la_i + lb_j)  (k x k, ld k)
template <typename T>
__global__ void sylvester_scale_kernel(T* __restrict__ G, int k, const T* __restrict__ la,
                                       const T* __restrict__ lb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * k) return;
  const int i = t % k, j = t / k;
  G[t] = G[t] / (la[i] + lb[j]);
}

// S = (C + C^T) / 2 (k x k, ld k): the Hermitian part of the solved C.
template <typename T>
__global__ void symmetrise_kernel(const T* __restrict__ C, int k, T* __restrict__ S) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * k) return;
  const int i = t % k, j = t / k;
  S[t] = T(0.5) * (C[i + j * k] + C[j + i * k]);
}

// For a symmetric S = Uh diag(sig) Vh^T (one-sided Jacobi), column j of Uh is
// an eigenvector with eigenvalue sig_j when Uh_j = Vh_j and -sig_j when
// Uh_j = -Vh_j: D_j = sig_j * sign(Uh_j . Vh_j).  One warp per column.
template <typename T>
__global__ void eig_sign_kernel(const T* __restrict__ Uh, const T* __restrict__ Vh, int k,
                                const T* __restrict__ sig, double* __restrict__ D) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= k) return;
  T d = T(0);
  for (int i = lane; i < k; i += 32) d += Uh[i + (int64_t)j * k] * Vh[i + (int64_t)j * k];
#pragma unroll
  for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if (lane == 0) D[j] = (double)(d < T(0) ? -sig[j] : sig[j]);
}

template <typename T>
cudaError_t small_gemm(const T* A, int64_t lda, bool ta, const T* B, int64_t ldb, bool tb, T* C,
                       int64_t ldc, int M, int N, int K, bool accumulate, cudaStream_t st) {
  dim3 grid((M + 31) / 32, (N + 31) / 32);
  small_gemm_kernel<T><<<grid, 256, 0, st>>>(A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, C, ldc, M, N,
                                             K, accumulate ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

int solve_singlepass(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k,
                     int p, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                     int64_t ldvt) {
  using T = double;
  const int l = k + p;
  Work<T> W = work_of<T>(P);
  cudaStream_t st = P->stream;
  DeviceStatus* status = dstatus(P);
  // workspace slots (each l x l, ld as noted) and vectors
  char* base = P->ws + P->lay.sp;
  const size_t ss = P->lay.small_stride;
  auto slot = [&](int i) { return (T*)(base + (size_t)i * ss); };
  T *Rc = slot(0), *Rr = slot(1), *Uc = slot(2), *Ur = slot(3), *E = slot(4), *E2 = slot(5);
  T *Mm = slot(6), *Nt = slot(7), *Pm = slot(8), *Rt = slot(9), *X1 = slot(10), *X2 = slot(11);
  T *F = slot(12), *A1 = slot(13), *B1 = slot(14), *Va = slot(15), *Vb = slot(16);
  T *T1 = slot(17), *G = slot(18), *C = slot(19), *Uh = slot(20), *Vh = slot(21);
  T* vec = slot(kSinglePassSlots);
  T *sc = vec, *sr = vec + l, *la = vec + 2 * l, *lb = vec + 3 * l, *sig = vec + 4 * l;
  int rc;

  // 1-2. Omega_c, Omega_r; Y_c = A Omega_c (in W.y), Y_r = A^T Omega_r (in W.z)
  RSVD_CK(launch_gaussian(n, l, seed, 0u, RSVD_F64, W.om, n, st));
  RSVD_CK(launch_gaussian(m, l, seed, 1u, RSVD_F64, W.qm, m, st));
  if ((rc = gemm<T>(P, A, lda, false, W.om, n, W.y, m, m, n, l))) return rc;
  if ((rc = gemm<T>(P, A, lda, true, W.qm, m, W.z, n, n, m, l))) return rc;
  // 3. Y = Q1 R (Q1 in place of Y), R = Ur diag(s) W^T
  if ((rc = orth<T>(P, W.y, m, l, m, W.y, m, Rc, false))) return rc;
  if ((rc = orth<T>(P, W.z, n, l, n, W.z, n, Rr, false))) return rc;
  if ((rc = svd64_u(P, Rc, l, sc, Uc))) return rc;
  if ((rc = svd64_u(P, Rr, l, sr, Ur))) return rc;
  // 4. the joint least-squares system
  if ((rc = gemm<T>(P, W.qm, m, true, W.y, m, E, l, l, m, l))) return rc;    // Omega_r^T Q1c
  if ((rc = gemm<T>(P, W.om, n, true, W.z, n, E2, l, l, n, l))) return rc;   // Omega_c^T Q1r
  RSVD_CK(small_gemm<T>(E, l, false, Uc, l, false, Mm, l, l, k, l, false, st));   // M = E Uc_k
  RSVD_CK(small_gemm<T>(E2, l, false, Ur, l, false, Nt, l, l, k, l, false, st));  // N^T
  RSVD_CK(small_gemm<T>(Rr, l, true, Ur, l, false, Pm, l, l, k, l, false, st));   // P
  RSVD_CK(small_gemm<T>(Rc, l, true, Uc, l, false, Rt, l, l, k, l, false, st));   // R^T
  RSVD_CK(small_gemm<T>(Mm, l, true, Pm, l, false, F, k, k, k, l, false, st));    // M^T P
  RSVD_CK(small_gemm<T>(Rt, l, true, Nt, l, false, F, k, k, k, l, true, st));     // + R N^T
  RSVD_CK(small_gemm<T>(Mm, l, true, Mm, l, false, A1, k, k, k, l, false, st));   // M^T M
  RSVD_CK(small_gemm<T>(Nt, l, true, Nt, l, false, B1, k, k, k, l, false, st));   // N N^T
  if ((rc = svd64_u(P, A1, k, la, Va))) return rc;
  if ((rc = svd64_u(P, B1, k, lb, Vb))) return rc;
  RSVD_CK(small_gemm<T>(Va, k, true, F, k, false, T1, k, k, k, k, false, st));    // Va^T F
  RSVD_CK(small_gemm<T>(T1, k, false, Vb, k, false, G, k, k, k, k, false, st));   // ... Vb
  sylvester_scale_kernel<T><<<(k * k + 255) / 256, 256, 0, st>>>(G, k, la, lb);
  note_launch();
  RSVD_CK(cudaGetLastError());
  RSVD_CK(small_gemm<T>(Va, k, false, G, k, false, T1, k, k, k, k, false, st));
  RSVD_CK(small_gemm<T>(T1, k, false, Vb, k, true, C, k, k, k, k, false, st));    // C
  // 5. C = U^ diag(sig) V^^T
  RSVD_CK(launch_jacobi_svd<T>(C, k, k, sig, Uh, k, Vh, k, nullptr, W.jw, status, st));
  // 6. U = Q1c (Uc_k U^), V = Q1r (Ur_k V^)
  RSVD_CK(small_gemm<T>(Uc, l, false, Uh, k, false, X1, l, l, k, k, false, st));
  RSVD_CK(small_gemm<T>(Ur, l, false, Vh, k, false, X2, l, l, k, k, false, st));
  if ((rc = gemm<T>(P, W.y, m, false, X1, l, U, ldu, m, l, k))) return rc;
  if ((rc = gemm<T>(P, W.z, n, false, X2, l, W.qb, n, n, l, k))) return rc;
  RSVD_CK(launch_finalize<T>(U, m, ldu, k, W.qb, n, VT, ldvt, sig, S, W.sign, st));
  return RSVD_OK;
}

}  // namespace rsvd

namespace rsvd {

// Algorithm 5 (Section 3.4.1), FP64, A symmetric n x n, l = k + p:
//   1-2. Omega (n x l, Philox stream 0); Y = A Omega       (the only pass over A)
//   3.   Y = Q1 R (CholeskyQR2), R = Ur diag(s) W^T: Q = Q1 Ur_k, the k
//        dominant left singular vectors of Y (never formed)
//   4.   C (k x k) least squares of C N = H with N = Q^T Omega = Ur_k^T (Q1^T
//        Omega) and H = Q^T Y = Ur_k^T R (k x l each): the normal equations
//        C (N N^T) = H N^T, with N N^T = Vb diag(lb) Vb^T (one-sided Jacobi
//        of the SPD matrix), C = (H N^T) Vb diag(1/lb) Vb^T
//   5.   S = (C + C^T)/2 = Uh diag(sig) Vh^T, eigenvalues D_j = +-sig_j
//   6.   U = Q1 (Ur_k Uh), each column's largest-|.| entry made positive
int solve_hermitian(rsvd_plan_t P, const double* A, int64_t n, int64_t lda, int k, int p,
                    uint64_t seed, double* U, int64_t ldu, double* D) {
  using T = double;
  const int l = k + p;
  Work<T> W = work_of<T>(P);
  cudaStream_t st = P->stream;
  DeviceStatus* status = dstatus(P);
  char* base = P->ws + P->lay.sp;
  const size_t ss = P->lay.small_stride;
  auto slot = [&](int i) { return (T*)(base + (size_t)i * ss); };
  T *R = slot(0), *Ur = slot(1), *E = slot(2), *Nt = slot(3), *Ht = slot(4), *F = slot(5);
  T *B1 = slot(6), *Vb = slot(7), *G = slot(8), *C = slot(9), *Cs = slot(10), *Uh = slot(11);
  T *Vh = slot(12), *X1 = slot(13);
  T* vec = slot(kSinglePassSlots);
  T *sr = vec, *la = vec + l, *lb = vec + 2 * l, *sig = vec + 3 * l;
  int rc;

  // 1-2
  RSVD_CK(launch_gaussian(n, l, seed, 0u, RSVD_F64, W.om, n, st));
  if ((rc = gemm<T>(P, A, lda, false, W.om, n, W.y, n, n, n, l))) return rc;
  // 3
  if ((rc = orth<T>(P, W.y, n, l, n, W.y, n, R, false))) return rc;
  if ((rc = svd64_u(P, R, l, sr, Ur))) return rc;
  // 4: E = Omega^T Q1 (l x l); N^T = E Ur_k (l x k); H^T = R^T Ur_k (l x k)
  if ((rc = gemm<T>(P, W.om, n, true, W.y, n, E, l, l, n, l))) return rc;
  RSVD_CK(small_gemm<T>(E, l, false, Ur, l, false, Nt, l, l, k, l, false, st));
  RSVD_CK(small_gemm<T>(R, l, true, Ur, l, false, Ht, l, l, k, l, false, st));
  RSVD_CK(small_gemm<T>(Ht, l, true, Nt, l, false, F, k, k, k, l, false, st));    // H N^T
  RSVD_CK(small_gemm<T>(Nt, l, true, Nt, l, false, B1, k, k, k, l, false, st));   // N N^T
  if ((rc = svd64_u(P, B1, k, lb, Vb))) return rc;
  RSVD_CK(small_gemm<T>(F, k, false, Vb, k, false, G, k, k, k, k, false, st));    // F Vb
  RSVD_CK(cudaMemsetAsync(la, 0, sizeof(T) * (size_t)k, st));
  sylvester_scale_kernel<T><<<(k * k + 255) / 256, 256, 0, st>>>(G, k, la, lb);   // / lb_j
  note_launch();
  RSVD_CK(cudaGetLastError());
  RSVD_CK(small_gemm<T>(G, k, false, Vb, k, true, C, k, k, k, k, false, st));     // C
  // 5
  symmetrise_kernel<T><<<(k * k + 255) / 256, 256, 0, st>>>(C, k, Cs);
  note_launch();
  RSVD_CK(cudaGetLastError());
  RSVD_CK(launch_jacobi_svd<T>(Cs, k, k, sig, Uh, k, Vh, k, nullptr, W.jw, status, st));
  eig_sign_kernel<T><<<(k + 7) / 8, 256, 0, st>>>(Uh, Vh, k, sig, D);
  note_launch();
  RSVD_CK(cudaGetLastError());
  // 6
  RSVD_CK(small_gemm<T>(Ur, l, false, Uh, k, false, X1, l, l, k, k, false, st));
  if ((rc = gemm<T>(P, W.y, n, false, X1, l, U, ldu, n, l, k))) return rc;
  RSVD_CK(launch_sign_columns<T>(U, n, ldu, k, W.sign, st));
  return RSVD_OK;
}

}  // namespace rsvd
