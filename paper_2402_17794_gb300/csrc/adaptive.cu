// Adaptive randomized range finder (Adaptive_randRF of the toolbox, Section
// 4; Algorithm 4.2 of Halko, Martinsson and Tropp, SIAM Review 53, 2011),
// FP64, and the rank-revealing SVD built on it.
//
// The published algorithm takes one Gaussian sample at a time: it accepts
// the next sample's component orthogonal to the current basis as a new
// column q_j, and stops at the first j where the residuals
// ||(I - Q_j Q_j^T) A omega_i|| of the next r samples are all at most
// eps / (10 sqrt(2/pi)).  Its q_j are the Gram-Schmidt vectors of the
// samples A omega_1, A omega_2, ... in order, so the result is fixed by the
// samples and the stopping rule, not by the one-vector-at-a-time schedule.
//
// GPU form, a block of b samples per pass over A:
//   1. Y (m x b): the r-1 samples carried over from the previous block,
//      then A Omega for the next b - (r-1) columns of the generator's Omega;
//   2. Y <- (I - Q Q^T) Y against the J accepted columns;
//   3. Y = Q_b R_b by block Gram-Schmidt with re-orthogonalisation (shifted
//      CholeskyQR3 of Y, its Q projected against Q once more, CholeskyQR2;
//      all factors upper triangular, so the columns of Q_b are the
//      Gram-Schmidt vectors of Y in order), and R_b = Q_b^T Y formed
//      directly, accurate to rounding of ||Y||;
//   4. with t columns of the block accepted, the residual of block column
//      i >= t is sqrt(sum_{s=t..i} R_b(s, i)^2); one warp finds the
//      smallest t whose next r residuals are all below the threshold;
//   5. the host reads that t (one wait per block): it accepts t columns and
//      stops, or accepts b - r + 1 columns and carries the other r - 1
//      samples into the next block.
// Blocks hold b = min(64, l_max, l_cap - J + r) samples: no more than
// l_cap - J + r can decide the outcome.
// Every Gaussian column is multiplied by A once.  A block column that
// CholeskyQR drops as numerically dependent (its residual is below about
// 1e-12 of the block's norm) ends the search there: the numerical rank of
// the sample is reached.
#include <algorithm>
#include <cmath>

#include "pipeline.h"

namespace rsvd {
namespace {

constexpr int kBlock = 64;      // samples per block (largest)

// Y -= T (rows x c, both ld ld)
__global__ void subtract_kernel(double* __restrict__ Y, const double* __restrict__ T,
                                int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    Y[t] -= T[t];
}

// Stopping rule of the block (one warp).  R (b x b, ld b) upper triangular.
// Candidate t (0 <= t <= t_max) accepts block columns 0..t-1; it passes
// when the residuals of block columns t..t+r-1 are all <= thr.  Writes the
// smallest passing t (or -1) and the first dropped column (R(s,s) == 0; b
// when none).
__global__ void adaptive_stop_kernel(const double* __restrict__ R, int b, int r, int t_max,
                                     double thr, DeviceStatus* status) {
  const int lane = threadIdx.x;
  int first_pass = 0x7fffffff, first_drop = b;
  for (int t = lane; t < b; t += 32) {
    if (R[t + (int64_t)t * b] == 0.0) first_drop = min(first_drop, t);
    if (t > t_max || t + r > b) continue;
    bool ok = true;
    for (int i = t; i < t + r && ok; ++i) {
      double s = 0.0;
      for (int u = t; u <= i; ++u) s = fma(R[u + (int64_t)i * b], R[u + (int64_t)i * b], s);
      ok = sqrt(s) <= thr;
    }
    if (ok) first_pass = min(first_pass, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    first_pass = min(first_pass, __shfl_xor_sync(0xffffffffu, first_pass, o));
    first_drop = min(first_drop, __shfl_xor_sync(0xffffffffu, first_drop, o));
  }
  if (lane == 0) {
    status->ad_stop = first_pass == 0x7fffffff ? -1 : first_pass;
    status->ad_dropped = first_drop;
  }
}

int subtract(rsvd_plan_t P, double* Y, const double* T, int64_t total) {
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)P->num_sms * 8);
  subtract_kernel<<<blocks, 256, 0, P->stream>>>(Y, T, total);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

// X (m x c, ld m) <- (I - Q Q^T) X for Q's J columns (ldq); C: J x c scratch.
int project_out(rsvd_plan_t P, const double* Q, int64_t ldq, int J, double* X, int64_t m, int c,
                double* C) {
  Work<double> W = work_of<double>(P);
  int rc;
  if ((rc = gemm<double>(P, Q, ldq, true, X, m, C, J, J, m, c))) return rc;
  if ((rc = gemm<double>(P, Q, ldq, false, C, J, W.tmp, m, m, J, c))) return rc;
  return subtract(P, X, W.tmp, m * (int64_t)c);
}

// Columns [0, c) of `src` (ld lds) -> columns [0, c) of `dst` (ld ldd), m rows.
int copy_cols(rsvd_plan_t P, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t m,
              int c) {
  if (c <= 0) return RSVD_OK;
  RSVD_CK(cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), src, (size_t)lds * sizeof(double),
                            (size_t)m * sizeof(double), (size_t)c, cudaMemcpyDeviceToDevice,
                            P->stream));
  return RSVD_OK;
}

}  // namespace

int range_adaptive(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, double eps,
                   int r, int l_cap, uint64_t seed, double* Q, int64_t ldq, int* rank) {
  Work<double> W = work_of<double>(P);
  DeviceStatus* dst = dstatus(P);
  const int b_max = std::min(kBlock, P->l_max);   // callers guarantee r < b_max
  const double thr = eps / (10.0 * std::sqrt(2.0 / 3.14159265358979323846));
  double* Y = W.y;
  double* Y2 = (double*)(P->ws + P->lay.ad);
  double* C = W.Mt;    // J x b projection coefficients (ld J)
  double* Rb = W.Um;   // b x b
  int J = 0, carried = 0, rc;
  int64_t drawn = 0;
  *rank = 0;
  // status bits already set by earlier work on the plan are not this call's
  RSVD_CK(cudaMemcpyAsync(P->h_status, dst, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  RSVD_CK(cudaStreamSynchronize(P->stream));
  const int earlier = P->h_status[0];
  for (;;) {
    // 1. complete the block with fresh samples (no more than l_cap - J + r
    //    columns can matter)
    const int b = std::min(b_max, l_cap - J + r);
    const int fresh = b - carried;
    RSVD_CK(launch_gaussian(n, fresh, seed, 0u, RSVD_F64, W.om, n, P->stream, drawn));
    if ((rc = gemm<double>(P, A, lda, false, W.om, n, Y + (int64_t)carried * m, m, m, n, fresh)))
      return rc;
    drawn += fresh;
    // 2-3. block Gram-Schmidt with re-orthogonalisation against the J
    //      accepted columns: Y <- (I - QQ^T) Y; Y = Q1 R1 (shifted
    //      CholeskyQR3); Q1 <- (I - QQ^T) Q1; Q1 = Q_b R2 (CholeskyQR2).
    //      Projecting the orthonormal Q1 rather than Y a second time keeps
    //      Q_b orthogonal to Q when R1^-1 is large (samples whose residuals
    //      span many orders of magnitude).  Then R_b = Q_b^T Y.
    if (J > 0 && (rc = project_out(P, Q, ldq, J, Y, m, b, C))) return rc;
    if ((rc = orth_shifted<double>(P, Y, m, b, m, Y2, m))) return rc;
    if (J > 0) {
      if ((rc = project_out(P, Q, ldq, J, Y2, m, b, C))) return rc;
      if ((rc = orth<double>(P, Y2, m, b, m, Y2, m, nullptr, false))) return rc;
    }
    if ((rc = gemm<double>(P, Y2, m, true, Y, m, Rb, b, b, m, b))) return rc;
    // 4. the stopping rule, read back on the host
    const int t_max = std::min(b - r, l_cap - J);
    adaptive_stop_kernel<<<1, 32, 0, P->stream>>>(Rb, b, r, t_max, thr, dst);
    note_launch();
    RSVD_CK(cudaGetLastError());
    RSVD_CK(cudaMemcpyAsync(P->h_status, dst, 5 * sizeof(int), cudaMemcpyDeviceToHost,
                            P->stream));
    RSVD_CK(cudaStreamSynchronize(P->stream));
    const int fresh_flags = P->h_status[0] & ~earlier;
    if (status_from_flags(fresh_flags) != RSVD_OK) return status_from_flags(fresh_flags);
    const int stop = P->h_status[3], drop = P->h_status[4];
    // 5. accept, and stop or carry the rest over
    int accept;
    int result = -1;
    if (stop >= 0 && stop <= drop) {
      accept = stop;
      result = RSVD_OK;
    } else if (drop < b && drop <= l_cap - J && drop <= b - r + 1) {
      accept = drop;   // numerical rank of the sample reached
      result = RSVD_OK;
    } else if (l_cap - J <= b - r) {
      accept = l_cap - J;
      result = RSVD_ERR_NOT_REACHED;
    } else {
      accept = b - r + 1;
    }
    if ((rc = copy_cols(P, Q + (int64_t)J * ldq, ldq, Y2, m, m, accept))) return rc;
    J += accept;
    if (result >= 0) {
      *rank = J;
      return result;
    }
    carried = b - accept;
    if ((rc = copy_cols(P, Y2, m, Y + (int64_t)accept * m, m, m, carried))) return rc;
    std::swap(Y, Y2);
  }
}

int solve_adaptive(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, double eps,
                   int r, int l_cap, uint64_t seed, double* U, int64_t ldu, double* S, double* VT,
                   int64_t ldvt, int* rank) {
  Work<double> W = work_of<double>(P);
  int J = 0;
  const int found = range_adaptive(P, A, m, n, lda, eps, r, l_cap, seed, W.qm, m, &J);
  if (found != RSVD_OK && found != RSVD_ERR_NOT_REACHED) return found;
  *rank = J;
  if (J == 0) return found;
  int rc;
  cudaStream_t st = P->stream;
  // B^T = A^T Q (n x J).  Every column is kept, so B's singular values span
  // sigma_1 down to about the tolerance (condition numbers up to ~1/u when
  // eps is small): B^T = Q_B R_B by shifted CholeskyQR3, R_B^T = B Q_B
  // formed directly, and V = Q_B V_J from the Jacobi rotations, with no
  // division by sigma.
  if ((rc = gemm<double>(P, A, lda, true, W.qm, m, W.z, n, n, m, J))) return rc;
  if ((rc = orth_shifted<double>(P, W.z, n, J, n, W.qb, n))) return rc;
  if ((rc = gemm<double>(P, W.z, n, true, W.qb, n, W.Mt, J, J, n, J))) return rc;
  // R_B^T = U~ Sigma V_J^T (one-sided Jacobi with the rotations accumulated)
  RSVD_CK(launch_jacobi_svd<double>(W.Mt, J, J, W.sig, W.Um, J, W.Vm, J, nullptr, W.jw, dstatus(P),
                                    st));
  // U = Q U~, V = Q_B V_J; signs and output layout
  if ((rc = gemm<double>(P, W.qm, m, false, W.Um, J, U, ldu, m, J, J))) return rc;
  if ((rc = gemm<double>(P, W.qb, n, false, W.Vm, J, W.tmp, n, n, J, J))) return rc;
  RSVD_CK(launch_finalize<double>(U, m, ldu, J, W.tmp, n, VT, ldvt, W.sig, S, W.sign, st));
  return found;
}

}  // namespace rsvd
