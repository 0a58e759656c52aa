// The l x l steps of the path (l = k + p <= 288), in FP64 (plain path) or
// FP32 (mixed path):
//
//  * chol_inv: Cholesky factor R of the Gram matrix G = Y^T Y and its inverse,
//    the middle of CholeskyQR (Q = Y R^-1), used for every orth() of
//    Algorithm 4 (steps 3 and 5, Section 3.3).  Columns whose Gram pivot falls
//    below l * eps * max(diag G) are numerically in the span of the earlier
//    ones; they are dropped (zero row of R, zero row and column of R^-1), so
//    the matching column of Q is exactly zero and contributes nothing to
//    B = Q^T A.  This keeps exactly rank-deficient samples (rank(A) < k + p)
//    well defined.
//  * tri_product: R = R2 R1 (the R factor of CholeskyQR2), optionally
//    transposed.
//  * jacobi_svd: one-sided (Hestenes) Jacobi SVD of an l x l matrix, step 7 of
//    Algorithm 4 applied to R_B^T where B^T = Q_B R_B; round-robin pair
//    ordering, one warp per column pair, Rutishauser's rotation formulas.
//  * finalize: the sign convention and the output layout of step 8.
//
// Each runs as one CTA: the whole problem is O(l^3) work, which fits in
// one SM's L1/shared memory and needs a block-wide barrier per elimination
// step or Jacobi round.
#include <algorithm>

#include "small_body.cuh"

namespace rsvd {
namespace {

using namespace dense;

template <typename T>
__global__ void tri_product_kernel(const T* __restrict__ R2, const T* __restrict__ R1,
                                   int l, T* __restrict__ out, int transpose_out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < l * l; t += gridDim.x * blockDim.x) {
    int i = t % l, j = t / l;
    T s = 0.0;
    if (i <= j)
      for (int u = i; u <= j; ++u) s = fma(R2[i + u * l], R1[u + j * l], s);
    if (transpose_out) out[j + i * l] = s;
    else out[t] = s;
  }
}

template <typename T>
__global__ void vt_kernel(const T* __restrict__ Vk, int64_t n, int k,
                          const T* __restrict__ sign, T* __restrict__ VT, int64_t ldvt,
                          const T* __restrict__ sig, double* __restrict__ S) {
  // VT (k x n): VT[i + j*ldvt] = sign[i] * Vk[j + i*n]
  const int64_t total = n * (int64_t)k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = t / k;
    int i = (int)(t - j * k);
    VT[i + j * ldvt] = sign[i] * Vk[j + (int64_t)i * n];
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) S[i] = (double)sig[i];
}

template <typename T>
__global__ void __launch_bounds__(CHOL_THREADS)
chol_inv_kernel(const T* __restrict__ G, int64_t ldg, int l, T* __restrict__ R,
                T* __restrict__ Rinv, T* __restrict__ gwork, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* W = gwork ? gwork : reinterpret_cast<T*>(smem_raw);
  chol_inv_blocked<T, CholPanel<T>::value>(G, ldg, l, R, Rinv, W, status);
}

template <typename T>
__global__ void __launch_bounds__(CHOL_THREADS)
chol_inv_panels_kernel(const T* __restrict__ G, int64_t ldg, int l, T* __restrict__ R,
                       T* __restrict__ Rinv, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char cpan_raw[];
  chol_inv_panels<T>(G, ldg, l, R, Rinv, reinterpret_cast<T*>(cpan_raw), status);
}

template <int E>
__global__ void __launch_bounds__(CHOL_REG_THREADS)
chol_inv_regs_kernel(const float* __restrict__ G, int64_t ldg, int l, float* __restrict__ R,
                     float* __restrict__ Rinv, DeviceStatus* status) {
  chol_inv_regs<E>(G, ldg, l, R, Rinv, status);
}

template <typename T>
__global__ void __launch_bounds__(JACOBI_THREADS)
jacobi_svd_kernel(const T* __restrict__ M, int l, int64_t ldm, T* __restrict__ sig,
                  T* __restrict__ Um, int64_t ldu, T* __restrict__ Vm, int64_t ldv,
                  T* __restrict__ UsInv, T* __restrict__ gwork, int use_smem,
                  DeviceStatus* status, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char jsm_raw[];
  T* Wm = use_smem ? reinterpret_cast<T*>(jsm_raw) : gwork;
  jacobi_body<T>(M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv, Wm, jacobi_ld<T>(l, use_smem != 0),
                 status);
}

// FP32, 80 < l <= 160: eight threads per column pair fixed at compile time
__global__ void __launch_bounds__(JACOBI_THREADS)
jacobi_svd_g8_kernel(const float* __restrict__ M, int l, int64_t ldm, float* __restrict__ sig,
                     float* __restrict__ Um, int64_t ldu, float* __restrict__ Vm, int64_t ldv,
                     float* __restrict__ UsInv, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char jg8_raw[];
  jacobi_body<float, JacobiRegs<float>::value, 8>(M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv,
                                                  reinterpret_cast<float*>(jg8_raw),
                                                  jacobi_ld<float>(l, true), status);
}

// FP32, 40 < l <= 80: sixteen threads per column pair fixed at compile time
__global__ void __launch_bounds__(JACOBI_THREADS)
jacobi_svd_g16_kernel(const float* __restrict__ M, int l, int64_t ldm, float* __restrict__ sig,
                      float* __restrict__ Um, int64_t ldu, float* __restrict__ Vm, int64_t ldv,
                      float* __restrict__ UsInv, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char jg16_raw[];
  jacobi_body<float, 5, 16>(M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv,
                            reinterpret_cast<float*>(jg16_raw), jacobi_ld<float>(l, true), status);
}

template <typename T>
__global__ void __cluster_dims__(JACOBI_CLUSTER, 1, 1) __launch_bounds__(JACOBI_CL_THREADS)
jacobi_cluster_kernel(const T* __restrict__ M, int l, int64_t ldm, T* __restrict__ sig,
                      T* __restrict__ Um, int64_t ldu, T* __restrict__ Vm, int64_t ldv,
                      T* __restrict__ UsInv, DeviceStatus* status, const int* __restrict__ skip) {
  // every CTA of the cluster reads the same flag and leaves before any
  // cluster barrier
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char jcl_raw[];
  jacobi_cluster_body<T>(M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv, reinterpret_cast<T*>(jcl_raw),
                         status);
}

// G_ii += coeff * trace(G): the shift of shifted CholeskyQR (one block).
template <typename T>
__global__ void shift_diag_kernel(T* __restrict__ G, int l, int64_t ldg, double coeff) {
  __shared__ double s_part[32];
  double tr = 0.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) tr += (double)G[i + (int64_t)i * ldg];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = tr;
  __syncthreads();
  double total = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += s_part[w];
  const T s = (T)(coeff * total);
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += blockDim.x) G[i + (int64_t)i * ldg] += s;
}

template <typename T>
__global__ void sign_kernel(T* __restrict__ U, int64_t m, int64_t ldu, T* __restrict__ sign) {
  sign_body<T>(U + (int64_t)blockIdx.x * ldu, m, sign + blockIdx.x);
}

}  // namespace

template <typename T>
cudaError_t launch_chol_inv(const T* G, int64_t ldg, int l, T* R, T* Rinv, T* work,
                            DeviceStatus* status, cudaStream_t st) {
  const size_t smem = chol_work_elems(l) * sizeof(T);
  const size_t pan = chol_panel_elems(l) * sizeof(T);
  // FP32: the panel variant (its one-warp pivot blocks run at the FP32 rate;
  // in FP64 the blocked variant's narrower panels are faster)
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (chol_panels_fit<T>(l) && pan <= dynamic_smem_cap((const void*)chol_inv_panels_kernel<T>)) {
      chol_inv_panels_kernel<T><<<1, CHOL_THREADS, pan, st>>>(G, ldg, l, R, Rinv, status);
      done = true;
    }
  }
  if (done) {
  } else if (chol_in_regs<T>(l)) {
    const float* g = (const float*)G;
    float *r = (float*)R, *ri = (float*)Rinv;
    constexpr int nt = CHOL_REG_THREADS;
    switch (chol_reg_edge(l)) {
      case 1: chol_inv_regs_kernel<1><<<1, nt, 0, st>>>(g, ldg, l, r, ri, status); break;
      case 2: chol_inv_regs_kernel<2><<<1, nt, 0, st>>>(g, ldg, l, r, ri, status); break;
      case 3: chol_inv_regs_kernel<3><<<1, nt, 0, st>>>(g, ldg, l, r, ri, status); break;
      case 4: chol_inv_regs_kernel<4><<<1, nt, 0, st>>>(g, ldg, l, r, ri, status); break;
      default: chol_inv_regs_kernel<5><<<1, nt, 0, st>>>(g, ldg, l, r, ri, status);
    }
  } else if (smem <= dynamic_smem_cap((const void*)chol_inv_kernel<T>))
    chol_inv_kernel<T><<<1, CHOL_THREADS, smem, st>>>(G, ldg, l, R, Rinv, nullptr, status);
  else
    chol_inv_kernel<T><<<1, CHOL_THREADS, 0, st>>>(G, ldg, l, R, Rinv, work, status);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_shift_diag(T* G, int l, int64_t ldg, double coeff, cudaStream_t st) {
  shift_diag_kernel<T><<<1, 256, 0, st>>>(G, l, ldg, coeff);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tri_product(const T* R2, const T* R1, int l, T* out, bool transpose_out,
                               cudaStream_t st) {
  int total = l * l;
  tri_product_kernel<T><<<(total + 255) / 256, 256, 0, st>>>(R2, R1, l, out,
                                                             transpose_out ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_svd(const T* M, int l, int64_t ldm, T* sig, T* Um, int64_t ldu, T* Vm,
                              int64_t ldv, T* UsInv, T* work, DeviceStatus* status,
                              cudaStream_t st, const int* skip) {
  if (sizeof(T) == 4) skip = nullptr;
  // FP64, l >= 24: the cluster version (rows over JACOBI_CLUSTER SMs), as one
  // SM's FP64 pipe (2 FMA per clock) bounds the one-CTA kernel; measured
  // 3.9 ms against 6.7 ms at l = 80.  FP32 (and small l) stay on one CTA: a
  // cluster round's barrier and remote stores (~1.3k clocks) cost as much as
  // the one-CTA round itself.
  if (sizeof(T) == 8 && l >= 24) {
    const size_t cneed = jacobi_cluster_elems(l, Vm != nullptr) * sizeof(T);
    if (cneed <= dynamic_smem_cap((const void*)jacobi_cluster_kernel<T>)) {
      jacobi_cluster_kernel<T><<<JACOBI_CLUSTER, JACOBI_CL_THREADS, cneed, st>>>(
          M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv, status, skip);
      note_launch();
      return cudaGetLastError();
    }
  }
  const int twoP = (l + 1) & ~1;
  const size_t need = (size_t)(Vm ? 2 : 1) * jacobi_ld<T>(l, true) * twoP * sizeof(T);
  if constexpr (sizeof(T) == 4) {
    if (jacobi_group(l) == 8 && (l + 7) / 8 <= JacobiRegs<float>::value &&
        need <= dynamic_smem_cap((const void*)jacobi_svd_g8_kernel)) {
      jacobi_svd_g8_kernel<<<1, JACOBI_THREADS, need, st>>>(M, l, ldm, sig, Um, ldu, Vm, ldv,
                                                            UsInv, status);
      note_launch();
      return cudaGetLastError();
    }
    if (jacobi_group(l) == 16 && (l + 15) / 16 <= 5 &&
        need <= dynamic_smem_cap((const void*)jacobi_svd_g16_kernel)) {
      jacobi_svd_g16_kernel<<<1, JACOBI_THREADS, need, st>>>(M, l, ldm, sig, Um, ldu, Vm, ldv,
                                                             UsInv, status);
      note_launch();
      return cudaGetLastError();
    }
  }
  const bool smem = need <= dynamic_smem_cap((const void*)jacobi_svd_kernel<T>);
  jacobi_svd_kernel<T><<<1, JACOBI_THREADS, smem ? need : 0, st>>>(
      M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv, work, smem ? 1 : 0, status, skip);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(T* U, int64_t m, int64_t ldu, int k, const T* Vk, int64_t n, T* VT,
                            int64_t ldvt, const T* sig, double* S, T* sign_work,
                            cudaStream_t st) {
  sign_kernel<T><<<k, 1024, 0, st>>>(U, m, ldu, sign_work);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t total = n * (int64_t)k;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  vt_kernel<T><<<blocks, 256, 0, st>>>(Vk, n, k, sign_work, VT, ldvt, sig, S);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sign_columns(T* U, int64_t m, int64_t ldu, int k, T* sign_work,
                                cudaStream_t st) {
  sign_kernel<T><<<k, 1024, 0, st>>>(U, m, ldu, sign_work);
  note_launch();
  return cudaGetLastError();
}

#define RSVD_INSTANTIATE_SMALL(T)                                                              \
  template cudaError_t launch_chol_inv<T>(const T*, int64_t, int, T*, T*, T*, DeviceStatus*,   \
                                          cudaStream_t);                                       \
  template cudaError_t launch_tri_product<T>(const T*, const T*, int, T*, bool, cudaStream_t); \
  template cudaError_t launch_shift_diag<T>(T*, int, int64_t, double, cudaStream_t);           \
  template cudaError_t launch_jacobi_svd<T>(const T*, int, int64_t, T*, T*, int64_t, T*,       \
                                            int64_t, T*, T*, DeviceStatus*, cudaStream_t,      \
                                            const int*);                                       \
  template cudaError_t launch_finalize<T>(T*, int64_t, int64_t, int, const T*, int64_t, T*,    \
                                          int64_t, const T*, double*, T*, cudaStream_t);       \
  template cudaError_t launch_sign_columns<T>(T*, int64_t, int64_t, int, T*, cudaStream_t);
RSVD_INSTANTIATE_SMALL(double)
RSVD_INSTANTIATE_SMALL(float)

}  // namespace rsvd
