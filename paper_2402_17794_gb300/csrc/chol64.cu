// Cholesky factor R (G = R^T R) and its inverse of the l x l Gram matrix of
// CholeskyQR (Algorithm 4, steps 3 and 5, Section 3.3), in FP64 arithmetic
// whatever the element type of G, R and R^-1, spread over the GPU.
//
// One SM's FP64 pipe does 2 FMA per clock on this part, so a one-CTA
// factorisation of l = 80 needs at least 60 us and one of l = 288 several
// milliseconds; here every step but the 32 x 32 diagonal blocks runs on
// many SMs.  Right-looking blocked Cholesky with 32-wide panels
// P = [p0, p0 + 32):
//   1. R_PP = chol(G_PP) and X_PP = R_PP^-1 (one CTA);
//   2. the panel row R_PJ = X_PP^T G_PJ for J beyond the panel;
//   3. the trailing update G_JK -= R_PJ^T R_PK (upper triangle);
// then X = R^-1 by block rows from the bottom up:
//   X_IJ = -X_II sum_{I < K <= J} R_IK X_KJ.
// A pivot d_j <= tol (tol = drop * max diag(G)) marks a dependent column: its
// row of R and its row and column of R^-1 are zero, as in the one-CTA
// kernels, and the count goes to DeviceStatus::deficient.  A non-finite
// diagonal raises RSVD_ERR_NONFINITE and zeroes R and R^-1.
#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace rsvd {
namespace {

constexpr int CB = 32;    // panel width
constexpr int TB = 16;    // output tile of the panel-row, update and inverse kernels

struct CholCtl {
  double tol;
  int bad;
  int def;
};

template <typename T>
__global__ void chol64_setup_kernel(const T* __restrict__ G, int64_t ldg, int l, double drop,
                                    double* __restrict__ W, double* __restrict__ R,
                                    double* __restrict__ X, CholCtl* ctl) {
  if (blockIdx.x == 0) {
    __shared__ double s_mx[32];
    __shared__ int s_bad[32];
    double mx = 0.0;
    int bad = 0;
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
      const double d = (double)G[j + (int64_t)j * ldg];
      if (!isfinite(d)) bad = 1;
      mx = fmax(mx, fabs(d));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      s_mx[w] = mx;
      s_bad[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
        mx = fmax(mx, s_mx[i]);
        bad |= s_bad[i];
      }
      ctl->tol = drop * mx;
      ctl->bad = bad;
      ctl->def = 0;
    }
  }
  const int64_t ll = (int64_t)l * l;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ll;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % l), j = (int)(t / l);
    W[t] = i <= j ? (double)G[i + (int64_t)j * ldg] : 0.0;
    R[t] = 0.0;
    X[t] = 0.0;
  }
}

// Step 1 for the panel at p0: the nb x nb diagonal block, by one elimination
// on [G_PP | I] (Gauss without pivoting, stable for an SPD matrix): with
// G_PP = L D L^T, pivot j subtracts (a_ji / d_j) row_j from every row i > j,
// which turns G's upper triangle into D L^T and the identity into L^-1, so
//   R_PP = D^1/2 L^T,  R_PP^-1 = L^-T D^-1/2.
// One 32 x 32 array holds both halves: entry (i, k) is the upper part for
// k >= i and the strict lower part of L^-1 for k < i (unit diagonal
// implicit).  Warp w keeps rows 4w .. 4w+3 in registers, lane k column k.
// For pivot j the warp owning row j publishes the row (a_j) and the row
// times 1/d_j (r_j, with r_jj = 1/d_j for L^-1's unit diagonal) in shared
// memory; every later row i then takes one FMA per entry,
//   e_ik -= a_ji r_jk   for k >= i (upper part) or k <= j (L^-1 part),
// and the owner of row j + 1 forms the next pivot as soon as its own rows
// are updated.  Pivot rows are double-buffered, so each pivot costs one
// barrier; warps whose rows are all above the pivot skip the update.
// On that critical path only 1/d_j is needed: the FP32 reciprocal of d
// scaled into [1, 2), refined by two Newton steps y <- y (2 - d y) in FP64
// (each squares the relative error: about 2^-22 -> 2^-44 -> FP64 rounding).
// The square roots for R and R^-1 (same Newton scheme on 1/sqrt(d),
// y <- y (3 - d y^2) / 2) are formed once, after the elimination.
__device__ __forceinline__ double pow2_of(int e) {   // 2^e, |e| <= 1022
  return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ int exp_of(double d) {    // d normal and positive
  return (int)((__double_as_longlong(d) >> 52) & 0x7FF) - 1023;
}
__device__ __forceinline__ double rcp64(double d) {
  const int e = exp_of(d);
  const double dn = d * pow2_of(-e);                  // [1, 2)
  double y = (double)__frcp_rn((float)dn);
  y = y * fma(-dn, y, 2.0);
  y = y * fma(-dn, y, 2.0);
  return y * pow2_of(-e);
}
__device__ __forceinline__ double rsqrt64(double d) {
  const int h = exp_of(d) >> 1;                        // d 2^-2h in [1, 4)
  const double dn = d * pow2_of(-2 * h);
  double y = (double)rsqrtf((float)dn);
  y = y * fma(-0.5 * dn, y * y, 1.5);
  y = y * fma(-0.5 * dn, y * y, 1.5);
  return y * pow2_of(-h);
}

__global__ void __launch_bounds__(256) chol64_diag_kernel(const double* __restrict__ W, int l,
                                                          int p0, double* __restrict__ R,
                                                          double* __restrict__ X,
                                                          CholCtl* ctl) {
  if (ctl->bad) return;
  __shared__ double pa[2][CB], pr[2][CB];
  __shared__ double s_d[CB], s_rs[CB];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int nb = min(CB, l - p0);
  const double tol = ctl->tol;
  double a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * warp + q;
    a[q] = (i <= k && k < nb) ? W[p0 + i + (int64_t)(p0 + k) * l] : 0.0;
  }
  // the owner of row j (this warp, register q) publishes pivot j; a dropped
  // pivot (d <= tol) publishes a zero scaled row and records d = 0
  auto publish = [&](int j, double v, int buf) {
    double d = __shfl_sync(0xffffffffu, v, j);
    double inv = 0.0;
    if (d > tol && d >= DBL_MIN) {
      inv = rcp64(d);
    } else {
      d = 0.0;
      if (k == 0) atomicAdd(&ctl->def, 1);
    }
    pa[buf][k] = v;
    pr[buf][k] = (k == j) ? inv : v * inv;
    if (k == 0) s_d[j] = d;
  };
  if (warp == 0) publish(0, a[0], 0);
  __syncthreads();
  for (int t = 0; t < 8; ++t) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * t + u;
      if (j >= nb) break;
      const int buf = j & 1;
      if (4 * warp + 3 > j) {
        const double rk = pr[buf][k];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 4 * warp + q;
          if (i > j && (k >= i || k <= j)) a[q] = fma(-pa[buf][i], rk, a[q]);
        }
      }
      if (j + 1 < nb && warp == ((j + 1) >> 2)) publish(j + 1, a[(u + 1) & 3], buf ^ 1);
      __syncthreads();
    }
  }
  if (warp == 0) s_rs[k] = (k < nb && s_d[k] > 0.0) ? rsqrt64(s_d[k]) : 0.0;
  __syncthreads();
  // R_PP[i][k] = a_ik / sqrt(d_i) (k > i), sqrt(d_i) (k = i);
  // R_PP^-1[k][i] = (L^-1)_ik / sqrt(d_i) (k < i), 1 / sqrt(d_i) (k = i)
  if (k >= nb) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * warp + q;
    if (i >= nb) continue;
    const double rs = s_rs[i];
    if (k > i) {
      R[p0 + i + (int64_t)(p0 + k) * l] = a[q] * rs;
    } else if (k == i) {
      R[p0 + i + (int64_t)(p0 + i) * l] = s_d[i] * rs;
      X[p0 + i + (int64_t)(p0 + i) * l] = rs;
    } else {
      X[p0 + k + (int64_t)(p0 + i) * l] = a[q] * rs;
    }
  }
}

// Step 2: R[P][J0 .. J0+TB) = X_PP^T W[P][J0 .. J0+TB) for columns beyond
// the panel; one block per TB columns, 256 threads, two outputs each.
__global__ void chol64_panel_kernel(const double* __restrict__ W, int l, int p0,
                                    double* __restrict__ R, const double* __restrict__ X,
                                    const CholCtl* ctl) {
  if (ctl->bad) return;
  __shared__ double Xp[CB][CB + 1];
  __shared__ double Gp[CB][TB + 1];
  const int tid = threadIdx.x;
  const int nb = min(CB, l - p0);
  const int p1 = p0 + nb;
  const int j0 = p1 + blockIdx.x * TB;
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int b = e % CB, a = e / CB;
    Xp[b][a] = (b < nb && a < nb) ? X[p0 + b + (int64_t)(p0 + a) * l] : 0.0;
  }
  for (int e = tid; e < CB * TB; e += blockDim.x) {
    const int b = e % CB, c = e / CB;
    const int j = j0 + c;
    Gp[b][c] = (b < nb && j < l) ? W[p0 + b + (int64_t)j * l] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < CB * TB; e += blockDim.x) {
    const int a = e % CB, c = e / CB;
    const int j = j0 + c;
    if (a >= nb || j >= l) continue;
    double s = 0.0;
    for (int b = 0; b <= a; ++b) s = fma(Xp[b][a], Gp[b][c], s);   // X_PP upper: b <= a
    R[p0 + a + (int64_t)j * l] = s;
  }
}

// Step 3: W[i][k] -= sum_a R[p0+a][i] R[p0+a][k] for p1 <= i <= k < l, one
// block per TB x TB tile (ti <= tk), one output per thread.
__global__ void chol64_update_kernel(double* __restrict__ W, int l, int p0,
                                     const double* __restrict__ R, const CholCtl* ctl) {
  if (ctl->bad) return;
  // tile pair from the linear block index: tiles over [p1, l), upper only
  const int nb = min(CB, l - p0);
  const int p1 = p0 + nb;
  const int nt = (l - p1 + TB - 1) / TB;
  int b = blockIdx.x, ti = 0;
  while (b >= nt - ti) {
    b -= nt - ti;
    ++ti;
  }
  const int tk = ti + b;
  __shared__ double Ri[CB][TB + 1];
  __shared__ double Rk[CB][TB + 1];
  const int tid = threadIdx.x;
  const int i0 = p1 + ti * TB, k0 = p1 + tk * TB;
  for (int e = tid; e < CB * TB; e += blockDim.x) {
    const int a = e % CB, c = e / CB;
    Ri[a][c] = (a < nb && i0 + c < l) ? R[p0 + a + (int64_t)(i0 + c) * l] : 0.0;
    Rk[a][c] = (a < nb && k0 + c < l) ? R[p0 + a + (int64_t)(k0 + c) * l] : 0.0;
  }
  __syncthreads();
  const int ii = tid % TB, kk = tid / TB;
  const int i = i0 + ii, k = k0 + kk;
  if (i >= l || k >= l || i > k) return;
  double s = 0.0;
#pragma unroll 8
  for (int a = 0; a < CB; ++a) s = fma(Ri[a][ii], Rk[a][kk], s);
  W[i + (int64_t)k * l] -= s;
}

// Inverse, block row I = [q0, q0 + nq), in two steps (the rows below are
// final; X is upper, so the terms with k > j vanish):
//   S[a][j] = sum_{q1 <= k <= j} R[q0 + a][k] X[k][j]     (chol64_inv_s_kernel)
//   X[q0 + a][j] = -sum_{a <= b < nq} X_II[a][b] S[b][j]  (chol64_inv_x_kernel)
// for j in [q1, l).  8 x 8 output tiles, one output per thread, so the FP64
// work of a block row spreads over many SMs.  S: nq x (l - q1), ld CB.
constexpr int IT = 8;
__global__ void __launch_bounds__(64) chol64_inv_s_kernel(const double* __restrict__ R,
                                                          const double* __restrict__ X, int l,
                                                          int q0, double* __restrict__ S,
                                                          const CholCtl* ctl) {
  if (ctl->bad) return;
  const int nq = min(CB, l - q0);
  const int q1 = q0 + nq;
  const int c = threadIdx.x & (IT - 1), a = threadIdx.x / IT;
  const int j0 = q1 + blockIdx.x * IT, a0 = blockIdx.y * IT;
  __shared__ double Rc[IT][CB + 1];
  __shared__ double Xc[CB][IT + 1];
  const int j = j0 + c, ar = a0 + a;
  const int kend = min(l, j0 + IT);   // X[k][j] = 0 for k > j
  double s = 0.0;
  for (int k0 = q1; k0 < kend; k0 += CB) {
    for (int e = threadIdx.x; e < IT * CB; e += 64) {
      const int rr = e / CB, kk = e % CB;
      Rc[rr][kk] = (a0 + rr < nq && k0 + kk < l) ? R[q0 + a0 + rr + (int64_t)(k0 + kk) * l] : 0.0;
      const int kx = e % CB, cx = e / CB;
      Xc[kx][cx] = (k0 + kx < l && j0 + cx < l) ? X[k0 + kx + (int64_t)(j0 + cx) * l] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < CB; ++kk) s = fma(Rc[a][kk], Xc[kk][c], s);
    __syncthreads();
  }
  if (ar < nq && j < l) S[ar + (int64_t)(j - q1) * CB] = s;
}

__global__ void __launch_bounds__(64) chol64_inv_x_kernel(double* __restrict__ X, int l, int q0,
                                                          const double* __restrict__ S,
                                                          const CholCtl* ctl) {
  if (ctl->bad) return;
  const int nq = min(CB, l - q0);
  const int q1 = q0 + nq;
  const int c = threadIdx.x & (IT - 1), a = threadIdx.x / IT;
  const int j = q1 + blockIdx.x * IT + c, ar = blockIdx.y * IT + a;
  if (ar >= nq || j >= l) return;
  double t = 0.0;
  for (int b = ar; b < nq; ++b)
    t = fma(X[q0 + ar + (int64_t)(q0 + b) * l], S[b + (int64_t)(j - q1) * CB], t);
  X[q0 + ar + (int64_t)j * l] = -t;
}

template <typename T>
__global__ void chol64_out_kernel(const double* __restrict__ R, const double* __restrict__ X,
                                  int l, T* __restrict__ Ro, T* __restrict__ Xo, CholCtl* ctl,
                                  DeviceStatus* status) {
  const int64_t ll = (int64_t)l * l;
  const bool bad = ctl->bad != 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ll;
       t += (int64_t)gridDim.x * blockDim.x) {
    Ro[t] = bad ? T(0) : (T)R[t];
    Xo[t] = bad ? T(0) : (T)X[t];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (bad) atomicOr(&status->flags, 1 << RSVD_ERR_NONFINITE);
    else if (ctl->def) atomicAdd(&status->deficient, ctl->def);
  }
}

}  // namespace

size_t chol64_work_bytes(int l) {
  return (size_t)3 * l * l * sizeof(double) + (size_t)CB * l * sizeof(double) + 256;
}

// drop: FP64 Grams drop pivots below l eps64 max diag(G), FP32 Grams below
// eps32 max diag(G): the rules of the one-CTA kernels for each element type.
template <typename T>
cudaError_t launch_chol64(const T* G, int64_t ldg, int l, T* R, T* Rinv, void* work,
                          DeviceStatus* status, cudaStream_t st) {
  const double drop = sizeof(T) == 8 ? (double)l * DBL_EPSILON : (double)FLT_EPSILON;
  const size_t ll = (size_t)l * l;
  double* W = (double*)work;
  double* Rb = W + ll;
  double* Xb = Rb + ll;
  double* Sb = Xb + ll;
  CholCtl* ctl = (CholCtl*)(Sb + (size_t)CB * l);
  const int blocks = (int)std::min<size_t>((ll + 255) / 256, 64);
  chol64_setup_kernel<T><<<blocks, 256, 0, st>>>(G, ldg, l, drop, W, Rb, Xb, ctl);
  note_launch();
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int p0 = 0; p0 < l; p0 += CB) {
    chol64_diag_kernel<<<1, 256, 0, st>>>(W, l, p0, Rb, Xb, ctl);
    note_launch();
    const int p1 = std::min(l, p0 + CB);
    if (p1 < l) {
      const int nt = (l - p1 + TB - 1) / TB;
      chol64_panel_kernel<<<nt, 256, 0, st>>>(W, l, p0, Rb, Xb, ctl);
      note_launch();
      chol64_update_kernel<<<nt * (nt + 1) / 2, TB * TB, 0, st>>>(W, l, p0, Rb, ctl);
      note_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int nblk = (l + CB - 1) / CB;
  for (int I = nblk - 2; I >= 0; --I) {
    const int q0 = I * CB;
    const int q1 = std::min(l, q0 + CB);
    const dim3 g((unsigned)((l - q1 + IT - 1) / IT), (unsigned)((q1 - q0 + IT - 1) / IT));
    chol64_inv_s_kernel<<<g, 64, 0, st>>>(Rb, Xb, l, q0, Sb, ctl);
    note_launch();
    chol64_inv_x_kernel<<<g, 64, 0, st>>>(Xb, l, q0, Sb, ctl);
    note_launch();
  }
  chol64_out_kernel<T><<<blocks, 256, 0, st>>>(Rb, Xb, l, R, Rinv, ctl, status);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_chol64<double>(const double*, int64_t, int, double*, double*, void*,
                                           DeviceStatus*, cudaStream_t);
template cudaError_t launch_chol64<float>(const float*, int64_t, int, float*, float*, void*,
                                          DeviceStatus*, cudaStream_t);

}  // namespace rsvd
