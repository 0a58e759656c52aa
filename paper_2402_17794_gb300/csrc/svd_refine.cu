// FP64 refinement of an approximate SVD of the small l x l matrix of step 7
// (Algorithm 4, Section 3.3): the FP32 one-sided Jacobi gives U, sigma to
// about 1e-7; a few refinement steps carried out in FP64 take them to FP64
// accuracy at the cost of l x l matrix products, which spread over the whole
// GPU (one-sided Jacobi sweeps in FP64 run on one SM's FP64 pipe, 2 FMA per
// clock on this part).
//
// The step (Ogita and Aishima, "Iterative refinement for singular value
// decomposition based on matrix multiplication", J. Comput. Appl. Math. 369,
// 2020), derived to first order: with R = I - U^T U, S = I - V^T V and
// T = U^T M V, corrections U <- U (I + F), V <- V (I + G) that make U, V
// orthogonal and U^T M V diagonal satisfy
//   F + F^T = R,  G + G^T = S,  T + F^T D + D G = diagonal  (D = diag s~).
// The diagonal gives F_ii = r_ii / 2, G_ii = s_ii / 2 and
// s~_i = t_ii / (1 - (r_ii + s_ii) / 2).  For i != j the four equations in
// F_ij, F_ji, G_ij, G_ji reduce to the 2 x 2 system
//   -s~_j F_ij + s~_i G_ij = -t_ij - s~_j r_ij
//    s~_i F_ij - s~_j G_ij = -t_ji - s~_j s_ij
// (determinant s~_j^2 - s~_i^2).  Singular values closer than cluster_tol *
// s~_1 form a cluster: there only the symmetric parts F_ij = r_ij / 2,
// G_ij = s_ij / 2 are applied (orthonormality is restored, the cluster's
// vectors and values keep the accuracy of the start).  Each step squares the
// error of a start whose error is small against the relative gaps; pairs
// closer than the start's error would make the linearised step diverge,
// which is what the cluster tolerance guards against.
#include <algorithm>

#include "internal.h"

namespace rsvd {
namespace {

// C = alpha op(A) op(B) + beta C0 (all l x l, ld l, FP64), blockIdx.z selects
// one of up to three independent products.  16 x 16 output tiles, one output
// per thread, so an l = 160 product spreads over 100 SMs.
struct Prod {
  const double* A;
  const double* B;
  const double* C0;   // may be NULL (beta ignored)
  double* C;
  int ta, tb;
  double alpha, beta;
};
struct Prods {
  Prod p[3];
};

__global__ void small_prod_kernel(const __grid_constant__ Prods P, int l) {
  const Prod& q = P.p[blockIdx.z];
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < l; k0 += 16) {
    {   // As[tx][ty] = op(A)(i, k0 + ty)
      const int kk = k0 + ty;
      As[tx][ty] = (i < l && kk < l) ? (q.ta ? q.A[kk + (int64_t)i * l] : q.A[i + (int64_t)kk * l])
                                     : 0.0;
    }
    {   // Bs[tx][ty] = op(B)(k0 + tx, j)
      const int kk = k0 + tx;
      Bs[tx][ty] = (kk < l && j < l) ? (q.tb ? q.B[j + (int64_t)kk * l] : q.B[kk + (int64_t)j * l])
                                     : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(As[tx][t], Bs[t][ty], acc);
    __syncthreads();
  }
  if (i < l && j < l) {
    const int64_t o = i + (int64_t)j * l;
    q.C[o] = q.alpha * acc + (q.C0 ? q.beta * q.C0[o] : 0.0);
  }
}

// F, G (ld l) and s~ from R = I - U^T U (given as U^T U), S = I - V^T V
// (given as V^T V) and T; one thread per (i, j).
__global__ void refine_coef_kernel(const double* __restrict__ UtU, const double* __restrict__ VtV,
                                   const double* __restrict__ T, int l, double cluster_tol,
                                   double* __restrict__ F, double* __restrict__ G,
                                   double* __restrict__ s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= l * l) return;
  const int i = t % l, j = t / l;
  auto sig = [&](int a) {
    const double r = 1.0 - UtU[a + (int64_t)a * l], ss = 1.0 - VtV[a + (int64_t)a * l];
    return T[a + (int64_t)a * l] / (1.0 - 0.5 * (r + ss));
  };
  const double r_ij = (i == j ? 1.0 : 0.0) - UtU[t];
  const double s_ij = (i == j ? 1.0 : 0.0) - VtV[t];
  if (i == j) {
    F[t] = 0.5 * r_ij;
    G[t] = 0.5 * s_ij;
    s[i] = sig(i);
    return;
  }
  const double si = sig(i), sj = sig(j);
  const double s1 = fmax(fabs(sig(0)), fmax(fabs(si), fabs(sj)));
  if (fabs(si - sj) <= cluster_tol * s1) {
    F[t] = 0.5 * r_ij;
    G[t] = 0.5 * s_ij;
    return;
  }
  const double a = -T[t] - sj * r_ij;                       // -t_ij - s~_j r_ij
  const double b = -T[j + (int64_t)i * l] - sj * s_ij;      // -t_ji - s~_j s_ij
  const double det = sj * sj - si * si;                     // of [[-sj, si], [si, -sj]]
  F[t] = (-sj * a - si * b) / det;
  G[t] = (-si * a - sj * b) / det;
}

// Us (ld l) = U diag(1 / s) for s_i > 0 (0 otherwise); sig_out[i] = s_i.
__global__ void scale_cols_kernel(const double* __restrict__ U, const double* __restrict__ s, int l,
                                  double* __restrict__ Us) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= l * l) return;
  const int j = t / l;
  Us[t] = s[j] > 0.0 ? U[t] / s[j] : 0.0;
}

cudaError_t prods(const Prods& P, int count, int l, cudaStream_t st) {
  const dim3 grid((unsigned)((l + 15) / 16), (unsigned)((l + 15) / 16), (unsigned)count);
  small_prod_kernel<<<grid, 256, 0, st>>>(P, l);
  note_launch();
  return cudaGetLastError();
}

Prod prod(const double* A, int ta, const double* B, int tb, double* C, double alpha = 1.0,
          const double* C0 = nullptr, double beta = 0.0) {
  Prod q;
  q.A = A;
  q.B = B;
  q.C0 = C0;
  q.C = C;
  q.ta = ta;
  q.tb = tb;
  q.alpha = alpha;
  q.beta = beta;
  return q;
}

}  // namespace

cudaError_t launch_svd_refine(const double* M, int l, double* U, double* V, double* s, int steps,
                              double cluster_tol, double* work, cudaStream_t st) {
  const size_t ll = (size_t)l * l;
  double *P = work, *UtU = work + ll, *VtV = work + 2 * ll, *T = work + 3 * ll;
  double *F = work + 4 * ll, *G = work + 5 * ll, *U2 = work + 6 * ll, *V2 = work + 7 * ll;
  cudaError_t e;
  for (int it = 0; it < steps; ++it) {
    Prods a;
    a.p[0] = prod(M, 0, V, 0, P);          // P = M V
    a.p[1] = prod(U, 1, U, 0, UtU);        // U^T U
    a.p[2] = prod(V, 1, V, 0, VtV);        // V^T V
    if ((e = prods(a, 3, l, st)) != cudaSuccess) return e;
    Prods b;
    b.p[0] = prod(U, 1, P, 0, T);          // T = U^T M V
    if ((e = prods(b, 1, l, st)) != cudaSuccess) return e;
    refine_coef_kernel<<<(int)((ll + 255) / 256), 256, 0, st>>>(UtU, VtV, T, l, cluster_tol, F,
                                                                G, s);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Prods c;
    c.p[0] = prod(U, 0, F, 0, U2, 1.0, U, 1.0);   // U (I + F)
    c.p[1] = prod(V, 0, G, 0, V2, 1.0, V, 1.0);   // V (I + G)
    if ((e = prods(c, 2, l, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(U, U2, ll * sizeof(double), cudaMemcpyDeviceToDevice, st)))
      return e;
    if ((e = cudaMemcpyAsync(V, V2, ll * sizeof(double), cudaMemcpyDeviceToDevice, st)))
      return e;
  }
  return cudaSuccess;
}

namespace {
// accept[0] = 1 when U, V are orthogonal to 1e-13 (max |I - U^T U|,
// max |I - V^T V|) and U^T M V is diagonal to 1e-12 of the larger singular
// value of each pair (|T_ij| <= 1e-12 max(s_i, s_j, eps s_1)), everything
// finite; else 0.  Then the refined s carries each sigma to about
// T_ij^2 / (s_i |s_i - s_j|) <= 1e-24 s / |s_i - s_j| relative, far below
// the rounding of the FP64 solve except for pairs closer than ~1e-10, whose
// sigmas the bound still holds to ~1e-14.  One block.
__global__ void svd_accept_kernel(const double* __restrict__ UtU, const double* __restrict__ VtV,
                                  const double* __restrict__ T, const double* __restrict__ s,
                                  int l, int* __restrict__ accept) {
  __shared__ int s_bad;
  __shared__ double s_max;
  if (threadIdx.x == 0) {
    s_bad = 0;
    double mx = 0.0;
    for (int i = 0; i < l; ++i) mx = fmax(mx, fabs(s[i]));
    s_max = mx;
  }
  __syncthreads();
  const double floor_s = 2.220446049250313e-16 * s_max;
  int bad = !(s_max > 0.0) || !isfinite(s_max);
  for (int t = threadIdx.x; t < l * l; t += blockDim.x) {
    const int i = t % l, j = t / l;
    const double e = i == j ? 1.0 : 0.0;
    const double u = UtU[t], v = VtV[t], x = T[t];
    if (!(fabs(e - u) <= 1e-13) || !(fabs(e - v) <= 1e-13)) bad = 1;
    if (i != j) {
      const double den = fmax(fmax(fabs(s[i]), fabs(s[j])), floor_s);
      if (!(fabs(x) <= 1e-12 * den)) bad = 1;
    }
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) *accept = s_bad ? 0 : 1;
}
}  // namespace

cudaError_t launch_svd_accept(const double* M, int l, const double* U, const double* V,
                              const double* s, double* work, int* accept, cudaStream_t st) {
  const size_t ll = (size_t)l * l;
  double *P = work, *UtU = work + ll, *VtV = work + 2 * ll, *T = work + 3 * ll;
  cudaError_t e;
  Prods a;
  a.p[0] = prod(M, 0, V, 0, P);          // P = M V
  a.p[1] = prod(U, 1, U, 0, UtU);        // U^T U
  a.p[2] = prod(V, 1, V, 0, VtV);        // V^T V
  if ((e = prods(a, 3, l, st)) != cudaSuccess) return e;
  Prods b;
  b.p[0] = prod(U, 1, P, 0, T);          // T = U^T M V
  if ((e = prods(b, 1, l, st)) != cudaSuccess) return e;
  svd_accept_kernel<<<1, 1024, 0, st>>>(UtU, VtV, T, s, l, accept);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_cols(const double* U, const double* s, int l, double* Us,
                              cudaStream_t st) {
  scale_cols_kernel<<<(l * l + 255) / 256, 256, 0, st>>>(U, s, l, Us);
  note_launch();
  return cudaGetLastError();
}

// V (ld l) = M^T U diag(1 / s): the right singular vectors implied by U, s.
cudaError_t launch_right_vectors(const double* M, const double* Us, int l, double* V,
                                 cudaStream_t st) {
  Prods a;
  a.p[0] = prod(M, 1, Us, 0, V);
  return prods(a, 1, l, st);
}

// V <- V (3 I - V^T V) / 2, `steps` times (Newton-Schulz iteration for the
// orthogonal polar factor: each step squares ||I - V^T V|| when it is below
// one).  work: 2 l^2 doubles.
cudaError_t launch_orthonormalize(double* V, int l, int steps, double* work, cudaStream_t st) {
  const size_t ll = (size_t)l * l;
  double *N = work, *V2 = work + ll;
  cudaError_t e;
  for (int it = 0; it < steps; ++it) {
    Prods a;
    a.p[0] = prod(V, 1, V, 0, N);                     // N = V^T V
    if ((e = prods(a, 1, l, st)) != cudaSuccess) return e;
    Prods b;
    b.p[0] = prod(V, 0, N, 0, V2, -0.5, V, 1.5);      // 1.5 V - 0.5 V N
    if ((e = prods(b, 1, l, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(V, V2, ll * sizeof(double), cudaMemcpyDeviceToDevice, st)))
      return e;
  }
  return cudaSuccess;
}

// C (ld l) = A B, all l x l FP64.
cudaError_t launch_small_product(const double* A, const double* B, int l, double* C,
                                 cudaStream_t st) {
  Prods a;
  a.p[0] = prod(A, 0, B, 0, C);
  return prods(a, 1, l, st);
}

namespace {
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ in, int64_t count, Tout* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (Tout)in[t];
}
}  // namespace

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* in, int64_t count, Tout* out, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
  convert_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(in, count, out);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double*, int64_t, float*, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, int64_t, double*,
                                                    cudaStream_t);

}  // namespace rsvd
