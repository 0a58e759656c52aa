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
#include <cfloat>

#include <algorithm>

#include "internal.h"

namespace rsvd {
namespace {

constexpr int SMALL_THREADS = 1024;

template <typename T>
struct Eps;
// drop_factor: a Gram pivot below drop_factor * eps * max(diag G) marks a
// dependent column.  FP64 uses l (exactly dependent columns leave pivots of a
// few ulps times l); FP32 uses 1 -- its Gram already blurs pivots near
// sqrt(eps) relative, and dropping there would discard directions the mixed
// path still resolves; exactly dependent FP32 columns are instead kept as
// directions orthogonal to range(Y) after the second CholeskyQR pass.
template <>
struct Eps<double> {
  static constexpr double value = DBL_EPSILON;
  __device__ static double drop_factor(int l) { return (double)l; }
};
template <>
struct Eps<float> {
  static constexpr float value = FLT_EPSILON;
  __device__ static float drop_factor(int) { return 1.0f; }
};

__device__ __forceinline__ void set_flag(DeviceStatus* s, int code) {
  atomicOr(&s->flags, 1 << code);
}

// G (ldg) -> R (ld l, upper; lower part zeroed), Rinv (ld l, upper).
// W (l*l) and the scratch S (33*(l+64) elements) live in dynamic shared
// memory when they fit, else in `gwork` (l*l + 33*(l+64) elements).
//
// Cholesky: right-looking, one pivot per step, trailing update of the upper
// triangle by a 32 x 32 thread grid.  Inverse (in place, LAPACK trtri's
// block-column order with 32 x 32 blocks):
//   1. every diagonal block D_b is inverted in parallel, one warp per block
//      and one lane per column (back substitution against a copy of D_b);
//   2. for block columns b = 1, 2, ...:  X(0:b, b) = -X(0:b, 0:b) R(0:b, b) X(b, b)
//      as two small dense products over all threads.
template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS)
chol_inv_kernel(const T* __restrict__ G, int64_t ldg, int l, T* __restrict__ R,
                T* __restrict__ Rinv, T* __restrict__ gwork, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* W = gwork ? gwork : reinterpret_cast<T*>(smem_raw);  // column-major l x l
  T* S = W + (int64_t)l * l;                                  // 33 x (l + 64) scratch
  __shared__ T s_maxdiag;
  __shared__ T s_r, s_inv;
  __shared__ int s_bad;
  __shared__ int s_deficient;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tx = tid & 31, ty = tid >> 5;   // 32 x 32 grid

  for (int t = tid; t < l * l; t += nt) {
    int i = t % l, j = t / l;
    W[t] = (i <= j) ? G[i + (int64_t)j * ldg] : T(0);
  }
  if (tid == 0) {
    s_bad = 0;
    s_deficient = 0;
  }
  __syncthreads();
  if (tid == 0) {
    T mx = T(0);
    int bad = 0;
    for (int j = 0; j < l; ++j) {
      T d = W[j + j * l];
      if (!isfinite(d)) bad = 1;
      mx = fmax(mx, fabs(d));
    }
    s_maxdiag = mx;
    s_bad = bad;
  }
  __syncthreads();
  if (s_bad) {
    for (int t = tid; t < l * l; t += nt) {
      R[t] = T(0);
      Rinv[t] = T(0);
    }
    if (tid == 0) set_flag(status, RSVD_ERR_NONFINITE);
    return;
  }
  const T tol = Eps<T>::drop_factor(l) * Eps<T>::value * s_maxdiag;

  // ---- Cholesky: G = R^T R on the upper triangle, 32-wide panels ----
  // Per panel k (rows/columns k0 .. k0+kw-1):
  //  (i)   warp 0 factors the diagonal block in a padded copy (S, 32 x 33);
  //  (ii)  the panel rows R[k0:k0+kw, c] = D^-T G[k0:k0+kw, c] for the columns
  //        right of the block, one thread per column, in a transposed padded
  //        copy P (c-major, stride 33) so threads touch distinct banks;
  //  (iii) trailing update G[i][c] -= sum_t P[i][t] P[c][t] for i <= c.
  T* Dg = S;                 // 32 x 33 diagonal block (column-major, ld 33)
  T* Dinv = S + 32 * 33;     // 32 reciprocal pivots
  T* Pp = S + 33 * 33;       // (l - k0 - kw) x 33 transposed panel
  for (int k0 = 0; k0 < l; k0 += 32) {
    const int kw = min(32, l - k0);
    const int c_beg = k0 + kw, nc = l - c_beg;
    // load the diagonal block (upper) and the panel rows (transposed)
    for (int t = tid; t < 32 * 32; t += nt) {
      const int i = t & 31, c = t >> 5;
      Dg[i + c * 33] = (i < kw && c < kw && i <= c) ? W[k0 + i + (k0 + c) * l] : T(0);
    }
    for (int t = tid; t < nc * 32; t += nt) {
      const int i = t & 31, c = t >> 5;   // i: panel row, c: column offset
      Pp[c * 33 + i] = (i < kw) ? W[k0 + i + (c_beg + c) * l] : T(0);
    }
    __syncthreads();
    if (ty == 0) {
      // (i) one warp, lane = column within the block
      const int c = tx;
      for (int j = 0; j < kw; ++j) {
        const T d = Dg[j + j * 33];
        T r, inv;
        if (!(d > tol)) {
          r = T(0);
          inv = T(0);
          if (c == 0) s_deficient++;
        } else {
          r = sqrt(d);
          inv = T(1) / r;
        }
        __syncwarp();
        if (c > j && c < kw) Dg[j + c * 33] *= inv;
        if (c == j) {
          Dg[j + j * 33] = r;
          Dinv[j] = inv;
        }
        __syncwarp();
        if (c > j && c < kw) {
          const T rjc = Dg[j + c * 33];
          for (int i = j + 1; i <= c; ++i) Dg[i + c * 33] -= Dg[j + i * 33] * rjc;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // (ii) panel rows: solve D^T x = g per column (forward substitution)
    for (int c = tid; c < nc; c += nt) {
      T* x = Pp + c * 33;
      for (int i = 0; i < kw; ++i) {
        T acc = x[i];
        for (int t2 = 0; t2 < i; ++t2) acc -= Dg[t2 + i * 33] * x[t2];
        x[i] = acc * Dinv[i];   // a dropped pivot (Dinv 0) zeroes the row
      }
    }
    __syncthreads();
    // write the factored block and panel rows back; (iii) trailing update
    for (int t = tid; t < 32 * 32; t += nt) {
      const int i = t & 31, c = t >> 5;
      if (i < kw && c < kw && i <= c) W[k0 + i + (k0 + c) * l] = Dg[i + c * 33];
    }
    for (int t = tid; t < nc * 32; t += nt) {
      const int i = t & 31, c = t >> 5;
      if (i < kw) W[k0 + i + (c_beg + c) * l] = Pp[c * 33 + i];
    }
    for (int cc = ty; cc < nc; cc += 32) {
      const T* pc = Pp + cc * 33;
      for (int ii = tx; ii <= cc; ii += 32) {
        const T* pi = Pp + ii * 33;
        T acc = T(0);
#pragma unroll 8
        for (int t2 = 0; t2 < kw; ++t2) acc = fma(pi[t2], pc[t2], acc);
        W[c_beg + ii + (c_beg + cc) * l] -= acc;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < l * l; t += nt) {
    int i = t % l, j = t / l;
    R[t] = (i <= j) ? W[t] : T(0);
  }
  __syncthreads();

  // ---- Inverse, step 1: diagonal 32 x 32 blocks, one warp each ----
  const int nb = (l + 31) / 32;
  // copy every diagonal block to S (block b at S + b*1024, column-major 32 x 32)
  for (int t = tid; t < nb * 1024; t += nt) {
    const int b = t >> 10, e = t & 1023, i = e & 31, c = e >> 5;
    const int gi = b * 32 + i, gc = b * 32 + c;
    S[t] = (gi < l && gc < l) ? W[gi + gc * l] : T(0);
  }
  __syncthreads();
  for (int b = ty; b < nb; b += 32) {
    const int c = tx, gc = b * 32 + c;
    const T* D = S + b * 1024;
    if (gc < l) {
      const T dcc = D[c + c * 32];
      if (dcc == T(0)) {
        for (int i = 0; i <= c; ++i) W[b * 32 + i + gc * l] = T(0);
      } else {
        W[gc + gc * l] = T(1) / dcc;
        for (int i = c - 1; i >= 0; --i) {
          const T dii = D[i + i * 32];
          T acc = T(0);
          for (int t2 = i + 1; t2 <= c; ++t2) acc = fma(D[i + t2 * 32], W[b * 32 + t2 + gc * l], acc);
          W[b * 32 + i + gc * l] = (dii == T(0)) ? T(0) : -acc / dii;
        }
      }
    }
  }
  __syncthreads();

  // ---- Inverse, step 2: block columns left to right ----
  for (int bj = 1; bj < nb; ++bj) {
    const int c0 = bj * 32, cw = min(32, l - c0);
    const int rows = c0;  // rows 0 .. c0-1
    // (a) S(r, c) = sum_{u=r}^{c0-1} X[r][u] R[u][c0+c]   (X upper, already final)
    for (int t = tid; t < rows * cw; t += nt) {
      const int r = t % rows, c = t / rows;
      T acc = T(0);
      for (int u = r; u < c0; ++u) acc = fma(W[r + u * l], W[u + (c0 + c) * l], acc);
      S[r + c * rows] = acc;
    }
    __syncthreads();
    // (b) X[r][c0+c] = - sum_{s=0}^{c} S(r, s) X[c0+s][c0+c]
    for (int t = tid; t < rows * cw; t += nt) {
      const int r = t % rows, c = t / rows;
      T acc = T(0);
      for (int s2 = 0; s2 <= c; ++s2) acc = fma(S[r + s2 * rows], W[c0 + s2 + (c0 + c) * l], acc);
      W[r + (c0 + c) * l] = -acc;
    }
    __syncthreads();
  }
  for (int t = tid; t < l * l; t += nt) {
    int i = t % l, j = t / l;
    Rinv[t] = (i <= j) ? W[t] : T(0);
  }
  if (tid == 0 && s_deficient) atomicAdd(&status->deficient, s_deficient);
}

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

// ---------------------------------------------------------------------------
// One-sided Jacobi
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// player at position `pos` in round `r` of a round-robin on 2P players
__device__ __forceinline__ int rr_player(int pos, int r, int twoP) {
  if (pos == 0) return 0;
  return 1 + (pos - 1 + r) % (twoP - 1);
}

// Work layout: Wm (l x twoP) and, if V is accumulated, Wv (l x twoP), both
// column-major with ld l; in dynamic shared memory when they fit, else in
// `gwork`.  Each round of the round-robin ordering runs in three phases so
// that the FP64 pipe (2 lanes per clock per SM) is spent on useful work:
//   A. G threads per column pair form partial |c_p|^2, |c_q|^2, c_p.c_q over
//      interleaved rows and reduce them with shuffles inside the group;
//   B. one thread per pair turns (a, b, g) into a rotation (c, s);
//   C. the G threads of each pair apply it to their rows.
template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS)
jacobi_svd_kernel(const T* __restrict__ M, int l, int64_t ldm, T* __restrict__ sig,
                  T* __restrict__ Um, int64_t ldu, T* __restrict__ Vm, int64_t ldv,
                  T* __restrict__ UsInv, T* __restrict__ gwork, int use_smem,
                  DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char jsm_raw[];
  T* jsm = reinterpret_cast<T*>(jsm_raw);
  const int twoP = (l + 1) & ~1;  // even number of columns (one zero column if l is odd)
  const int P = twoP / 2;
  const bool want_v = Vm != nullptr;
  T* Wm = use_smem ? jsm : gwork;
  T* Wv = Wm + (int64_t)l * twoP;
  __shared__ int s_rot;
  __shared__ T s_norm[RSVD_L_MAX + 1];
  __shared__ T s_abg[(RSVD_L_MAX + 1) / 2][3];
  __shared__ T s_cs[(RSVD_L_MAX + 1) / 2][2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  // threads per pair: power of two, at most 16 rows each
  int G = 1;
  while (G < 32 && (l + G - 1) / G > 16) G <<= 1;
  const int items = P * G;
  const int items_pad = (items + 31) & ~31;

  for (int t = tid; t < l * twoP; t += nt) {
    int i = t % l, j = t / l;
    Wm[t] = (j < l) ? M[i + (int64_t)j * ldm] : 0.0;
    if (want_v) Wv[t] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) s_rot = 0;
  __syncthreads();
  const T tol = sqrt((T)l) * Eps<T>::value;
  int sweep = 0;
  const int max_sweeps = 30;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < twoP - 1; ++r) {
      // A: partial dot products
      for (int it = tid; it < items_pad; it += nt) {
        const int pr = it / G, sub = it % G;
        T a = 0.0, b = 0.0, g = 0.0;
        if (it < items) {
          int p = rr_player(pr, r, twoP), q = rr_player(twoP - 1 - pr, r, twoP);
          if (p > q) { int t = p; p = q; q = t; }
          const T* cp = Wm + (int64_t)p * l;
          const T* cq = Wm + (int64_t)q * l;
          for (int i = sub; i < l; i += G) {
            T x = cp[i], y = cq[i];
            a = fma(x, x, a);
            b = fma(y, y, b);
            g = fma(x, y, g);
          }
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (it < items && sub == 0) {
          s_abg[pr][0] = a;
          s_abg[pr][1] = b;
          s_abg[pr][2] = g;
        }
      }
      __syncthreads();
      // B: rotation parameters (Rutishauser): zeta = (b - a) / (2g),
      // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t
      for (int pr = tid; pr < P; pr += nt) {
        const T a = s_abg[pr][0], b = s_abg[pr][1], g = s_abg[pr][2];
        T c = T(1), sn = T(0);
        if (g != 0.0 && fabs(g) > tol * sqrt(a) * sqrt(b)) {
          const T zeta = (b - a) / (T(2) * g);
          const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
          c = rsqrt(fma(t, t, T(1)));
          sn = c * t;
          s_rot = 1;
        }
        s_cs[pr][0] = c;
        s_cs[pr][1] = sn;
      }
      __syncthreads();
      // C: apply
      for (int it = tid; it < items; it += nt) {
        const int pr = it / G, sub = it % G;
        const T c = s_cs[pr][0], sn = s_cs[pr][1];
        if (sn == 0.0) continue;
        int p = rr_player(pr, r, twoP), q = rr_player(twoP - 1 - pr, r, twoP);
        if (p > q) { int t = p; p = q; q = t; }
        T* cp = Wm + (int64_t)p * l;
        T* cq = Wm + (int64_t)q * l;
        for (int i = sub; i < l; i += G) {
          T x = cp[i], y = cq[i];
          cp[i] = c * x - sn * y;
          cq[i] = sn * x + c * y;
        }
        if (want_v) {
          T* vp = Wv + (int64_t)p * l;
          T* vq = Wv + (int64_t)q * l;
          for (int i = sub; i < l; i += G) {
            T x = vp[i], y = vq[i];
            vp[i] = c * x - sn * y;
            vq[i] = sn * x + c * y;
          }
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (tid == 0) s_rot = 0;
    __syncthreads();
    if (!rot) break;
  }
  if (tid == 0) {
    status->jacobi_sweeps = sweep + 1;
    if (sweep >= max_sweeps) set_flag(status, RSVD_ERR_JACOBI);
  }
  // column norms
  for (int c = warp; c < l; c += nwarps) {
    const T* cp = Wm + (int64_t)c * l;
    T a = 0.0;
    for (int i = lane; i < l; i += 32) a = fma(cp[i], cp[i], a);
    a = warp_sum(a);
    if (lane == 0) s_norm[c] = sqrt(a);
  }
  __syncthreads();
  // sort descending by rank; ties keep column order
  for (int c = warp; c < l; c += nwarps) {
    const T sc = s_norm[c];
    int rank = 0;
    for (int d = lane; d < l; d += 32) {
      T sd = s_norm[d];
      rank += (sd > sc || (sd == sc && d < c)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const T inv = sc > T(0) ? T(1) / sc : T(0);
    if (lane == 0) sig[rank] = sc;
    for (int i = lane; i < l; i += 32) {
      const T u = Wm[i + (int64_t)c * l] * inv;
      Um[i + (int64_t)rank * ldu] = u;
      if (UsInv) UsInv[i + (int64_t)rank * l] = u * inv;
      if (want_v) Vm[i + (int64_t)rank * ldv] = Wv[i + (int64_t)c * l];
    }
  }
}

// ---------------------------------------------------------------------------
// Sign convention and outputs
// ---------------------------------------------------------------------------

template <typename T>
__global__ void sign_kernel(T* __restrict__ U, int64_t m, int64_t ldu,
                            T* __restrict__ sign) {
  const int col = blockIdx.x;
  T* u = U + (int64_t)col * ldu;
  T best = -1.0;
  int64_t bidx = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    T v = fabs(u[i]);
    if (v > best) { best = v; bidx = i; }
  }
  __shared__ T sv[1024];
  __shared__ int64_t si[1024];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      T o = sv[threadIdx.x + s];
      int64_t oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  __shared__ T s_sign;
  if (threadIdx.x == 0) {
    s_sign = (u[si[0]] < 0.0) ? -1.0 : 1.0;
    sign[col] = s_sign;
  }
  __syncthreads();
  if (s_sign < 0.0)
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
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

}  // namespace

template <typename T>
cudaError_t launch_chol_inv(const T* G, int64_t ldg, int l, T* R, T* Rinv, T* work,
                            DeviceStatus* status, cudaStream_t st) {
  const size_t smem = ((size_t)l * l + 33 * (size_t)(l + 64)) * sizeof(T);
  const size_t cap = 200 * 1024;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    attr_set = true;
  }
  if (smem <= cap)
    chol_inv_kernel<T><<<1, SMALL_THREADS, smem, st>>>(G, ldg, l, R, Rinv, nullptr, status);
  else
    chol_inv_kernel<T><<<1, SMALL_THREADS, 0, st>>>(G, ldg, l, R, Rinv, work, status);
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
                              cudaStream_t st) {
  const int twoP = (l + 1) & ~1;
  const size_t need = (size_t)(Vm ? 2 : 1) * l * twoP * sizeof(T);
  const size_t cap = 200 * 1024;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(jacobi_svd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cap);
    attr_set = true;
  }
  const bool smem = need <= cap;
  jacobi_svd_kernel<T><<<1, SMALL_THREADS, smem ? need : 0, st>>>(
      M, l, ldm, sig, Um, ldu, Vm, ldv, UsInv, work, smem ? 1 : 0, status);
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

#define RSVD_INSTANTIATE_SMALL(T)                                                              \
  template cudaError_t launch_chol_inv<T>(const T*, int64_t, int, T*, T*, T*, DeviceStatus*,   \
                                          cudaStream_t);                                       \
  template cudaError_t launch_tri_product<T>(const T*, const T*, int, T*, bool, cudaStream_t); \
  template cudaError_t launch_jacobi_svd<T>(const T*, int, int64_t, T*, T*, int64_t, T*,       \
                                            int64_t, T*, T*, DeviceStatus*, cudaStream_t);     \
  template cudaError_t launch_finalize<T>(T*, int64_t, int64_t, int, const T*, int64_t, T*,    \
                                          int64_t, const T*, double*, T*, cudaStream_t);
RSVD_INSTANTIATE_SMALL(double)
RSVD_INSTANTIATE_SMALL(float)

}  // namespace rsvd
