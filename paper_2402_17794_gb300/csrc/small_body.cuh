// Shared bodies of the l x l kernels (single-problem and grouped launches):
// one CTA of SMALL_THREADS threads runs one problem.
#pragma once

#include <cfloat>

#include "internal.h"

namespace rsvd {
namespace dense {

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
__device__ __forceinline__ void chol_inv_body(const T* __restrict__ G, int64_t ldg, int l,
                                              T* __restrict__ R, T* __restrict__ Rinv,
                                              T* __restrict__ W, DeviceStatus* status) {
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


// ---------------------------------------------------------------------------
// One-sided Jacobi
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// player at position `pos` in round `r` (0 <= r < 2P-1) of a round-robin
// on 2P players: position 0 is fixed, the others rotate by one per round
__device__ __forceinline__ int rr_player(int pos, int r, int twoP) {
  if (pos == 0) return 0;
  int v = pos - 1 + r;
  if (v >= twoP - 1) v -= twoP - 1;
  return 1 + v;
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
__device__ __forceinline__ void jacobi_body(const T* __restrict__ M, int l, int64_t ldm,
                                            T* __restrict__ sig, T* __restrict__ Um, int64_t ldu,
                                            T* __restrict__ Vm, int64_t ldv,
                                            T* __restrict__ UsInv, T* __restrict__ Wm,
                                            DeviceStatus* status) {
  const int twoP = (l + 1) & ~1;  // even number of columns (one zero column if l is odd)
  const int P = twoP / 2;
  const bool want_v = Vm != nullptr;
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

// One CTA of 1024 threads per column: flips u so its largest-|.| entry (lowest
// index on ties) is positive and stores the sign taken.
template <typename T>
__device__ __forceinline__ void sign_body(T* __restrict__ u, int64_t m, T* __restrict__ sign_out) {
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
    *sign_out = s_sign;
  }
  __syncthreads();
  if (s_sign < 0.0)
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
}



}  // namespace dense
}  // namespace rsvd
