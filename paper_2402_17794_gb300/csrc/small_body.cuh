// Shared bodies of the l x l kernels (single-problem and grouped launches):
// one CTA of SMALL_THREADS threads runs one problem.
#pragma once

#include <cfloat>

#include <cooperative_groups.h>

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

// Leading dimension of the Cholesky work matrix: odd, so that a warp reading
// one row (stride ld) touches 32 distinct banks.
__host__ __device__ constexpr int chol_ld(int l) { return (l + 1) | 1; }

// Elements of work the blocked Cholesky needs: l x chol_ld(l).
__host__ __device__ constexpr size_t chol_work_elems(int l) { return (size_t)l * chol_ld(l); }

// Both Cholesky variants below (blocked, and register-resident for FP32
// l <= 160) compute G = R^T R and R^-1 by one elimination
// on [G | I] (Gauss without pivoting, stable for an SPD matrix): with
// G = L D L^T, L unit lower triangular,
//   step j, every row i > j:  row_i -= (G_ij / D_j) row_j
// turns G's upper triangle into D L^T and the identity into L^-1.  Both live
// in one matrix W: W[i][c] for c >= i is the upper part (D L^T), for c < i
// the strictly lower part of L^-1 (its unit diagonal is implicit).  Then
//   R = D^{1/2} L^T:       R[i][c]    = W[i][c] / sqrt(D_i)
//   R^-1 = L^-T D^{-1/2}:  R^-1[i][c] = W[c][i] / sqrt(D_c)   (i < c)
// Step j reads only row j and writes only rows below it, so one barrier per
// pivot orders the steps.  A pivot D_j <= tol marks a dependent column: its
// multipliers and 1/sqrt(D_j) are taken as zero, so row j of R and column j
// of R^-1 vanish (Q = Y R^-1 gets a zero column) and the count is recorded.

// Diagonal check of G: returns false (after zeroing R, Rinv and raising
// RSVD_ERR_NONFINITE) on a non-finite diagonal; else the drop tolerance.
template <typename T>
__device__ __forceinline__ bool chol_prologue(const T* __restrict__ G, int64_t ldg, int l,
                                              T* __restrict__ R, T* __restrict__ Rinv,
                                              DeviceStatus* status, T* tol_out) {
  __shared__ T s_maxdiag;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    T mx = T(0);
    int bad = 0;
    for (int j = lane; j < l; j += 32) {
      const T d = G[j + (int64_t)j * ldg];
      if (!isfinite(d)) bad = 1;
      mx = fmax(mx, fabs(d));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      s_maxdiag = mx;
      s_bad = bad;
    }
  }
  __syncthreads();
  if (s_bad) {
    for (int t = tid; t < l * l; t += blockDim.x) {
      R[t] = T(0);
      Rinv[t] = T(0);
    }
    if (tid == 0) set_flag(status, RSVD_ERR_NONFINITE);
    return false;
  }
  *tol_out = Eps<T>::drop_factor(l) * Eps<T>::value * s_maxdiag;
  return true;
}

// 1/D, 1/sqrt(D) and sqrt(D) of a kept pivot.  FP32: rsqrt plus one Newton
// step (y <- y (3 - D y^2) / 2), a few ulp from the rounded values, which the
// elimination's own rounding dominates.  FP64: correctly rounded operations.
__device__ __forceinline__ void pivot_scales(float d, float& invd, float& rs, float& sq) {
  float y = rsqrtf(d);
  y = y * (1.5f - 0.5f * d * y * y);
  rs = y;
  invd = y * y;
  sq = d * y;
}
__device__ __forceinline__ void pivot_scales(double d, double& invd, double& rs, double& sq) {
  sq = sqrt(d);
  rs = 1.0 / sq;
  invd = 1.0 / d;
}

// Step A of the blocked Cholesky, run by one warp: eliminates inside the
// nb x nb diagonal block [p0, p0 + nb)^2 of W.  Lane t holds block column t
// in registers; row j's value at block column r comes from lane r by a
// shuffle, so the pivots run without shared-memory round trips.
template <typename T, int NB>
__device__ __forceinline__ void chol_block_factor(T* __restrict__ W, int ld, int p0, int nb, T tol,
                                                  T* s_invd, T* s_rs, T* s_sq, int* s_def) {
  const int t = threadIdx.x & 31;
  const bool col_ok = t < nb;
  const int c = p0 + t;
  T col[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) col[r] = (col_ok && r < nb) ? W[p0 + r + c * ld] : T(0);
#pragma unroll
  for (int jj = 0; jj < NB; ++jj) {
    if (jj < nb) {
      const T d = __shfl_sync(0xffffffffu, col[jj], jj);
      T invd = T(0), rs = T(0), sq = T(0);
      const bool keep = d > tol;
      if (sizeof(T) == 4 || t == 0) {
        if (keep) pivot_scales(d, invd, rs, sq);
      }
      if (sizeof(T) == 8) invd = __shfl_sync(0xffffffffu, invd, 0);
      // one lane records the pivot (FP32: lane jj, every lane has the scales;
      // FP64: lane 0, which formed them)
      if (t == (sizeof(T) == 4 ? jj : 0)) {
        s_invd[p0 + jj] = invd;
        s_rs[p0 + jj] = rs;
        s_sq[p0 + jj] = sq;
        if (!keep) atomicAdd(s_def, 1);
      }
      const T wj = col[jj];
      // per lane (no branches): t == jj starts column j of L^-1; t < jj updates
      // L^-1 rows below j; t > jj updates the Schur complement rows j < r <= t
#pragma unroll
      for (int r = jj + 1; r < NB; ++r) {
        const T f = __shfl_sync(0xffffffffu, col[jj], r) * invd;   // W[j][p0 + r] * invd
        const T upd = fma(-f, wj, col[r]);
        const bool live = col_ok && r < nb;
        const T nv = (t == jj) ? -f : ((t < jj || r <= t) ? upd : col[r]);
        col[r] = live ? nv : col[r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (col_ok && r < nb) W[p0 + r + c * ld] = col[r];
}

// Blocked variant (FP64, and FP32 beyond l = 160): panels of NB pivots.  W:
// chol_work_elems(l) elements (shared memory when it fits, else global).  Per
// panel P = [p0, p1):
//  A. one warp eliminates inside the NB x NB diagonal block only (lane =
//     block column), leaving D_P, (D L^T)_PP and (L^-1)_PP in place;
//  B. the panel rows' other columns take the panel's row operations:
//     W[P][c] <- (L^-1)_PP W[P][c]  (c < p0: L^-1 part, c >= p1: G part);
//  C. every row below the panel takes all NB pivots at once:
//     W[i][c] -= sum_{j in P} (W[j][i] / D_j) M[j][c]   for c < p1 or c >= i,
//     with M = the panel rows and, inside the block, L^-1's unit diagonal.
// The multiplier of row i for pivot j is read from the final panel row j
// (the Schur complement is symmetric), so the NB pivots commute into one
// rank-NB update.  Two barriers per panel instead of one per pivot.
template <typename T, int NB>
__device__ __forceinline__ void chol_inv_blocked(const T* __restrict__ G, int64_t ldg, int l,
                                                 T* __restrict__ R, T* __restrict__ Rinv,
                                                 T* __restrict__ W, DeviceStatus* status) {
  constexpr int BMAX = 16;  // step B elements per thread: NB * (l - NB) <= BMAX * blockDim.x
  __shared__ T s_invd[RSVD_L_MAX + 32], s_rs[RSVD_L_MAX + 32], s_sq[RSVD_L_MAX + 32];
  __shared__ int s_def;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int ld = chol_ld(l);
  T tol;
  for (int t = tid; t < l * l; t += nt) {
    const int i = t % l, c = t / l;
    W[i + c * ld] = (i <= c) ? G[i + (int64_t)c * ldg] : T(0);
  }
  if (tid == 0) s_def = 0;
  if (!chol_prologue<T>(G, ldg, l, R, Rinv, status, &tol)) return;

  for (int p0 = 0; p0 < l; p0 += NB) {
    const int p1 = (p0 + NB < l) ? p0 + NB : l;
    const int nb = p1 - p0;
    // ---- A: the diagonal block, one warp, lane = block column ----
    if (warp == 0) chol_block_factor<T, NB>(W, ld, p0, nb, tol, s_invd, s_rs, s_sq, &s_def);
    __syncthreads();
    // ---- B: panel rows, columns outside the block ----
    const int nco = l - nb;
    if (nco > 0) {
      T bv[BMAX];
#pragma unroll
      for (int k = 0; k < BMAX; ++k) {
        const int e = tid + k * nt;
        if (e < nb * nco) {
          const int ii = e / nco, cc = e - ii * nco;
          const int c = cc < p0 ? cc : cc + nb, i = p0 + ii;
          T acc = W[i + c * ld];
          for (int r = 0; r < ii; ++r) acc = fma(W[i + (p0 + r) * ld], W[p0 + r + c * ld], acc);
          bv[k] = acc;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BMAX; ++k) {
        const int e = tid + k * nt;
        if (e < nb * nco) {
          const int ii = e / nco, cc = e - ii * nco;
          const int c = cc < p0 ? cc : cc + nb;
          W[p0 + ii + c * ld] = bv[k];
        }
      }
      __syncthreads();
    }
    // ---- C: rows below the panel, rank-nb update ----
    for (int rb = p1; rb < l; rb += 32) {
      const int i = rb + lane;
      T f[NB];
#pragma unroll
      for (int jj = 0; jj < NB; ++jj)
        f[jj] = (jj < nb && i < l) ? W[p0 + jj + i * ld] * s_invd[p0 + jj] : T(0);
      if (i < l) {
        for (int c = warp; c < l; c += nwarps) {
          if (c >= p1 && c < i) continue;   // row i's L^-1 part beyond the panel is still zero
          T acc = T(0);
          if (c >= p0 && c < p1) {          // inside the block: L^-1 with its unit diagonal
            const int jc = c - p0;
#pragma unroll
            for (int jj = 0; jj < NB; ++jj)
              if (jj >= jc && jj < nb)
                acc = fma(f[jj], jj == jc ? T(1) : W[p0 + jj + c * ld], acc);
          } else {
#pragma unroll
            for (int jj = 0; jj < NB; ++jj)
              if (jj < nb) acc = fma(f[jj], W[p0 + jj + c * ld], acc);
          }
          W[i + c * ld] -= acc;
        }
      }
    }
    __syncthreads();
  }

  for (int t = tid; t < l * l; t += nt) {
    const int i = t % l, c = t / l;
    T r = T(0), ri = T(0);
    if (i == c) {
      r = s_sq[i];
      ri = s_rs[i];
    } else if (i < c) {
      r = W[i + c * ld] * s_rs[i];
      ri = W[c + i * ld] * s_rs[c];
    }
    R[t] = r;
    Rinv[t] = ri;
  }
  if (tid == 0 && s_def) atomicAdd(&status->deficient, s_def);
}

// Panel variant: the Cholesky factor and its inverse as separate blocked
// computations, every pass between barriers a small dense product in 4 x 4
// register tiles (about 25 barriers at l = 160, against one per pivot).
// Sizes are padded to lp = 32 ceil(l / 32) with zeros.  W (lp x ld, ld a
// multiple of 4 with ld / 4 odd, so 16-byte accesses down a column or along
// a stride-ld row are conflict-free) holds R in its upper triangle and
// X = R^-1 transposed in its strict lower triangle (X[i][c] at W[c][i]);
// X's diagonal is s_rs.  S (32 x ldt) holds a panel's rows with the column
// index contiguous; Xs / Xt (32 x 36) a diagonal block of X and its
// transpose.  Per panel P = [p0, p0 + 32):
//  a. one warp eliminates [G_PP | I] (chol_block_factor); scaling its result
//     gives R_PP = D^1/2 L^T and X_PP = L^-T D^-1/2;
//  b. R[P][t] = X_PP^T G[P][t] for the later columns t (the panel's rows of R);
//  c. G[t1][t2] -= sum_{k in P} R[k][t1] R[k][t2] for later t1 <= t2.
// Then, panel rows from the last but one up:
//  d. T[i][c] = sum_{p1 <= s <= c} R[p0 + i][s] X[s][c]   (c >= p1 = p0 + 32),
//  e. X[p0 + i][c] = -sum_{k >= i} X_PP[i][k] T[k][c].
// A dropped pivot (D_j <= tol) gives a zero row of R and a zero row and
// column of X, as in the other variants.
__host__ __device__ constexpr int chol_pad(int l) { return (l + 31) / 32 * 32; }
__host__ __device__ constexpr int chol_tld(int l) {
  return (chol_pad(l) / 4) % 2 ? chol_pad(l) : chol_pad(l) + 4;
}
__host__ __device__ constexpr size_t chol_panel_elems(int l) {
  return (size_t)chol_pad(l) * chol_tld(l) + 2 * 32 * (size_t)chol_tld(l) + 2 * 32 * 36;
}



template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// Step a of the panel variant, one warp: the same elimination of
// [G_PP | I] as chol_block_factor, with lane t holding ROW t of the block,
// two pivots per round.  Lanes j and j+1 write their rows to shared memory;
// every lane reads both back (16-byte loads, all issued before the first
// use), forms row j+1 after pivot j itself (the same operations lane j+1
// would do, so every lane has the same bits), and applies both pivots to
// its own row: one shared-memory round trip per two pivots.  buf: 64
// elements of 16-byte aligned shared memory.
template <typename T>
__device__ __forceinline__ void chol_block_rows(T* W, int ld, int p0, int nb, T tol, T* s_invd,
                                                T* s_rs, T* s_sq, int* s_def, T* buf) {
  const int t = threadIdx.x & 31;
  T w[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) w[c] = (t < nb && c < nb) ? W[p0 + t + (p0 + c) * ld] : T(0);
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    if (j < nb) {
      const bool pair = j + 1 < nb;
      if (t == j || t == j + 1) {
        T* dst = buf + (t == j ? 0 : 32);
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          const T v[4] = {w[c], w[c + 1], w[c + 2], w[c + 3]};
          st4(dst + c, v);
        }
      }
      __syncwarp();
      asm volatile("" ::: "memory");   // every lane reloads the new pivot rows
      const T ga = buf[t], gb = buf[32 + t];
      T ra[32], rb[32];
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        T v[4], u[4];
        ld4(buf + c, v);
        ld4(buf + 32 + c, u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ra[c + e] = v[e];
          rb[c + e] = u[e];
        }
      }
      // pivot j
      const T d0 = buf[j];
      T invd0 = T(0), rs0 = T(0), sq0 = T(0);
      const bool keep0 = d0 > tol;
      if (keep0) pivot_scales(d0, invd0, rs0, sq0);
      // row j+1 after pivot j, then pivot j+1
      const T a1 = buf[j + 1];
      const T mlt = a1 * invd0;
#pragma unroll
      for (int c = 0; c < 32; ++c) rb[c] = (c == j) ? -mlt : fma(-mlt, ra[c], rb[c]);
      const T d1 = fma(-mlt, a1, buf[32 + j + 1]);
      T invd1 = T(0), rs1 = T(0), sq1 = T(0);
      const bool keep1 = pair && d1 > tol;
      if (keep1) pivot_scales(d1, invd1, rs1, sq1);
      if (t == j) {
        s_invd[p0 + j] = invd0;
        s_rs[p0 + j] = rs0;
        s_sq[p0 + j] = sq0;
        if (!keep0) atomicAdd(s_def, 1);
      }
      if (t == j + 1 && pair) {
        s_invd[p0 + j + 1] = invd1;
        s_rs[p0 + j + 1] = rs1;
        s_sq[p0 + j + 1] = sq1;
        if (!keep1) atomicAdd(s_def, 1);
#pragma unroll
        for (int c = 0; c < 32; ++c) w[c] = rb[c];
      }
      if (t > j + 1 && t < nb) {
        const T f0 = ga * invd0;
        const T f1 = fma(-mlt, ga, gb) * invd1;   // G[t][j+1] after pivot j, / D_{j+1}
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          if (c < j) w[c] = fma(-f1, rb[c], fma(-f0, ra[c], w[c]));   // L^-1 part
          else if (c == j) w[c] = fma(f1, mlt, -f0);
          else if (c == j + 1) w[c] = -f1;
          else w[c] = (c >= t) ? fma(-f1, rb[c], fma(-f0, ra[c], w[c])) : w[c];
        }
      }
      __syncwarp();
      asm volatile("" ::: "memory");
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (t < nb && c < nb) W[p0 + t + (p0 + c) * ld] = w[c];
}

template <typename T>
__device__ __forceinline__ void chol_inv_panels(const T* __restrict__ G, int64_t ldg, int l,
                                                T* __restrict__ R, T* __restrict__ Rinv,
                                                T* __restrict__ W, DeviceStatus* status) {
  __shared__ T s_invd[RSVD_L_MAX + 32], s_rs[RSVD_L_MAX + 32], s_sq[RSVD_L_MAX + 32];
  __shared__ __align__(16) T s_buf[64];
  __shared__ int s_def;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lp = chol_pad(l), ld = chol_tld(l), ldt = ld;
  T* S = W + (size_t)lp * ld;   // 32 x ldt
  T* Xs = S + 32 * ldt;         // Xs[k * 36 + i] = X_PP[k][i]
  T* Xt = Xs + 32 * 36;         // Xt[k * 36 + i] = X_PP[i][k]
  T tol;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int c = warp; c < lp; c += nwarps) {   // one column per warp, coalesced
#pragma unroll 4
    for (int i = lane; i < lp; i += 32)
      W[i + c * ld] = (i <= c && c < l) ? G[i + (int64_t)c * ldg] : T(0);
  }
  for (int t = tid; t < lp; t += nt) {
    s_invd[t] = T(0);
    s_rs[t] = T(0);
    s_sq[t] = T(0);
  }
  if (tid == 0) s_def = 0;
  if (!chol_prologue<T>(G, ldg, l, R, Rinv, status, &tol)) return;

  // X_PP of the panel at p0 into Xs (k-major) and Xt (transposed)
  auto build_x = [&](int p0) {
    for (int e = tid; e < 32 * 32; e += nt) {
      const int k = e >> 5, i = e & 31;
      T v = T(0);
      if (k < i) v = W[p0 + i + (p0 + k) * ld];
      else if (k == i) v = s_rs[p0 + i];
      Xs[k * 36 + i] = v;   // X_PP[k][i]
      Xt[i * 36 + k] = v;   // Xt[i][k] = X_PP[k][i]
    }
  };

  for (int p0 = 0; p0 < l; p0 += 32) {
    const int nb = min(32, l - p0), p1 = p0 + 32, nt2 = lp - p1;
    // a. the diagonal block
    if (tid < 32) chol_block_rows<T>(W, ld, p0, nb, tol, s_invd, s_rs, s_sq, &s_def, s_buf);
    __syncthreads();
    for (int e = tid; e < nb * nb; e += nt) {
      const int i = e % nb, c = e / nb;
      const int gi = p0 + i, gc = p0 + c;
      if (i != c) W[gi + gc * ld] *= s_rs[gi];   // R_PP above, X_PP^T below
      else W[gi + gc * ld] = s_sq[gi];
    }
    __syncthreads();
    if (nt2 <= 0) break;
    build_x(p0);
    for (int e = tid; e < 32 * nt2; e += nt) {     // G[P][t] with t contiguous
      const int k = e % 32, t = e / 32;
      S[k * ldt + t] = W[p0 + k + (p1 + t) * ld];
    }
    __syncthreads();
    // b. R[P][t] = X_PP^T G[P][t]: tiles (4 rows i, 4 columns t); at most
    //    8 (lp - 32) / 4 <= 2 lp <= 384 tiles, one per thread
    {
      const int ttiles = nt2 / 4, ntile = 8 * ttiles;
      T acc[4][4] = {};
      const int i0 = (tid / ttiles) * 4, t0 = (tid % ttiles) * 4;
      if (tid < ntile) {
        for (int k = 0; k < i0 + 4; ++k) {
          T x[4], g[4];
          ld4(Xs + k * 36 + i0, x);
          ld4(S + k * ldt + t0, g);
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = fma(x[a2], g[b2], acc[a2][b2]);
        }
      }
      __syncthreads();
      if (tid < ntile) {
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) st4(S + (i0 + a2) * ldt + t0, acc[a2]);
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
          T col[4] = {acc[0][b2], acc[1][b2], acc[2][b2], acc[3][b2]};
          st4(W + p0 + i0 + (p1 + t0 + b2) * ld, col);
        }
      }
      __syncthreads();
    }
    // c. trailing upper triangle, tiles (u <= v) of 4 x 4
    {
      const int nt4 = nt2 / 4, ntile = nt4 * (nt4 + 1) / 2;
      for (int tile = tid; tile < ntile; tile += nt) {
        int u = 0, rem = tile;   // row u of the tile triangle holds nt4 - u tiles
        while (rem >= nt4 - u) {
          rem -= nt4 - u;
          ++u;
        }
        const int v = u + rem;
        const int t1 = u * 4, t2 = v * 4;
        T acc[4][4];
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
          T col[4];
          ld4(W + p1 + t1 + (p1 + t2 + b2) * ld, col);
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2) acc[a2][b2] = col[a2];
        }
        for (int k = 0; k < nb; ++k) {
          T r1[4], r2[4];
          ld4(S + k * ldt + t1, r1);
          ld4(S + k * ldt + t2, r2);
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = fma(-r1[a2], r2[b2], acc[a2][b2]);
        }
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
          if (u == v) {   // diagonal tile: the upper part only (W's lower part holds X)
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2)
              if (a2 <= b2) W[p1 + t1 + a2 + (p1 + t2 + b2) * ld] = acc[a2][b2];
          } else {
            T col[4] = {acc[0][b2], acc[1][b2], acc[2][b2], acc[3][b2]};
            st4(W + p1 + t1 + (p1 + t2 + b2) * ld, col);
          }
        }
      }
      __syncthreads();
    }
  }
  // d, e: X's off-diagonal blocks, last panel row first.  Step d's sums run
  // in two halves over s (threads tid and tid + 256 of a tile) into S and
  // S2, which step e adds.
  T* S2 = Xt + 32 * 36;   // 32 x ldt
  for (int p0 = lp - 64; p0 >= 0; p0 -= 32) {
    const int p1 = p0 + 32, nt2 = lp - p1, ctiles = nt2 / 4, ntile = 8 * ctiles;
    build_x(p0);
    // d. T[i][c] = sum_{p1 <= s <= c} R[p0 + i][s] X[s][c]  -> S + S2 (i-major)
    for (int tt = tid; tt < 2 * ntile; tt += nt) {
      const int tile = tt % ntile, half = tt / ntile;
      const int i0 = (tile / ctiles) * 4, c0 = p1 + (tile % ctiles) * 4;
      const int smid = p1 + ((c0 - p1) / 8) * 4;   // the first half's end (a multiple of 4)
      T acc[4][4] = {};
      const int sb = half ? smid : p1, se = half ? c0 : smid;
      for (int s2 = sb; s2 < se; ++s2) {
        T r[4], x[4];
        ld4(W + p0 + i0 + s2 * ld, r);   // R[p0 + i0 + a][s2]
        ld4(W + c0 + s2 * ld, x);        // X[s2][c0 + b]
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = fma(r[a2], x[b2], acc[a2][b2]);
      }
      if (half) {
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {   // s2 = c0 + d2: X[s2][c0 + b] for b >= d2
          const int s2 = c0 + d2;
          T r[4];
          ld4(W + p0 + i0 + s2 * ld, r);
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) {
            const T x = (b2 == d2) ? s_rs[s2] : (b2 > d2 ? W[c0 + b2 + s2 * ld] : T(0));
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) acc[a2][b2] = fma(r[a2], x, acc[a2][b2]);
          }
        }
      }
      T* dst = half ? S2 : S;
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2) st4(dst + (i0 + a2) * ldt + (c0 - p1), acc[a2]);
    }
    __syncthreads();
    // e. X[p0 + i][c] = -sum_k X_PP[i][k] T[k][c]
    for (int tile = tid; tile < ntile; tile += nt) {
      const int i0 = (tile / ctiles) * 4, c0 = p1 + (tile % ctiles) * 4;
      T acc[4][4] = {};
      for (int k = i0; k < 32; ++k) {
        T x[4], t4[4], u4[4];
        ld4(Xt + k * 36 + i0, x);   // X_PP[i0 + a][k]
        ld4(S + k * ldt + (c0 - p1), t4);
        ld4(S2 + k * ldt + (c0 - p1), u4);
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) t4[b2] += u4[b2];
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = fma(x[a2], t4[b2], acc[a2][b2]);
      }
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2) {
        T v[4] = {-acc[a2][0], -acc[a2][1], -acc[a2][2], -acc[a2][3]};
        st4(W + c0 + (p0 + i0 + a2) * ld, v);
      }
    }
    __syncthreads();
  }
  for (int c = warp; c < l; c += nwarps) {
#pragma unroll 4
    for (int i = lane; i < l; i += 32) {
      T r = T(0), ri = T(0);
      if (i == c) {
        r = W[i + i * ld];
        ri = s_rs[i];
      } else if (i < c) {
        r = W[i + c * ld];
        ri = W[c + i * ld];
      }
      R[i + (int64_t)c * l] = r;
      Rinv[i + (int64_t)c * l] = ri;
    }
  }
  if (tid == 0 && s_def) atomicAdd(&status->deficient, s_def);
}

// Whether the panel variant covers (T, l) in shared memory.
template <typename T>
__host__ __device__ constexpr bool chol_panels_fit(int l) {
  return chol_panel_elems(l) * sizeof(T) <= 200 * 1024;
}

// Threads of a blocked-Cholesky CTA (NB * (l - NB) <= 16 * CHOL_THREADS for l <= 288).
constexpr int CHOL_THREADS = 512;

// Panel width of the blocked variant: NB multipliers per thread in step C.
template <typename T>
struct CholPanel {
  static constexpr int value = sizeof(T) == 4 ? 32 : 16;
};

// Register variant (FP32, l <= 32 E): 1024 threads as a 32 x 32 grid;
// thread (tr, tc) = (lane, warp) holds W[tr + 32 a][tc + 32 b] (a, b < E) in
// registers for the whole factorisation.  Row j is published to shared memory
// by its holders at the end of step j - 1, so a step is: read row j at this
// thread's rows (distinct per lane) and columns (one per warp: a broadcast),
// at most E x E multiply-adds, publish row j + 1, one barrier.  Blocks of
// rows that are final are skipped; with eight warps per scheduler the FMA
// and shared-memory latencies are hidden.
constexpr int CHOL_REG_THREADS = 1024;

template <int E>
__device__ __forceinline__ void chol_inv_regs(const float* __restrict__ G, int64_t ldg, int l,
                                              float* __restrict__ R, float* __restrict__ Rinv,
                                              DeviceStatus* status) {
  constexpr int N = 32 * E;
  __shared__ float s_row[2][N];
  __shared__ float s_rs[N], s_sq[N];
  __shared__ int s_def;
  const int tid = threadIdx.x;
  const int tr = tid & 31, tc = tid >> 5;
  const bool diag_upper = tr <= tc;
  float w[E][E];
#pragma unroll
  for (int a = 0; a < E; ++a)
#pragma unroll
    for (int b = 0; b < E; ++b) {
      const int i = tr + 32 * a, c = tc + 32 * b;
      w[a][b] = (i < l && c < l && i <= c) ? G[i + (int64_t)c * ldg] : 0.f;
    }
  if (tid == 0) s_def = 0;
  float tol;
  if (!chol_prologue<float>(G, ldg, l, R, Rinv, status, &tol)) return;
  // publish row 0 (zeros past l)
  if (tr == 0) {
#pragma unroll
    for (int b = 0; b < E; ++b) s_row[0][tc + 32 * b] = w[0][b];
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    const float* row = s_row[j & 1];
    // every thread forms 1/D_j from the published pivot (no divergent
    // divide on the critical path); thread 0 records the scales
    const float d = row[j];
    const bool keep = d > tol;
    float invd = 0.f, rs = 0.f, sq = 0.f;
    if (keep) pivot_scales(d, invd, rs, sq);
    if (tid == 0) {
      s_rs[j] = rs;
      s_sq[j] = sq;
      if (!keep) ++s_def;
    }
    const int a0 = (j + 1) >> 5;            // blocks a < a0 hold only final rows
    float wu[E], wl[E], wd[E];
#pragma unroll
    for (int b = 0; b < E; ++b) {
      const int c = tc + 32 * b;
      wu[b] = row[c];
      wl[b] = (c < j) ? wu[b] : (c == j ? 1.f : 0.f);
      wd[b] = diag_upper ? wu[b] : wl[b];
    }
#pragma unroll
    for (int a = 0; a < E; ++a) {
      if (a < a0) continue;
      const int i = tr + 32 * a;
      const float f = (i > j) ? row[i] * invd : 0.f;
#pragma unroll
      for (int b = 0; b < E; ++b)
        w[a][b] = fmaf(-f, (a < b) ? wu[b] : (a > b ? wl[b] : wd[b]), w[a][b]);
    }
    // publish row j + 1 (its holders are the lanes tr == (j + 1) % 32)
    const int jn = j + 1;
    if (jn < l && tr == (jn & 31)) {
      const int an = jn >> 5;
      float* nrow = s_row[jn & 1];
#pragma unroll
      for (int a = 0; a < E; ++a)
        if (a == an) {
#pragma unroll
          for (int b = 0; b < E; ++b) nrow[tc + 32 * b] = w[a][b];
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < E; ++a)
#pragma unroll
    for (int b = 0; b < E; ++b) {
      const int i = tr + 32 * a, c = tc + 32 * b;
      if (i >= l || c >= l) continue;
      if (i == c) {
        R[i + i * l] = s_sq[i];
        Rinv[i + i * l] = s_rs[i];
      } else if (i < c) {
        R[i + c * l] = w[a][b] * s_rs[i];
        Rinv[c + i * l] = 0.f;
      } else {
        R[i + c * l] = 0.f;
        Rinv[c + i * l] = w[a][b] * s_rs[i];
      }
    }
  if (tid == 0 && s_def) atomicAdd(&status->deficient, s_def);
}

// Block edge of the register variant for l (0: not covered).
__host__ __device__ constexpr int chol_reg_edge(int l) { return l <= 160 ? (l + 31) / 32 : 0; }

// Whether (T, l) takes the register variant.
template <typename T>
__host__ __device__ constexpr bool chol_in_regs(int l) {
  return sizeof(T) == 4 && l <= 160;
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

// Rotation (c, s) that zeroes the cosine of columns p, q with |c_p|^2 = a,
// |c_q|^2 = b, c_p.c_q = g (Rutishauser): zeta = (b - a) / (2g),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t.
// Near convergence the angles are tiny: for |zeta| > Z the same t is
// g / (b - a) to relative 1 / (4 zeta^2) and c = 1 - t^2 / 2 to 3 t^4 / 8,
// both below the rounding unit (Z = 1e8 in FP64, 1e4 in FP32), which saves
// two divisions and two square roots on FP64's slow pipe.
template <typename T>
__device__ __forceinline__ void jacobi_cs(T a, T b, T g, T& c, T& sn) {
  const T d = b - a;
  const T zmax = sizeof(T) == 8 ? T(2e8) : T(2e4);   // 2 Z
  if (fabs(d) > zmax * fabs(g)) {
    const T t = g / d;
    c = fma(T(-0.5) * t, t, T(1));
    sn = c * t;
    return;
  }
  const T zeta = d / (T(2) * g);
  const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
  c = rsqrt(fma(t, t, T(1)));
  sn = c * t;
}

// Threads a Jacobi CTA runs with: P column pairs x G threads per pair, G a
// power of two chosen so that P * G <= JACOBI_THREADS.
constexpr int JACOBI_THREADS = 640;

__host__ __device__ inline int jacobi_group(int l) {
  const int P = ((l + 1) & ~1) / 2;
  int G = 32;
  while (G > 1 && P * G > JACOBI_THREADS) G >>= 1;
  return G;
}

// Column stride of the Jacobi work matrix.  FP32 in shared memory: columns
// padded to a stride of G (mod 32) elements, so the 32/G column pairs a warp
// works on start in distinct banks.  Otherwise l.
template <typename T>
__host__ __device__ inline int jacobi_ld(int l, bool in_smem) {
  const int G = jacobi_group(l);
  if (sizeof(T) != 4 || !in_smem || G == 32) return l;
  return (l + 31) / 32 * 32 + G;
}

// Rows of a column pair a thread keeps in registers across one round (a
// kernel serving only small l takes fewer, and so no spills).
template <typename T>
struct JacobiRegs {
  static constexpr int value = sizeof(T) == 4 ? 20 : 10;
};
// ... for the grouped kernels (l <= 80: 16 threads per pair leave <= 5 rows)
constexpr int JACOBI_REGS_SMALL = 6;

// Work layout: Wm (ldw x twoP) and, if V is accumulated, Wv (ldw x twoP),
// column-major; in dynamic shared memory when they fit, else in `gwork`.
// Round-robin ordering; in one round the G threads of each column pair load
// their rows of both columns (into registers when they fit) and form partial
// |c_p|^2, |c_q|^2, c_p.c_q, butterfly-reduced within the group (every lane
// ends with the same bits: floating addition is commutative).  FP32: every
// lane then derives the same rotation (Rutishauser) and applies it to the rows
// it holds -- one barrier per round.  FP64: the rotation costs tens of FP64
// operations at 2 per clock per SM, so one thread per pair forms it between
// two barriers and the group then applies it.
// GF > 0: the thread group per column pair is GF at compile time (the caller
// guarantees jacobi_group(l) == GF), so a thread's row offsets are constants.
template <typename T, int RMAX = JacobiRegs<T>::value, int GF = 0>
__device__ __forceinline__ void jacobi_body(const T* __restrict__ M, int l, int64_t ldm,
                                            T* __restrict__ sig, T* __restrict__ Um, int64_t ldu,
                                            T* __restrict__ Vm, int64_t ldv,
                                            T* __restrict__ UsInv, T* __restrict__ Wm, int ldw,
                                            DeviceStatus* status) {
  constexpr bool kFused = sizeof(T) == 4;
  const int twoP = (l + 1) & ~1;  // even number of columns (one zero column if l is odd)
  const int P = twoP / 2;
  const bool want_v = Vm != nullptr;
  T* Wv = Wm + (int64_t)ldw * twoP;
  __shared__ int s_rot, s_big;
  __shared__ T s_norm[RSVD_L_MAX + 1];
  __shared__ T s_abg[kFused ? 1 : (RSVD_L_MAX + 1) / 2][3];
  __shared__ T s_cs[kFused ? 1 : (RSVD_L_MAX + 1) / 2][2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  const int G = GF > 0 ? GF : jacobi_group(l);
  const int items = P * G;
  const int R = (l + G - 1) / G;          // rows per thread
  const bool in_regs = R <= RMAX;

  __shared__ T s_fro[32];
  T fro = T(0);
  for (int t = tid; t < l * twoP; t += nt) {
    int i = t % l, j = t / l;
    const T v = (j < l) ? M[i + (int64_t)j * ldm] : T(0);
    Wm[i + (int64_t)j * ldw] = v;
    fro = fma(v, v, fro);
    if (want_v) Wv[i + (int64_t)j * ldw] = (i == j) ? T(1) : T(0);
  }
  if constexpr (GF > 0) {
    // rows l .. G R - 1 of every column are zero, so the fixed-group path
    // reads and rotates them without a bounds test (ldw >= G R)
    const int pad = G * R - l;
    for (int t = tid; t < pad * twoP; t += nt) {
      const int i = l + t % pad, j = t / pad;
      Wm[i + (int64_t)j * ldw] = T(0);
      if (want_v) Wv[i + (int64_t)j * ldw] = T(0);
    }
  }
  fro = warp_sum(fro);
  if (lane == 0) s_fro[warp] = fro;
  if (tid == 0) s_rot = s_big = 0;
  __syncthreads();
  if (tid < 32) {
    T f = tid < nwarps ? s_fro[tid] : T(0);
    f = warp_sum(f);
    if (tid == 0) s_fro[0] = f;
  }
  __syncthreads();
  const T tol = sqrt((T)l) * Eps<T>::value;
  // Jacobi converges quadratically near the end: after a sweep whose largest
  // rotated cosine was below qtol, the next sweep's cosines are of order
  // qtol^2 / (relative gap), below tol, so that sweep would rotate nothing
  // and is skipped
  const T qtol = T(1e-3) * sqrt(tol);
  // a column whose squared norm is below (eps ||M||_F)^2 is numerically zero
  // (a rank-deficient M): pairs with one are left alone, as rotating rounding
  // noise against itself would never meet the relative test
  const T tiny = Eps<T>::value * Eps<T>::value * s_fro[0];
  const int pr = tid / G, sub = tid % G;
  const bool active = tid < items;
  int sweep = 0;
  const int max_sweeps = 30;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < twoP - 1; ++r) {
      int p = 0, q = 0;
      if (active) {
        p = rr_player(pr, r, twoP);
        q = rr_player(twoP - 1 - pr, r, twoP);
        if (p > q) { const int t = p; p = q; q = t; }
      }
      T* cp = Wm + (int64_t)p * ldw;
      T* cq = Wm + (int64_t)q * ldw;
      T x[RMAX], y[RMAX];
      T a = T(0), b = T(0), g = T(0);
      if (active) {
        if (in_regs) {
#pragma unroll
          for (int k = 0; k < RMAX; ++k) {
            const int i = sub + G * k;
            const bool ok = GF > 0 ? k < R : (k < R && i < l);
            x[k] = ok ? cp[i] : T(0);
            y[k] = ok ? cq[i] : T(0);
            a = fma(x[k], x[k], a);
            b = fma(y[k], y[k], b);
            g = fma(x[k], y[k], g);
          }
        } else {
          for (int i = sub; i < l; i += G) {
            const T xv = cp[i], yv = cq[i];
            a = fma(xv, xv, a);
            b = fma(yv, yv, b);
            g = fma(xv, yv, g);
          }
        }
      }
      for (int o = G >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
      }
      // zeta = (b - a) / (2g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
      // c = 1/sqrt(1+t^2), s = c t
      T c = T(1), sn = T(0);
      bool rotate = false;
      if constexpr (kFused) {
        if (active && g != T(0) && fmin(a, b) > tiny && fabs(g) > tol * sqrt(a) * sqrt(b)) {
          jacobi_cs<T>(a, b, g, c, sn);
          rotate = true;
          if (sub == 0) s_rot = 1;
          if (sub == 0 && fabs(g) > qtol * sqrt(a) * sqrt(b)) s_big = 1;
        }
      } else {
        if (active && sub == 0) {
          s_abg[pr][0] = a;
          s_abg[pr][1] = b;
          s_abg[pr][2] = g;
        }
        __syncthreads();
        for (int u = tid; u < P; u += nt) {
          const T ua = s_abg[u][0], ub = s_abg[u][1], ug = s_abg[u][2];
          T uc = T(1), us = T(0);
          if (ug != T(0) && fmin(ua, ub) > tiny && fabs(ug) > tol * sqrt(ua) * sqrt(ub)) {
            jacobi_cs<T>(ua, ub, ug, uc, us);
            s_rot = 1;
            if (fabs(ug) > qtol * sqrt(ua) * sqrt(ub)) s_big = 1;
          }
          s_cs[u][0] = uc;
          s_cs[u][1] = us;
        }
        __syncthreads();
        if (active) {
          c = s_cs[pr][0];
          sn = s_cs[pr][1];
          rotate = sn != T(0);
        }
      }
      if (rotate) {
        if (in_regs) {
#pragma unroll
          for (int k = 0; k < RMAX; ++k) {
            const int i = sub + G * k;
            if (GF > 0 ? k < R : (k < R && i < l)) {
              cp[i] = c * x[k] - sn * y[k];
              cq[i] = sn * x[k] + c * y[k];
            }
          }
        } else {
          for (int i = sub; i < l; i += G) {
            const T xv = cp[i], yv = cq[i];
            cp[i] = c * xv - sn * yv;
            cq[i] = sn * xv + c * yv;
          }
        }
        if (want_v) {
          T* vp = Wv + (int64_t)p * ldw;
          T* vq = Wv + (int64_t)q * ldw;
          for (int i = sub; i < l; i += G) {
            const T xv = vp[i], yv = vq[i];
            vp[i] = c * xv - sn * yv;
            vq[i] = sn * xv + c * yv;
          }
        }
      }
      __syncthreads();
    }
    const int rot = s_rot, big = s_big;
    __syncthreads();
    if (tid == 0) s_rot = s_big = 0;
    __syncthreads();
    if (!rot || !big) break;
  }
  if (tid == 0) {
    status->jacobi_sweeps = sweep + 1;
    if (sweep >= max_sweeps) set_flag(status, RSVD_ERR_JACOBI);
  }
  // column norms
  for (int c = warp; c < l; c += nwarps) {
    const T* cp = Wm + (int64_t)c * ldw;
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
      const T u = Wm[i + (int64_t)c * ldw] * inv;
      Um[i + (int64_t)rank * ldu] = u;
      if (UsInv) UsInv[i + (int64_t)rank * l] = u * inv;
      if (want_v) Vm[i + (int64_t)rank * ldv] = Wv[i + (int64_t)c * ldw];
    }
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi over a cluster of CTAs
// ---------------------------------------------------------------------------
//
// The same rotations as jacobi_body, spread over a thread-block cluster of
// JACOBI_CLUSTER CTAs (distributed shared memory): CTA r holds rows
// [r R, (r+1) R) of every column (R = ceil(l / JACOBI_CLUSTER)).  A round of
// the round-robin ordering:
//   1. each CTA forms the partial |c_p|^2, |c_q|^2, c_p.c_q of every pair over
//      its rows (a warp per pair, lanes over rows) into its own buffer;
//   2. cluster barrier; one thread per pair sums the JACOBI_CLUSTER partials,
//      read from each CTA's buffer in rank order, so every CTA forms the same
//      sums, the same rotation and the same convergence decision;
//   3. each CTA rotates its own rows.
// The partial buffers alternate between rounds, so one cluster barrier per
// round orders both the writes and the reads.  Per CTA, a round moves only
// R rows of each pair through shared memory and the FP64 work of a round is
// split over the cluster's SMs.  A CTA of the cluster never leaves before
// the others (a final cluster barrier): its shared memory is read remotely.
constexpr int JACOBI_CLUSTER = 8;
constexpr int JACOBI_CL_THREADS = 256;

// {a, b, g, 0} to a 16-byte aligned slot (possibly another CTA's), as vectors
__device__ __forceinline__ void store_triple(float* d, float a, float b, float g) {
  *reinterpret_cast<float4*>(d) = make_float4(a, b, g, 0.f);
}
__device__ __forceinline__ void store_triple(double* d, double a, double b, double g) {
  reinterpret_cast<double2*>(d)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(d)[1] = make_double2(g, 0.0);
}

__host__ __device__ inline int jacobi_cluster_rows(int l) {
  return (l + JACOBI_CLUSTER - 1) / JACOBI_CLUSTER;
}
// Shared-memory elements of one CTA: its rows of W (and of V), ld rows + 1.
__host__ __device__ inline size_t jacobi_cluster_elems(int l, bool want_v) {
  const int twoP = (l + 1) & ~1;
  return (size_t)(want_v ? 2 : 1) * (jacobi_cluster_rows(l) + 1) * twoP;
}

template <typename T>
__device__ __forceinline__ void jacobi_cluster_body(const T* __restrict__ M, int l, int64_t ldm,
                                                    T* __restrict__ sig, T* __restrict__ Um,
                                                    int64_t ldu, T* __restrict__ Vm, int64_t ldv,
                                                    T* __restrict__ UsInv, T* __restrict__ Wl,
                                                    DeviceStatus* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int twoP = (l + 1) & ~1;
  const int P = twoP / 2;
  const bool want_v = Vm != nullptr;
  const int R = jacobi_cluster_rows(l);
  const int ld = R + 1;
  const int r0 = rank * R;
  const int nr = max(0, min(l, r0 + R) - r0);
  T* Wv = Wl + (int64_t)ld * twoP;
  // partials pushed by every CTA of the cluster: [round parity][source rank][pair]
  // as {a, b, g, 0}, so one pair costs one (FP32) or two (FP64) 16-byte remote
  // stores per destination (a remote store costs the SM ~1.5 clocks)
  __shared__ __align__(16) T s_part[2][JACOBI_CLUSTER][(RSVD_L_MAX + 1) / 2][4];
  __shared__ T s_cs[(RSVD_L_MAX + 1) / 2][2];
  __shared__ T s_norm[RSVD_L_MAX + 1];
  __shared__ T s_fro[JACOBI_CL_THREADS / 32];
  __shared__ int s_rot, s_big;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;

  T fro = T(0);
  for (int t = tid; t < ld * twoP; t += nt) {
    const int i = t % ld, j = t / ld;
    const T v = (i < nr && j < l) ? M[r0 + i + (int64_t)j * ldm] : T(0);
    Wl[t] = v;
    fro = fma(v, v, fro);
    if (want_v) Wv[t] = (i < nr && r0 + i == j) ? T(1) : T(0);
  }
  fro = warp_sum(fro);
  if (lane == 0) s_fro[warp] = fro;
  if (tid == 0) s_rot = s_big = 0;
  __syncthreads();
  if (tid < JACOBI_CLUSTER) {   // this CTA's share of ||M||_F^2, pushed to CTA tid
    T f = T(0);
    for (int w = 0; w < nwarps; ++w) f += s_fro[w];
    *cluster.map_shared_rank(&s_part[1][rank][0][0], tid) = f;
  }
  cluster.sync();
  T fro_all = T(0);
  for (int q = 0; q < JACOBI_CLUSTER; ++q) fro_all += s_part[1][q][0][0];
  const T tol = sqrt((T)l) * Eps<T>::value;
  // Jacobi converges quadratically near the end: after a sweep whose largest
  // rotated cosine was below qtol, the next sweep's cosines are of order
  // qtol^2 / (relative gap), below tol, so that sweep would rotate nothing
  // and is skipped
  const T qtol = T(1e-3) * sqrt(tol);
  const T tiny = Eps<T>::value * Eps<T>::value * fro_all;

  int par = 0, sweep = 0;
  const int max_sweeps = 30;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < twoP - 1; ++r) {
      // 1. partial dots over this CTA's rows, a thread per pair (no cross-lane
      //    reductions: FP64 additions through shuffles cost the slow pipe)
      for (int pr = tid; pr < P; pr += nt) {
        int p = rr_player(pr, r, twoP), q = rr_player(twoP - 1 - pr, r, twoP);
        if (p > q) { const int t = p; p = q; q = t; }
        const T* cp = Wl + (int64_t)p * ld;
        const T* cq = Wl + (int64_t)q * ld;
        T a = T(0), b = T(0), g = T(0);
        for (int i = 0; i < nr; ++i) {
          const T x = cp[i], y = cq[i];
          a = fma(x, x, a);
          b = fma(y, y, b);
          g = fma(x, y, g);
        }
#pragma unroll
        for (int dst = 0; dst < JACOBI_CLUSTER; ++dst) {   // push into every CTA's buffer
          T* d = cluster.map_shared_rank(&s_part[par][rank][pr][0], dst);
          store_triple(d, a, b, g);
        }
      }
      cluster.sync();
      // 2. the cluster's sums, in rank order, and the rotations
      for (int pr = tid; pr < P; pr += nt) {
        T a = T(0), b = T(0), g = T(0);
#pragma unroll
        for (int q = 0; q < JACOBI_CLUSTER; ++q) {
          a += s_part[par][q][pr][0];
          b += s_part[par][q][pr][1];
          g += s_part[par][q][pr][2];
        }
        T c = T(1), sn = T(0);
        if (g != T(0) && fmin(a, b) > tiny && fabs(g) > tol * sqrt(a) * sqrt(b)) {
          jacobi_cs<T>(a, b, g, c, sn);
          s_rot = 1;
          if (fabs(g) > qtol * sqrt(a) * sqrt(b)) s_big = 1;
        }
        s_cs[pr][0] = c;
        s_cs[pr][1] = sn;
      }
      __syncthreads();
      // 3. rotate this CTA's rows: warps over pairs, lanes over rows
      for (int pr = warp; pr < P; pr += nwarps) {
        const T c = s_cs[pr][0], sn = s_cs[pr][1];
        if (sn == T(0)) continue;
        int p = rr_player(pr, r, twoP), q = rr_player(twoP - 1 - pr, r, twoP);
        if (p > q) { const int t = p; p = q; q = t; }
        T* cp = Wl + (int64_t)p * ld;
        T* cq = Wl + (int64_t)q * ld;
        for (int i = lane; i < nr; i += 32) {
          const T x = cp[i], y = cq[i];
          cp[i] = c * x - sn * y;
          cq[i] = sn * x + c * y;
        }
        if (want_v) {
          T* vp = Wv + (int64_t)p * ld;
          T* vq = Wv + (int64_t)q * ld;
          for (int i = lane; i < nr; i += 32) {
            const T xv = vp[i], yv = vq[i];
            vp[i] = c * xv - sn * yv;
            vq[i] = sn * xv + c * yv;
          }
        }
      }
      par ^= 1;
      // the next round's partials go to the other buffer; the rotations of
      // this round are read only locally, so a CTA barrier suffices
      __syncthreads();
    }
    const int rot = s_rot, big = s_big;   // the same in every CTA (same sums)
    __syncthreads();
    if (tid == 0) s_rot = s_big = 0;
    __syncthreads();
    if (!rot || !big) break;
  }
  if (rank == 0 && tid == 0) {
    status->jacobi_sweeps = sweep + 1;
    if (sweep >= max_sweeps) set_flag(status, RSVD_ERR_JACOBI);
  }
  // every CTA has read the last round's partials before they are overwritten
  cluster.sync();
  // column norms: partial over this CTA's rows, then the cluster's sum
  for (int c = warp; c < l; c += nwarps) {
    const T* cp = Wl + (int64_t)c * ld;
    T a = T(0);
    for (int i = lane; i < nr; i += 32) a = fma(cp[i], cp[i], a);
    a = warp_sum(a);
    if (lane < JACOBI_CLUSTER) *cluster.map_shared_rank(&s_part[0][rank][c >> 1][c & 1], lane) = a;
  }
  cluster.sync();
  for (int c = tid; c < l; c += nt) {
    T a = T(0);
#pragma unroll
    for (int q = 0; q < JACOBI_CLUSTER; ++q) a += s_part[0][q][c >> 1][c & 1];
    s_norm[c] = sqrt(a);
  }
  __syncthreads();
  // sort descending by rank (ties keep column order); write this CTA's rows
  for (int c = warp; c < l; c += nwarps) {
    const T sc = s_norm[c];
    int rk = 0;
    for (int d = lane; d < l; d += 32) {
      const T sd = s_norm[d];
      rk += (sd > sc || (sd == sc && d < c)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    const T inv = sc > T(0) ? T(1) / sc : T(0);
    if (rank == 0 && lane == 0) sig[rk] = sc;
    for (int i = lane; i < nr; i += 32) {
      const T u = Wl[i + (int64_t)c * ld] * inv;
      Um[r0 + i + (int64_t)rk * ldu] = u;
      if (UsInv) UsInv[r0 + i + (int64_t)rk * l] = u * inv;
      if (want_v) Vm[r0 + i + (int64_t)rk * ldv] = Wv[i + (int64_t)c * ld];
    }
  }
  cluster.sync();   // no CTA leaves while another may still read its buffers
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
