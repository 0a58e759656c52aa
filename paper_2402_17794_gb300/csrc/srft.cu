// The subsampled random Fourier transform (SRFT) test matrix and the fast
// randomized range finder built on it (the toolbox's SRFT and FastRandRF,
// Section 4; Algorithm 4.5 of Halko, Martinsson and Tropp 2011), FP64.
//
//   Omega = sqrt(n/l) D F R   (n x l, complex)
//     D  diagonal, d_j = exp(2 pi i u_j)  (u_j: Philox stream 2, counter j)
//     F  the unitary DFT, f_pq = n^-1/2 exp(-2 pi i p q / n)
//     R  l distinct coordinates r_0 < ... < r_{l-1} drawn by Floyd's algorithm
//        (Bentley and Floyd 1987; Philox stream 3, counter = step)
//   Y = A Omega,  Q = orth(Y)
//
// so Y(i, c) = l^-1/2 sum_j A(i, j) d_j exp(-2 pi i j r_c / n).
//
// Complex matrices are stored planar: an m x l complex matrix is the real
// m x 2l matrix [Re | Im] (one leading dimension).  A is real, so the sketch
// is one real product A [Re Omega | Im Omega] (dense form), or the two-level
// FFT of srft_fft.cu.
//
// orth of a complex Y without complex kernels: the complex Cholesky factor
// R of G = Y^H Y (real positive diagonal) realified in interleaved order --
// each entry z as the 2 x 2 block [[Re z, -Im z], [Im z, Re z]] -- is real,
// upper triangular with positive diagonal, and its normal product is the
// realified G.  By uniqueness it IS the real Cholesky factor of the
// realified G.  So each CholeskyQR pass is: the real Gram of [Re Y | Im Y]
// (2l x 2l), G's realification, the real one-CTA Cholesky + inverse, and
// [Re Q | Im Q] = [Re Y | Im Y] [[S_re, S_im], [-S_im, S_re]] with
// S = R^-1 read from the even columns of the real inverse.
#include <algorithm>
#include <cmath>

#include "omega_body.cuh"
#include "pipeline.h"

namespace rsvd {
namespace {

constexpr uint32_t kPhaseStream = 2;
constexpr uint32_t kSampleStream = 3;

// d_j = (cos 2 pi u_j, sin 2 pi u_j), j < n
__global__ void srft_phase_kernel(int64_t n, uint32_t k0, uint32_t k1, double* __restrict__ d_re,
                                  double* __restrict__ d_im) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c0, c1, c2, c3;
    omega::philox10((uint64_t)j, kPhaseStream, k0, k1, c0, c1, c2, c3);
    const double u = omega::uniform52(c0, c1);
    double s, c;
    sincospi(2.0 * u, &s, &c);
    d_re[j] = c;
    d_im[j] = s;
  }
}

// Floyd's sample of l distinct coordinates of [0, n), written ascending to r
// (one warp): step s (j = n-l+s) draws t = min(floor(u_s (j+1)), j) and adds
// t, or j when t is already in the set.
__global__ void srft_sample_kernel(int64_t n, int l, uint32_t k0, uint32_t k1,
                                   int* __restrict__ r) {
  __shared__ int set[RSVD_L_MAX];
  const int lane = threadIdx.x;
  for (int s = 0; s < l; ++s) {
    const int64_t j = n - l + s;
    int t = 0;
    if (lane == 0) {
      uint32_t c0, c1, c2, c3;
      omega::philox10((uint64_t)s, kSampleStream, k0, k1, c0, c1, c2, c3);
      const double u = omega::uniform52(c0, c1);
      const int64_t tt = (int64_t)floor(__dmul_rn(u, (double)(j + 1)));
      t = (int)(tt < j ? tt : j);
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    bool found = false;
    for (int k = lane; k < s; k += 32) found |= (set[k] == t);
    found = __any_sync(0xffffffffu, found);
    if (lane == 0) set[s] = found ? (int)j : t;
    __syncwarp();
  }
  // ascending order: each value goes to its rank (values are distinct)
  for (int a = lane; a < l; a += 32) {
    int rank = 0;
    for (int b = 0; b < l; ++b) rank += set[b] < set[a];
    r[rank] = set[a];
  }
}

// Dense Omega, planar: Om(:, c) = Re, Om(:, l + c) = Im of
// l^-1/2 d_j exp(-2 pi i (j r_c mod n) / n).
__global__ void srft_omega_kernel(int64_t n, int l, const double* __restrict__ d_re,
                                  const double* __restrict__ d_im, const int* __restrict__ r,
                                  double* __restrict__ Om, int64_t ldo) {
  const double scale = rsqrt((double)l);
  const int64_t total = n * (int64_t)l;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const int64_t j = t - (int64_t)c * n;
    const int64_t q = (j * (int64_t)r[c]) % n;
    double s, co;
    sincospi(2.0 * (double)q / (double)n, &s, &co);   // F's entry is co - i s
    const double fr = co, fi = -s;
    Om[j + (int64_t)c * ldo] = scale * (d_re[j] * fr - d_im[j] * fi);
    Om[j + (int64_t)(l + c) * ldo] = scale * (d_re[j] * fi + d_im[j] * fr);
  }
}

// Realification of the complex Gram G = Y^H Y from the real Gram Gr of
// [Re Y | Im Y] (2l x 2l, ld 2l): G_re = Gr11 + Gr22, G_im = Gr12 - Gr21,
// written interleaved: out(2i+a, 2j+b) = [[G_re, -G_im], [G_im, G_re]](a, b).
__global__ void realify_gram_kernel(const double* __restrict__ Gr, int l,
                                    double* __restrict__ out) {
  const int L = 2 * l;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * L; t += gridDim.x * blockDim.x) {
    const int a = t % L, b = t / L;
    const int i = a >> 1, j = b >> 1;
    const double gre = Gr[i + j * L] + Gr[(l + i) + (l + j) * L];
    const double gim = Gr[i + (l + j) * L] - Gr[(l + i) + j * L];
    const int pa = a & 1, pb = b & 1;
    out[t] = (pa == pb) ? gre : (pa ? gim : -gim);
  }
}

// M (2l x 2l, ld 2l) = [[S_re, S_im], [-S_im, S_re]] with S = R^-1 read from
// the even columns of the realified inverse Ri (ld 2l).
__global__ void complex_coef_kernel(const double* __restrict__ Ri, int l, double* __restrict__ M) {
  const int L = 2 * l;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < l * l; t += gridDim.x * blockDim.x) {
    const int i = t % l, j = t / l;
    const double sre = Ri[2 * i + (2 * j) * L];
    const double sim = Ri[(2 * i + 1) + (2 * j) * L];
    M[i + j * L] = sre;
    M[i + (l + j) * L] = sim;
    M[(l + i) + j * L] = -sim;
    M[(l + i) + (l + j) * L] = sre;
  }
}

// M_R (2l x 2l, ld 2l) = the block realification [[M_re, -M_im], [M_im, M_re]]
// of M = R^H, R = Q_B^H Z (l x l complex) read from the real product
// G2 = [Re Q_B | Im Q_B]^T [Re Z | Im Z] (2l x 2l, ld 2l):
// R_re = G2_11 + G2_22, R_im = G2_12 - G2_21.
__global__ void realify_rh_kernel(const double* __restrict__ G2, int l, double* __restrict__ MR) {
  const int L = 2 * l;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * L; t += gridDim.x * blockDim.x) {
    const int a = t % L, b = t / L;
    const int i = a % l, j = b % l;
    // M[i][j] = conj(R[j][i])
    const double mre = G2[j + i * L] + G2[(l + j) + (l + i) * L];
    const double mim = -(G2[j + (l + i) * L] - G2[(l + j) + i * L]);
    const bool top = a < l, left = b < l;
    MR[t] = (top == left) ? mre : (top ? -mim : mim);
  }
}

// The complex singular triplets of M (l x l) from the real SVD of its block
// realification M_R = Xu diag(sig) Xv^T (2l x 2l, ld 2l).  Every singular
// value of M appears twice in M_R, and the two real columns of a pair span
// {z, i z} for a complex singular vector z (column [Re z ; Im z]).  When
// singular values repeat, a real column may instead be any unit vector of
// the combined subspace, so the complex vectors are picked by structure, not
// by position: the real columns are taken in order (sig descending), each
// read as a complex vector x = Xu[:l, c] + i Xu[l:, c] and orthogonalised
// (complex classical Gram-Schmidt, two passes) against the vectors already
// accepted; x is accepted when more than half its unit norm remains (the
// second column of a pair, i z up to rounding, leaves none).  The matching
// right vector y = Xv[:l, c] + i Xv[l:, c] takes the same complex
// coefficients: M y_c = sig_c x_c, and within one value of sig the same
// combination maps the y's to the x's; across distinct values the
// coefficients are rounding-sized.  Outputs: Cu, Cv (2l x 2k, ld 2l) =
// [[X_re, X_im], [-X_im, X_re]] of the accepted vectors, sig_out[k].
// One block; dynamic shared memory (4 l + 2 k + 32) doubles.
__global__ void select_pairs_kernel(const double* __restrict__ Xu, const double* __restrict__ Xv,
                                    const double* __restrict__ sig, int l, int k,
                                    double* __restrict__ Cu, double* __restrict__ Cv,
                                    double* __restrict__ sig_out) {
  const int L = 2 * l;
  extern __shared__ double sh[];
  double *xr = sh, *xi = xr + l, *yr = xi + l, *yi = yr + l, *ar = yi + l, *ai = ar + k;
  double* red = ai + k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int count = 0;
  for (int c = 0; c < L && count < k; ++c) {
    for (int r = tid; r < l; r += blockDim.x) {
      xr[r] = Xu[r + (int64_t)c * L];
      xi[r] = Xu[l + r + (int64_t)c * L];
      yr[r] = Xv[r + (int64_t)c * L];
      yi[r] = Xv[l + r + (int64_t)c * L];
    }
    __syncthreads();
    for (int pass = 0; pass < 2 && count > 0; ++pass) {
      for (int j = warp; j < count; j += nw) {   // alpha_j = z_j^H x
        double sr = 0.0, si = 0.0;
        for (int r = lane; r < l; r += 32) {
          const double zr = Cu[r + (int64_t)j * L], zi = Cu[r + (int64_t)(k + j) * L];
          sr += zr * xr[r] + zi * xi[r];
          si += zr * xi[r] - zi * xr[r];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
          ar[j] = sr;
          ai[j] = si;
        }
      }
      __syncthreads();
      for (int r = tid; r < l; r += blockDim.x) {   // x -= sum alpha_j z_j, y -= sum alpha_j w_j
        double pxr = xr[r], pxi = xi[r], pyr = yr[r], pyi = yi[r];
        for (int j = 0; j < count; ++j) {
          const double a_r = ar[j], a_i = ai[j];
          const double zr = Cu[r + (int64_t)j * L], zi = Cu[r + (int64_t)(k + j) * L];
          const double wr = Cv[r + (int64_t)j * L], wi = Cv[r + (int64_t)(k + j) * L];
          pxr -= a_r * zr - a_i * zi;
          pxi -= a_r * zi + a_i * zr;
          pyr -= a_r * wr - a_i * wi;
          pyi -= a_r * wi + a_i * wr;
        }
        xr[r] = pxr;
        xi[r] = pxi;
        yr[r] = pyr;
        yi[r] = pyi;
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int r = tid; r < l; r += blockDim.x) s2 += xr[r] * xr[r] + xi[r] * xi[r];
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < nw; ++w) tot += red[w];
    if (tot > 0.25) {   // residual norm above 1/2: a new complex direction
      const double inv = 1.0 / sqrt(tot);
      for (int r = tid; r < l; r += blockDim.x) {
        const double a = xr[r] * inv, b = xi[r] * inv, e = yr[r] * inv, f = yi[r] * inv;
        Cu[r + (int64_t)count * L] = a;
        Cu[r + (int64_t)(k + count) * L] = b;
        Cu[(l + r) + (int64_t)count * L] = -b;
        Cu[(l + r) + (int64_t)(k + count) * L] = a;
        Cv[r + (int64_t)count * L] = e;
        Cv[r + (int64_t)(k + count) * L] = f;
        Cv[(l + r) + (int64_t)count * L] = -f;
        Cv[(l + r) + (int64_t)(k + count) * L] = e;
      }
      if (tid == 0) sig_out[count] = sig[c];
      ++count;
    }
    __syncthreads();
  }
}

// One block per triplet i: the phase that makes u_i's largest-magnitude entry
// (lowest row on ties) real and positive is removed from u_i and v_i; then
// V^H's row i is written planar ([Re V^H | Im V^H], ld ldvt) and S_i = sig_i
// (the singular values of the selected pairs).
// U: m x 2k planar (ld ldu), V: n x 2k planar (ld n).
__global__ void finalize_complex_kernel(double* __restrict__ U, int64_t m, int64_t ldu, int k,
                                        const double* __restrict__ V, int64_t n,
                                        const double* __restrict__ sig, double* __restrict__ S,
                                        double* __restrict__ VT, int64_t ldvt) {
  const int i = blockIdx.x;
  double* ure = U + (int64_t)i * ldu;
  double* uim = U + (int64_t)(k + i) * ldu;
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double best = -1.0;
  int64_t bidx = 0;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
    const double v = hypot(ure[r], uim[r]);
    if (v > best) {
      best = v;
      bidx = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bidx;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double o = sv[threadIdx.x + h];
      const int64_t oi = si[threadIdx.x + h];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double a = hypot(ure[si[0]], uim[si[0]]);
  const double pr = a > 0.0 ? ure[si[0]] / a : 1.0, pi = a > 0.0 ? uim[si[0]] / a : 0.0;
  __syncthreads();   // every thread has read the pivot entry before it changes
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {   // u <- u conj(ph)
    const double xr = ure[r], xi = uim[r];
    ure[r] = xr * pr + xi * pi;
    uim[r] = xi * pr - xr * pi;
  }
  const double* vre = V + (int64_t)i * n;
  const double* vim = V + (int64_t)(k + i) * n;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {   // (V^H)_ij = ph conj(v_j)
    const double vr = vre[j], vi = vim[j];
    VT[i + j * ldvt] = pr * vr + pi * vi;
    VT[i + (n + j) * ldvt] = pi * vr - pr * vi;
  }
  if (threadIdx.x == 0) S[i] = sig[i];
}

}  // namespace

int srft_setup(rsvd_plan_t P, int64_t n, int l, uint64_t seed, double* d_re, double* d_im,
               int* r) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)P->num_sms * 4);
  srft_phase_kernel<<<blocks, 256, 0, P->stream>>>(n, k0, k1, d_re, d_im);
  note_launch();
  RSVD_CK(cudaGetLastError());
  srft_sample_kernel<<<1, 32, 0, P->stream>>>(n, l, k0, k1, r);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

int srft_sketch_dense(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                      const double* d_re, const double* d_im, const int* r, double* Y,
                      int64_t ldy) {
  Work<double> W = work_of<double>(P);
  const int64_t total = n * (int64_t)l;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)P->num_sms * 8);
  srft_omega_kernel<<<blocks, 256, 0, P->stream>>>(n, l, d_re, d_im, r, W.om, n);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return gemm<double>(P, A, lda, false, W.om, n, Y, ldy, m, n, 2 * l);
}

int srft_sketch(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                const double* d_re, const double* d_im, const int* r, double* Y, int64_t ldy) {
  if (srft_fft_supported(n, l)) return srft_sketch_fft(P, A, m, n, lda, l, d_re, d_im, r, Y, ldy);
  return srft_sketch_dense(P, A, m, n, lda, l, d_re, d_im, r, Y, ldy);
}

int orth_complex(rsvd_plan_t P, const double* Y, int64_t rows, int l, int64_t ldy, double* Q,
                 int64_t ldq) {
  Work<double> W = work_of<double>(P);
  DeviceStatus* st = dstatus(P);
  const int L = 2 * l;
  int rc;
  const double* src = Y;
  int64_t lds = ldy;
  for (int pass = 0; pass < 2; ++pass) {
    if ((rc = gram<double>(P, src, lds, rows, L, W.G))) return rc;
    realify_gram_kernel<<<(L * L + 255) / 256, 256, 0, P->stream>>>(W.G, l, W.Mt);
    note_launch();
    RSVD_CK(cudaGetLastError());
    RSVD_CK(launch_chol_inv<double>(W.Mt, L, L, W.R1, W.R1i, W.cholw, st, P->stream));
    complex_coef_kernel<<<(l * l + 255) / 256, 256, 0, P->stream>>>(W.R1i, l, W.Um);
    note_launch();
    RSVD_CK(cudaGetLastError());
    double* dst = pass == 0 ? W.tmp : Q;
    const int64_t ldd = pass == 0 ? rows : ldq;
    if ((rc = gemm<double>(P, src, lds, false, W.Um, L, dst, ldd, rows, L, L))) return rc;
    src = dst;
    lds = ldd;
  }
  return RSVD_OK;
}

int range_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
               uint64_t seed, double* Q, int64_t ldq) {
  Work<double> W = work_of<double>(P);
  double* d_re = W.qb;
  double* d_im = W.qb + n;
  int* r = (int*)W.z;
  int rc;
  if ((rc = srft_setup(P, n, l, seed, d_re, d_im, r))) return rc;
  if ((rc = srft_sketch(P, A, m, n, lda, l, d_re, d_im, r, W.y, m))) return rc;
  return orth_complex(P, W.y, m, l, m, Q, ldq);
}

int solve_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int k, int p,
               uint64_t seed, double* U, int64_t ldu, double* S, double* VT, int64_t ldvt) {
  Work<double> W = work_of<double>(P);
  const int l = k + p, L = 2 * l;
  cudaStream_t st = P->stream;
  int rc;
  // FastRandRF: Q (m x l complex, planar) in W.qm
  if ((rc = range_srft(P, A, m, n, lda, l, seed, W.qm, m))) return rc;
  // B^H = A^T Q (A real): one real product with the 2l planar columns
  if ((rc = gemm<double>(P, A, lda, true, W.qm, m, W.z, n, n, m, L))) return rc;
  // B^H = Q_B R_B (complex CholeskyQR2), R_B = Q_B^H B^H
  if ((rc = orth_complex(P, W.z, n, l, n, W.qb, n))) return rc;
  if ((rc = gemm<double>(P, W.qb, n, true, W.z, n, W.G, L, L, n, L))) return rc;
  // R_B^H = U~ S W^H through the realified 2l x 2l matrix: each singular
  // value appears twice; the complex triplets are selected by structure
  realify_rh_kernel<<<(L * L + 255) / 256, 256, 0, st>>>(W.G, l, W.Mt);
  note_launch();
  RSVD_CK(cudaGetLastError());
  RSVD_CK(launch_jacobi_svd<double>(W.Mt, L, L, W.sig, W.Um, L, W.Vm, L, nullptr, W.jw, dstatus(P),
                                    st));
  const size_t sel_smem = (size_t)(4 * l + 2 * k + 32) * sizeof(double);
  select_pairs_kernel<<<1, 256, sel_smem, st>>>(W.Um, W.Vm, W.sig, l, k, W.R1, W.R2, W.sign);
  note_launch();
  RSVD_CK(cudaGetLastError());
  // U = Q U~ (into U, planar), V = Q_B W (into W.tmp, planar)
  if ((rc = gemm<double>(P, W.qm, m, false, W.R1, L, U, ldu, m, L, 2 * k))) return rc;
  if ((rc = gemm<double>(P, W.qb, n, false, W.R2, L, W.tmp, n, n, L, 2 * k))) return rc;
  finalize_complex_kernel<<<k, 256, 0, st>>>(U, m, ldu, k, W.tmp, n, W.sign, S, VT, ldvt);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

int sketch_srft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                uint64_t seed, double* Y, int64_t ldy) {
  Work<double> W = work_of<double>(P);
  double* d_re = W.qb;
  double* d_im = W.qb + n;
  int* r = (int*)W.z;
  int rc;
  if ((rc = srft_setup(P, n, l, seed, d_re, d_im, r))) return rc;
  return srft_sketch(P, A, m, n, lda, l, d_re, d_im, r, Y, ldy);
}

}  // namespace rsvd
