// The SRFT sketch Y = A Omega through the FFT, FP64, for n a multiple of 64.
//
// Row i of the sketch is the DFT of x_j = A(i, j) d_j sampled at l
// frequencies r_c (Omega = sqrt(n/l) D F R, so Y = l^-1/2 (x F~)(:, r) with
// F~ the unnormalised DFT, w = exp(-2 pi i / n)).  With n = 64 n2,
// j = n2 j1 + j2 and r = r1 + 64 r2:
//
//   Y(i, c) = l^-1/2 sum_{j2} w^{j2 r_c} Z_i(j2, r_c mod 64),
//   Z_i(j2, r1) = sum_{j1 < 64} x_{n2 j1 + j2} exp(-2 pi i j1 r1 / 64)
//
// i.e. n2 FFTs of length 64 per row (over columns n2 apart), then, for each
// of the l samples, one complex multiply-add per j2 with the twiddle
// w^{j2 r_c} (a table of n2 x l entries built once).  That is about
// 5 n log2 64 + 8 n l / 64 real operations per row, against 4 n l for the
// dense complex product -- at l = 80, 30 instead of 320 per element of A.
// On GB300 FP64 runs at 2 operations per clock per SM and A streams at
// ~6.8 TB/s, so the kernel is bound by the FP64 pipe, not by HBM.
//
// One CTA = 32 rows (one per lane: every column access is one 256-byte
// segment) x a range of j2; warp w holds the 8 inputs j1 = 8a + w
// (a < 8) of its lane's row.  The length-64 FFT is 8 x 8: an 8-point DFT
// over a in registers, the twiddle exp(-2 pi i w k1 / 64), a transpose
// through shared memory, an 8-point DFT over the other index.  Warp w then
// owns Z(j2, r1) for r1 = w + 8 k2 and updates the accumulators (shared
// memory, l x 32 complex) of the samples with r_c = w (mod 8).  The next
// j2's inputs are loaded before the current one is transformed.
#include <algorithm>
#include <cmath>

#include "pipeline.h"

namespace rsvd {
namespace {

constexpr int kRows = 32;      // rows per CTA (one per lane)
constexpr int kThreads = 256;  // 8 warps

__device__ __forceinline__ void dft4(double& r0, double& i0, double& r1, double& i1, double& r2,
                                     double& i2, double& r3, double& i3) {
  const double s0r = r0 + r2, s0i = i0 + i2;
  const double s1r = r0 - r2, s1i = i0 - i2;
  const double s2r = r1 + r3, s2i = i1 + i3;
  const double s3r = i1 - i3, s3i = r3 - r1;   // (p1 - p3) * (-i)
  r0 = s0r + s2r; i0 = s0i + s2i;
  r1 = s1r + s3r; i1 = s1i + s3i;
  r2 = s0r - s2r; i2 = s0i - s2i;
  r3 = s1r - s3r; i3 = s1i - s3i;
}

// In place: X_k = sum_a x_a exp(-2 pi i a k / 8) (decimation in frequency).
__device__ __forceinline__ void dft8(double (&xr)[8], double (&xi)[8]) {
  const double h = 0.70710678118654752440;
  double ar[4], ai[4], br[4], bi[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ar[a] = xr[a] + xr[a + 4];
    ai[a] = xi[a] + xi[a + 4];
    br[a] = xr[a] - xr[a + 4];
    bi[a] = xi[a] - xi[a + 4];
  }
  {  // x exp(-i pi/4)
    const double t = br[1];
    br[1] = h * (t + bi[1]);
    bi[1] = h * (bi[1] - t);
  }
  {  // x (-i)
    const double t = br[2];
    br[2] = bi[2];
    bi[2] = -t;
  }
  {  // x exp(-3 i pi/4)
    const double t = br[3];
    br[3] = h * (bi[3] - t);
    bi[3] = -h * (t + bi[3]);
  }
  dft4(ar[0], ai[0], ar[1], ai[1], ar[2], ai[2], ar[3], ai[3]);
  dft4(br[0], bi[0], br[1], bi[1], br[2], bi[2], br[3], bi[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xr[2 * k] = ar[k];
    xi[2 * k] = ai[k];
    xr[2 * k + 1] = br[k];
    xi[2 * k + 1] = bi[k];
  }
}

// dft8 of x_a = v_a (cr_a + i ci_a) for real v: the phase products are
// folded into the first butterflies (x_a +- x_{a+4} by one multiply and two
// fused multiply-adds per component).
__device__ __forceinline__ void dft8_phased(const double (&v)[8], const double (&cr)[8],
                                            const double (&ci)[8], double (&xr)[8],
                                            double (&xi)[8]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double pr = v[a] * cr[a], pi = v[a] * ci[a];
    xr[a] = fma(v[a + 4], cr[a + 4], pr);
    xi[a] = fma(v[a + 4], ci[a + 4], pi);
    xr[a + 4] = fma(-v[a + 4], cr[a + 4], pr);
    xi[a + 4] = fma(-v[a + 4], ci[a + 4], pi);
  }
  const double h = 0.70710678118654752440;
  double ar[4], ai[4], br[4], bi[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ar[a] = xr[a];
    ai[a] = xi[a];
    br[a] = xr[a + 4];
    bi[a] = xi[a + 4];
  }
  {
    const double t = br[1];
    br[1] = h * (t + bi[1]);
    bi[1] = h * (bi[1] - t);
  }
  {
    const double t = br[2];
    br[2] = bi[2];
    bi[2] = -t;
  }
  {
    const double t = br[3];
    br[3] = h * (bi[3] - t);
    bi[3] = -h * (t + bi[3]);
  }
  dft4(ar[0], ai[0], ar[1], ai[1], ar[2], ai[2], ar[3], ai[3]);
  dft4(br[0], bi[0], br[1], bi[1], br[2], bi[2], br[3], bi[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xr[2 * k] = ar[k];
    xi[2 * k] = ai[k];
    xr[2 * k + 1] = br[k];
    xi[2 * k + 1] = bi[k];
  }
}

__device__ __forceinline__ double pick8(const double (&v)[8], int k) {
  double x = v[0];
#pragma unroll
  for (int t = 1; t < 8; ++t) x = (k == t) ? v[t] : x;
  return x;
}

// Shared memory (doubles): transpose 2 x 8 x 8 x 32, accumulators 2 x l x 32,
// twiddles of the length-64 FFT 2 x 64; then ints: class lists 8 x l, the
// k2 of every sample (l), class counts (8).
__host__ __device__ inline size_t fft_smem_bytes(int l) {
  return sizeof(double) * (2 * 64 * kRows + 2 * (size_t)l * kRows + 2 * 64) +
         sizeof(int) * (8 * (size_t)l + l + 8);
}

__global__ void __launch_bounds__(kThreads)
srft_fft_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n, int l,
                const double* __restrict__ d_re, const double* __restrict__ d_im,
                const int* __restrict__ r, const double2* __restrict__ tw, int64_t j2_per_cta,
                double* __restrict__ out, int64_t ldo, int64_t out_split_stride, double scale) {
  extern __shared__ __align__(16) double fsm[];
  double* s_re = fsm;                        // [k1][b][lane]
  double* s_im = s_re + 64 * kRows;
  double* acc_re = s_im + 64 * kRows;        // [c][lane]
  double* acc_im = acc_re + (size_t)l * kRows;
  double* w64_re = acc_im + (size_t)l * kRows;
  double* w64_im = w64_re + 64;
  int* cls = reinterpret_cast<int*>(w64_im + 64);   // [w][idx]
  int* k2c = cls + 8 * l;
  int* cnt = k2c + l;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n2 = n / 64;
  const int64_t row = (int64_t)blockIdx.x * kRows + lane;
  const bool live = row < m;
  const int64_t j2_begin = (int64_t)blockIdx.y * j2_per_cta;
  const int64_t j2_end = min(n2, j2_begin + j2_per_cta);

  for (int t = threadIdx.x; t < 64; t += kThreads) {
    double s, c;
    sincospi(-(double)t / 32.0, &s, &c);   // exp(-2 pi i t / 64)
    w64_re[t] = c;
    w64_im[t] = s;
  }
  for (int t = threadIdx.x; t < l * kRows; t += kThreads) {
    acc_re[t] = 0.0;
    acc_im[t] = 0.0;
  }
  // class lists: warp w collects the samples with r_c = w (mod 8), ascending
  {
    int base = 0;
    for (int c0 = 0; c0 < l; c0 += 32) {
      const int c = c0 + lane;
      const bool mine = c < l && (r[c] & 7) == w;
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      if (mine) {
        cls[w * l + base + __popc(bal & ((1u << lane) - 1u))] = c;
        k2c[c] = (r[c] & 63) >> 3;
      }
      base += __popc(bal);
    }
    if (lane == 0) cnt[w] = base;
  }
  __syncthreads();

  // inputs of one j2: x_a = A(row, n2 (8a + w) + j2) d_j
  double nr[8];
  auto load = [&](int64_t j2) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t j = n2 * (8 * a + w) + j2;
      nr[a] = live ? A[row + j * lda] : 0.0;
    }
  };
  if (j2_begin < j2_end) load(j2_begin);
  const int my_cnt = cnt[w];
  for (int64_t j2 = j2_begin; j2 < j2_end; ++j2) {
    double xr[8], xi[8], v[8], dr[8], di[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t j = n2 * (8 * a + w) + j2;
      dr[a] = __ldg(d_re + j);
      di[a] = __ldg(d_im + j);
      v[a] = nr[a];
    }
    if (j2 + 1 < j2_end) load(j2 + 1);
    // pass 1: DFT over a of A d, twiddle exp(-2 pi i w k1 / 64) (1 at
    // k1 = 0), transpose
    dft8_phased(v, dr, di, xr, xi);
    s_re[w * kRows + lane] = xr[0];
    s_im[w * kRows + lane] = xi[0];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
      const double cr = w64_re[w * k1], ci = w64_im[w * k1];
      const double ur = fma(xr[k1], cr, -xi[k1] * ci);
      const double ui = fma(xr[k1], ci, xi[k1] * cr);
      s_re[(k1 * 8 + w) * kRows + lane] = ur;
      s_im[(k1 * 8 + w) * kRows + lane] = ui;
    }
    __syncthreads();
    // pass 2: k1 = w, DFT over b gives Z(r1 = w + 8 k2)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      xr[b] = s_re[(w * 8 + b) * kRows + lane];
      xi[b] = s_im[(w * 8 + b) * kRows + lane];
    }
    dft8(xr, xi);
    // the samples of class w: acc(c) += w^{j2 r_c} Z(r_c mod 64)
    const double2* twr = tw + j2 * l;
    for (int s = 0; s < my_cnt; ++s) {
      const int c = cls[w * l + s];
      const int k2 = k2c[c];
      const double zr = pick8(xr, k2), zi = pick8(xi, k2);
      const double2 t = twr[c];
      const int at = c * kRows + lane;
      acc_re[at] = fma(t.x, zr, fma(-t.y, zi, acc_re[at]));
      acc_im[at] = fma(t.x, zi, fma(t.y, zr, acc_im[at]));
    }
    __syncthreads();
  }
  // planar output (or this CTA's split slice), scaled by l^-1/2
  if (!live) return;
  double* o = out + (int64_t)blockIdx.y * out_split_stride;
  for (int c = w; c < l; c += 8) {
    o[row + (int64_t)c * ldo] = scale * acc_re[c * kRows + lane];
    o[row + (int64_t)(l + c) * ldo] = scale * acc_im[c * kRows + lane];
  }
}

// tw(j2, c) = exp(-2 pi i (j2 r_c mod n) / n), n2 x l, index j2 * l + c
__global__ void srft_twiddle_kernel(int64_t n, int l, const int* __restrict__ r,
                                    double2* __restrict__ tw) {
  const int64_t n2 = n / 64;
  const int64_t total = n2 * l;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j2 = t / l;
    const int c = (int)(t - j2 * l);
    const int64_t q = (j2 * (int64_t)r[c]) % n;
    double s, co;
    sincospi(-2.0 * (double)q / (double)n, &s, &co);
    tw[t] = make_double2(co, s);
  }
}

// Y = sum over the split slices, in slice order (ld m for the slices).
__global__ void srft_split_reduce_kernel(const double* __restrict__ part, int splits,
                                         int64_t stride, int64_t m, int cols,
                                         double* __restrict__ Y, int64_t ldy) {
  const int64_t total = m * (int64_t)cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / m, i = t - c * m;
    double s = 0.0;
    for (int p = 0; p < splits; ++p) s += part[p * stride + t];
    Y[i + c * ldy] = s;
  }
}

}  // namespace

bool srft_fft_supported(int64_t n, int l) {
  return n % 64 == 0 && n >= 64 && l >= 1 &&
         fft_smem_bytes(l) <= dynamic_smem_cap((const void*)srft_fft_kernel);
}

int srft_sketch_fft(rsvd_plan_t P, const double* A, int64_t m, int64_t n, int64_t lda, int l,
                    const double* d_re, const double* d_im, const int* r, double* Y,
                    int64_t ldy) {
  if (!srft_fft_supported(n, l)) return RSVD_ERR_UNSUPPORTED;
  Work<double> W = work_of<double>(P);
  const int64_t n2 = n / 64;
  double2* tw = reinterpret_cast<double2*>(W.om);   // n2 x l entries (W.om holds n x l_max)
  {
    const int64_t total = n2 * l;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)P->num_sms * 4);
    srft_twiddle_kernel<<<blocks, 256, 0, P->stream>>>(n, l, r, tw);
    note_launch();
    RSVD_CK(cudaGetLastError());
  }
  // Split the j2 range so that the CTAs fill whole waves: the split with
  // the best fraction of busy CTA slots (ties to fewer splits), since every
  // CTA does the same work.
  const int64_t row_tiles = (m + kRows - 1) / kRows;
  const size_t slice = (size_t)m * 2 * l;
  const size_t smem = fft_smem_bytes(l);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srft_fft_kernel, kThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t slots = (int64_t)P->num_sms * per_sm;
  const int64_t max_splits =
      std::max<int64_t>(1, std::min<int64_t>({n2, 16, (int64_t)(W.part_elems / slice)}));
  int64_t splits = 1;
  double best = 0.0;
  for (int64_t s = 1; s <= max_splits; ++s) {
    const int64_t per_s = (n2 + s - 1) / s;
    const int64_t eff_s = (n2 + per_s - 1) / per_s;
    const int64_t ctas = row_tiles * eff_s;
    const int64_t waves = (ctas + slots - 1) / slots;
    // busy fraction, discounted by the work imbalance of uneven j2 ranges
    const double fill = (double)ctas / (double)(waves * slots) * (double)n2 /
                        (double)(per_s * eff_s);
    if (fill > best + 0.02) {
      best = fill;
      splits = eff_s;
    }
  }
  const int64_t per = (n2 + splits - 1) / splits;
  splits = (n2 + per - 1) / per;
  dim3 grid((unsigned)row_tiles, (unsigned)splits);
  const double scale = 1.0 / std::sqrt((double)l);
  if (splits == 1) {
    srft_fft_kernel<<<grid, kThreads, smem, P->stream>>>(A, lda, m, n, l, d_re, d_im, r, tw, per,
                                                         Y, ldy, 0, scale);
    note_launch();
    RSVD_CK(cudaGetLastError());
    return RSVD_OK;
  }
  srft_fft_kernel<<<grid, kThreads, smem, P->stream>>>(A, lda, m, n, l, d_re, d_im, r, tw, per,
                                                       W.part, m, (int64_t)slice, scale);
  note_launch();
  RSVD_CK(cudaGetLastError());
  const int64_t total = (int64_t)slice;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)P->num_sms * 8);
  srft_split_reduce_kernel<<<blocks, 256, 0, P->stream>>>(W.part, (int)splits, (int64_t)slice, m,
                                                          2 * l, Y, ldy);
  note_launch();
  RSVD_CK(cudaGetLastError());
  return RSVD_OK;
}

}  // namespace rsvd
