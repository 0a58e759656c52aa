// FP64-accurate passes over A on the tcgen05 tensor cores: Y = A X and
// Z = A^T X for FP64 A and X, the products that carry the cost of the
// randomized SVD (the tau_A (k+p) terms of Section 3.1.1) in Algorithms 2-6.
// They are computed as exact sums of products of BF16 digit slices: the
// error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59,
// 2012), taken to integer digits so that the tensor cores' FP32 accumulation
// never rounds the leading terms.
//
// Digits.  Row i of A gets the exponent r_i with |a_ij| < 2^r_i for all j.
// Each element is written a_ij = 2^r_i (sum_{s<6} d_s 2^(-7-8s) + rho) with
// balanced base-256 integer digits |d_s| <= 128 (the last one rounded to
// nearest), so |rho| <= 2^-48.  Every digit is exact in BF16.  Column c of
// the operand X gets the exponent f_c and digits e_t the same way, after its
// rows are scaled by 2^r_k when the pass contracts over A's rows (A^T X), so
// that each output has one exponent: Y_ic = 2^(r_i + f_c - 14) sum_{s,t}
// 2^(-8(s+t)) sum_j d_s(i,j) e_t(j,c), and Z_jc = 2^(f_c - 14) (...).  A's six
// slices are built once per A (12 bytes per element); X's once per pass.
//
// Products.  The product of slices s and t is an integer sum of terms
// |d_s e_t| <= 2^14 of weight 2^(-8g), g = s + t.  Products of equal weight
// share one TMEM accumulator region of W = l rounded up to 16 columns; the
// 15 products of weight g >= 6 are dropped (at most 5 * 2^-48 relative to
// 2^(r_i + f_c) per term).  One tcgen05.mma multiplies A slice s with several
// X slices that sit side by side in shared memory (N = count * W <= 256),
// its result landing in consecutive regions.  Regions 0-3 are kept exact: in
// 256 contraction elements (4 k-blocks) region g <= 3 collects at most
// (g + 1) * 256 * 2^14 <= 2^24 in integer units, which FP32 holds exactly;
// so they are drained every 4 k-blocks into 64-bit integers in the
// epilogue's registers (T = sum 2^(8(3-g)) G_g) and restarted.  Regions 4-5
// (weight <= 2^-32 of the leading one) accumulate in FP32 over the whole
// tile; their rounding is below 2^-50 of the output scale.
//
// Error.  Per output, |computed - exact| <= (2 * 2^-48 + 5 * 2^-48 + 2^-50)
// * K * 2^(r_i + f_c) in the worst case (K the contraction length), i.e.
// within about 2^-45 K max_j |a_ij| max_j |x_jc|; with errors of random sign
// the observed error is near 2^-45 sqrt(K) of that scale.
//
// Kernel.  Persistent stream-K over (tile of 128 output rows, k-block of 64)
// as in the BF16 pass.  Warp 0 issues TMA: per k-block the six X slices
// (6 * W rows x 64, 128-byte swizzle) into one of two X buffers and the six
// A slices (128 x 64 each) into a ring of six 16 KB buffers.  One lane of
// warp 1 issues the MMAs, slice by slice, releasing each A buffer as soon
// as its products are done.  Warps 2-13 drain: each owns 32 TMEM lanes and
// a third of the W columns.  Outputs leave as raw (int64 T, FP32 R) pairs; a
// second kernel sums the split tiles' partials and forms the FP64 value.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "umma.h"
#include "umma_ptx.cuh"

namespace rsvd {
namespace {

constexpr int TC_S = 6;          // digits per operand
constexpr int TC_BM = 128;       // output rows per tile
constexpr int TC_BK = 64;        // contraction per k-block (one 128-byte swizzle row)
constexpr int TC_CHUNK = 4;      // k-blocks between drains of the exact regions
constexpr int TC_EXACT = 4;      // regions 0..3 exact
constexpr int TC_EPI = 12;       // epilogue warps (3 per TMEM lane quadrant): 14 warps in all,
                                 // at most 4 per SM sub-partition, so up to 128 registers each
constexpr int TC_THREADS = 32 * (2 + TC_EPI);
constexpr int A_SLAB = TC_BM * TC_BK * 2;   // one A slice of one k-block: 16 KB
constexpr int TC_MAX_MMA = 16;

// RSVD_ERR_CUDA after a failed step; with RSVD_DEBUG set in the environment
// the step and the CUDA error are printed to stderr.
int cuda_fail(const char* step, cudaError_t e) {
  if (std::getenv("RSVD_DEBUG"))
    std::fprintf(stderr, "rsvd: %s failed: %s\n", step,
                 e == cudaSuccess ? "tensor map encoding" : cudaGetErrorString(e));
  return RSVD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Digits
// ---------------------------------------------------------------------------

// Balanced base-256 digits of a * 2^(7 - e) (|a| < 2^e): six integers in
// [-128, 128] with a * 2^(7-e) = sum_s d_s 2^(-8s) + rho, |rho| <= 2^-41.
// Integer work only: the 53-bit significand is shifted to 40 fraction bits
// (rounded to nearest) and cut into bytes from the bottom up.
__device__ __forceinline__ void digits6(double a, int e, float (&d)[TC_S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = bits & ((1ull << 52) - 1);
  if (E != 0) M |= 1ull << 52;
  else E = 1;                                   // subnormal: no implicit bit
  // |a| = M 2^(E - 1075); W = round(|a| 2^(47 - e)) = round(M 2^-(1028 + e - E))
  const int sh = 1028 + e - E;
  unsigned long long W;
  if (M == 0 || sh >= 64) W = 0;
  else if (sh <= 0) W = M << (-sh);             // not reached when |a| < 2^e
  else W = (M + (1ull << (sh - 1))) >> sh;
  long long w = (bits >> 63) ? -(long long)W : (long long)W;
#pragma unroll
  for (int s = TC_S - 1; s >= 1; --s) {
    const int lo = (int)((w + 128) & 255) - 128;
    d[s] = (float)lo;
    w = (w - lo) >> 8;
  }
  d[0] = (float)w;
}

// Biased exponent field of |a| (0 for zero and subnormals); 2047 for Inf/NaN.
__device__ __forceinline__ int exp_field(double a) {
  return (int)(((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF);
}

// rmax[i] = max_j exponent field of a_ij (rmax zeroed beforehand).  A thread
// per row, columns split over blockIdx.y.
__global__ void rowexp_kernel(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                              int cols_per_block, int* __restrict__ rmax, int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_block;
  const int64_t j1 = std::min<int64_t>(n, j0 + cols_per_block);
  int mx = 0;
  for (int64_t j = j0; j < j1; ++j) mx = max(mx, exp_field(A[i + j * lda]));
  if (mx == 2047) atomicOr(status, 1 << RSVD_ERR_NONFINITE);
  if (mx > 0) atomicMax(&rmax[i], mx);
}

// The six digit slices of A: slice s of element (i, j) at
// sl[s * ncol * ldsl + i + j * ldsl]; columns n .. ncol-1 are zero.
__global__ void slice_a_kernel(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                               const int* __restrict__ rmax, __nv_bfloat16* __restrict__ sl,
                               int64_t ldsl, int64_t ncol) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const size_t sstride = (size_t)ncol * ldsl;
  const int e = rmax[i] - 1022;
  for (int64_t j = blockIdx.y; j < ncol; j += gridDim.y) {
    float d[TC_S];
    if (j < n) {
      digits6(A[i + j * lda], e, d);
    } else {
#pragma unroll
      for (int s = 0; s < TC_S; ++s) d[s] = 0.f;
    }
    __nv_bfloat16* o = sl + i + j * ldsl;
#pragma unroll
    for (int s = 0; s < TC_S; ++s) o[s * sstride] = __float2bfloat16_rn(d[s]);
  }
}

// The same with two consecutive rows per thread (A 16-byte aligned, lda and
// ldsl even): one 16-byte load and one 4-byte store per slice for the pair,
// so each warp writes whole 128-byte lines.
__global__ void slice_a2_kernel(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                const int* __restrict__ rmax, __nv_bfloat16* __restrict__ sl,
                                int64_t ldsl, int64_t ncol) {
  const int64_t i = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (i >= m) return;
  const bool pair = i + 1 < m;
  const size_t sstride = (size_t)ncol * ldsl;
  const int e0 = rmax[i] - 1022, e1 = pair ? rmax[i + 1] - 1022 : 0;
  for (int64_t j = blockIdx.y; j < ncol; j += gridDim.y) {
    float d0[TC_S], d1[TC_S];
    if (j < n) {
      double2 a;
      if (pair) {
        a = *reinterpret_cast<const double2*>(A + i + j * lda);
      } else {
        a.x = A[i + j * lda];
        a.y = 0.0;
      }
      digits6(a.x, e0, d0);
      digits6(a.y, e1, d1);
    } else {
#pragma unroll
      for (int t = 0; t < TC_S; ++t) d0[t] = d1[t] = 0.f;
    }
    __nv_bfloat16* o = sl + i + j * ldsl;
#pragma unroll
    for (int t = 0; t < TC_S; ++t) {
      if (pair)
        *reinterpret_cast<__nv_bfloat162*>(o + t * sstride) = __floats2bfloat162_rn(d0[t], d1[t]);
      else
        o[t * sstride] = __float2bfloat16_rn(d0[t]);
    }
  }
}

// The six digit slices of X (rows x l, ldx), one block per column c < W:
// f_c from the column's largest exponent (after the 2^r_k row scaling when
// rmax is given), slice t of element (k, c) at xs[(t * W + c) * ldxs + k].
// Columns l .. W-1 are zero.
__global__ void slice_x_kernel(const double* __restrict__ X, int64_t rows, int l, int64_t ldx,
                               const int* __restrict__ rmax, int W,
                               __nv_bfloat16* __restrict__ xs, int64_t ldxs,
                               int* __restrict__ fexp) {
  const int c = blockIdx.x;
  __shared__ int s_max;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  const double* x = X + (int64_t)c * ldx;
  if (c < l) {
    int mx = 0;
    for (int64_t k = threadIdx.x; k < rows; k += blockDim.x) {
      const int E = exp_field(x[k]);
      if (E > 0) mx = max(mx, E + (rmax ? rmax[k] - 1022 : 0));
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&s_max, mx);
  }
  __syncthreads();
  // f_c = exponent bound of the scaled column (field - 1022); all-zero: 0
  const int f = s_max > 0 ? s_max - 1022 : 0;
  if (threadIdx.x == 0) fexp[c] = f;
  const size_t tstride = (size_t)W * ldxs;
  for (int64_t k = threadIdx.x; k < rows; k += blockDim.x) {
    float d[TC_S];
    if (c < l) {
      // x 2^(r_k) has digits of x relative to 2^(f - r_k)
      digits6(x[k], f - (rmax ? rmax[k] - 1022 : 0), d);
    } else {
#pragma unroll
      for (int s = 0; s < TC_S; ++s) d[s] = 0.f;
    }
    __nv_bfloat16* o = xs + (size_t)c * ldxs + k;
#pragma unroll
    for (int s = 0; s < TC_S; ++s) o[s * tstride] = __float2bfloat16_rn(d[s]);
  }
}

// ---------------------------------------------------------------------------
// Pass kernel
// ---------------------------------------------------------------------------

// The MMA schedule of one k-block for region width W, fixed at compile
// time: per A slice s, the X slices t with s + t < 6, exact regions (g < 4)
// and tail regions apart, each run cut into balanced pieces of at most
// 256 / W slices (N = count * W <= 256).  With it the k-block's MMAs
// unroll into straight-line issue with constant descriptor offsets.
struct MmaSched {
  int n;
  int s[TC_MAX_MMA], t0[TC_MAX_MMA], cnt[TC_MAX_MMA], reg0[TC_MAX_MMA], tail[TC_MAX_MMA];
};

__host__ __device__ constexpr MmaSched make_sched(int W) {
  MmaSched m{};
  const int maxc = 256 / W;
  for (int s = 0; s < TC_S; ++s) {
    for (int tail = 0; tail < 2; ++tail) {
      const int g_lo = tail ? (TC_EXACT > s ? TC_EXACT : s) : s;
      const int g_hi = tail ? TC_S - 1 : TC_EXACT - 1;
      if (g_lo > g_hi) continue;
      const int cnt = g_hi - g_lo + 1;
      const int pieces = (cnt + maxc - 1) / maxc;
      int g = g_lo;
      for (int p = 0; p < pieces; ++p) {
        const int c = (cnt - (g - g_lo) + (pieces - p) - 1) / (pieces - p);
        m.s[m.n] = s;
        m.t0[m.n] = g - s;
        m.cnt[m.n] = c;
        m.reg0[m.n] = g;
        m.tail[m.n] = tail;
        ++m.n;
        g += c;
      }
    }
  }
  return m;
}

struct TcArgs {
  int64_t rows_out;     // m (AX) or n (A^T X)
  int64_t total;        // tiles * kt
  int kt;
  int l;                // output columns of this pass (<= W)
  int64_t ncol;         // columns per A slice in the slice buffer
  int64_t* raw_t;       // full tiles: rows_out x l (ld rows_out)
  float* raw_r;
  int64_t* part_t;      // split tiles: slot (cta * 2 + first/last) of 128 x l (ld 128)
  float* part_r;
  int* status;
  long long wait_cycles;
};

template <bool AX, int W, int QC>
__global__ void __launch_bounds__(TC_THREADS, 1)
apass_f64tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                   const TcArgs args) {
  // W: region width (l rounded up to 16); each epilogue warp owns up to QC
  // columns of it (three warps per TMEM lane quadrant)
  constexpr int X_SLAB = W * 128;              // one X slice of one k-block
  constexpr int X_BYTES = TC_S * X_SLAB;
  extern __shared__ uint8_t smem_raw[];
  uint64_t* xfull = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* xempty = xfull + 2;
  uint64_t* afull = xempty + 2;
  uint64_t* aempty = afull + TC_S;
  uint64_t* acc_full = aempty + TC_S;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t buf_off = ((raw + 256 + 1023) & ~1023u) - raw;
  uint8_t* xbuf = smem_raw + buf_off;          // 2 x X_BYTES
  uint8_t* abuf = xbuf + 2 * X_BYTES;          // TC_S x A_SLAB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g0 = range_begin(args.total, blockIdx.x, gridDim.x);
  const int64_t g1 = range_begin(args.total, blockIdx.x + 1, gridDim.x);
  if (g0 >= g1) return;
  constexpr uint32_t kTmemCols = (6 * W <= 128) ? 128 : (6 * W <= 256 ? 256 : 512);

  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&xfull[b], 1);
      mbar_init(&xempty[b], 1);
    }
    for (int s = 0; s < TC_S; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, TC_EPI);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int64_t t = g0 / args.kt;
      int kb = (int)(g0 - t * args.kt);
      int64_t x_issued[2] = {0, 0};
      int64_t a_issued = 0;           // k-blocks whose A slices were all issued
      int a_partial = 0;              // A slices issued for the current k-block
      bool ok = true;
      for (int64_t g = g0; g < g1 && ok; ++g) {
        const int64_t i = g - g0;
        a_partial = 0;
        const int xs = (int)(i & 1);
        const uint32_t xpar = (uint32_t)((i >> 1) & 1);
        if (!mbar_wait(&xempty[xs], xpar ^ 1u, abort_flag, args.wait_cycles)) { ok = false; break; }
        mbar_expect_tx(&xfull[xs], (uint32_t)X_BYTES);
        uint8_t* xb = xbuf + xs * X_BYTES;
#pragma unroll
        for (int tt = 0; tt < TC_S; ++tt)
          tma_load_2d(&tmX, &xfull[xs], xb + tt * X_SLAB, kb * TC_BK, tt * W);
        ++x_issued[xs];
        for (int s = 0; s < TC_S; ++s) {
          if (!mbar_wait(&aempty[s], (uint32_t)(i & 1) ^ 1u, abort_flag, args.wait_cycles)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&afull[s], (uint32_t)A_SLAB);
          uint8_t* as = abuf + s * A_SLAB;
          const int ycol = (int)(s * args.ncol);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (AX)
              tma_load_2d(&tmA, &afull[s], as + h * (A_SLAB / 2), (int)(t * TC_BM + h * 64),
                          ycol + kb * TC_BK);
            else
              tma_load_2d(&tmA, &afull[s], as + h * (A_SLAB / 2), kb * TC_BK,
                          ycol + (int)(t * TC_BM + h * 64));
          }
          ++a_partial;
        }
        if (ok) {
          ++a_issued;
          a_partial = 0;
        }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      if (!ok) {
        // wait (bounded) for every load already issued to land: the last
        // phase of each barrier that received loads
        for (int b = 0; b < 2; ++b) {
          if (x_issued[b] == 0) continue;
          const uint32_t par = (uint32_t)((x_issued[b] - 1) & 1);
          long long t0 = clock64();
          while (!mbar_try_wait(&xfull[b], par) && clock64() - t0 < kWaitCycles) {
          }
        }
        for (int s = 0; s < TC_S; ++s) {
          const int64_t cnt = a_issued + (s < a_partial ? 1 : 0);
          if (cnt == 0) continue;
          const uint32_t par = (uint32_t)((cnt - 1) & 1);
          long long t0 = clock64();
          while (!mbar_try_wait(&afull[s], par) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint64_t a_kstep = AX ? (2048 >> 4) : (32 >> 4);
      constexpr uint64_t b_kstep = 32 >> 4;
      const uint32_t abuf_u32 = smem_u32(abuf);
      int64_t t = g0 / args.kt;
      int kb = (int)(g0 - t * args.kt);
      int kc = 0;               // k-blocks since the segment began
      int chunks = 0;           // chunks committed to the epilogue
      bool ok = true;
      for (int64_t g = g0; g < g1; ++g) {
        const int64_t i = g - g0;
        const bool seg_first = (g == g0) || kb == 0;
        const bool seg_last = (g == g1 - 1) || kb == args.kt - 1;
        if (seg_first) kc = 0;
        const bool chunk_first = (kc % TC_CHUNK) == 0;
        const bool chunk_last = seg_last || (kc % TC_CHUNK) == TC_CHUNK - 1;
        if (chunk_first && chunks > 0) {
          if (!mbar_wait(acc_empty, (uint32_t)((chunks - 1) & 1), abort_flag, args.wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const int xs = (int)(i & 1);
        if (!mbar_wait(&xfull[xs], (uint32_t)((i >> 1) & 1), abort_flag, args.wait_cycles)) {
          ok = false;
          break;
        }
        const uint64_t xd = sdesc(smem_u32(xbuf + xs * X_BYTES), 16, 1024);
        constexpr MmaSched SC = make_sched(W);
#pragma unroll
        for (int s = 0; s < TC_S; ++s) {
          if (ok && !mbar_wait(&afull[s], (uint32_t)(i & 1), abort_flag, args.wait_cycles))
            ok = false;
          if (ok) {
            tc_fence_after();
            const uint32_t a_base = abuf_u32 + s * A_SLAB;
            // MN-major A (AX): two 64-row MN atoms 8192 bytes apart, 8-row K
            // groups 1024 apart; K-major A (A^T X): 8-row groups 1024 apart
            const uint64_t ad = AX ? sdesc(a_base, TC_BK * 128, 1024) : sdesc(a_base, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
              for (int e = 0; e < SC.n; ++e) {
                if (SC.s[e] != s) continue;
                // X slice t0 starts t0 * X_SLAB bytes into the buffer (16-byte units)
                const uint64_t bd = xd + (uint64_t)((SC.t0[e] * X_SLAB) >> 4) + kk * b_kstep;
                const bool init = (s == 0) && kk == 0 && (SC.tail[e] ? seg_first : chunk_first);
                umma_bf16(tmem_base + (uint32_t)(SC.reg0[e] * W), ad + kk * a_kstep, bd,
                          idesc_bf16(TC_BM, SC.cnt[e] * W, AX), init ? 0u : 1u);
              }
            }
            umma_commit(&aempty[s]);    // A buffer s is free once these finish
          }
        }
        if (!ok) break;
        umma_commit(&xempty[xs]);
        if (chunk_last) {
          umma_commit(acc_full);
          ++chunks;
        }
        ++kc;
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      if (!ok) {
        // one more commit tracks every MMA issued so far; wait for it
        // (bounded) so TMEM is idle before it is freed
        umma_commit(acc_full);
        long long t0 = clock64();
        while (!mbar_try_wait(acc_full, (uint32_t)(chunks & 1)) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 13) ----------------
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;
    const int col0 = part * QC;
    const int ncols = min(QC, W - col0);          // multiple of 4, warp-uniform
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    long long T[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) T[j] = 0;
    int chunks = 0;
    bool ok = true;
    int64_t g = g0;
    while (g < g1 && ok) {
      const int64_t t = g / args.kt;
      const int kb0 = (int)(g - t * args.kt);
      const int64_t gend = std::min<int64_t>(g1, (t + 1) * args.kt);
      const bool full_tile = (kb0 == 0) && (gend - t * args.kt == args.kt);
      for (int64_t c0 = g; c0 < gend; c0 += TC_CHUNK) {
        const bool last = c0 + TC_CHUNK >= gend;
        // warp-uniform outcome: tcgen05.ld below is a warp-wide instruction
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full, (uint32_t)(chunks & 1), abort_flag,
                                               args.wait_cycles))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // exact regions: T += sum_g 2^(8 (3 - g)) G_g
#pragma unroll
        for (int cb = 0; cb < QC / 4; ++cb) {
          if (cb * 4 < ncols) {
#pragma unroll
            for (int gi = 0; gi < TC_EXACT; ++gi) {
              uint32_t r[4];
              tmem_ld4(lane_base + (uint32_t)(gi * W + col0 + cb * 4), r);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const long long v = (long long)__float2int_rn(__uint_as_float(r[j]));
                T[cb * 4 + j] += v << (8 * (TC_EXACT - 1 - gi));
              }
            }
          }
        }
        if (last) {
          // tail regions, then the raw output of this segment
          const int64_t row_in = quad * 32 + lane;
          int64_t* dt;
          float* dr;
          int64_t ld, row;
          bool row_ok = true;
          if (full_tile) {
            row = t * TC_BM + row_in;
            row_ok = row < args.rows_out;
            dt = args.raw_t;
            dr = args.raw_r;
            ld = args.rows_out;
          } else {
            const int slot = (g == g0) ? 0 : 1;
            row = row_in;
            dt = args.part_t + ((size_t)blockIdx.x * 2 + slot) * (size_t)TC_BM * args.l;
            dr = args.part_r + ((size_t)blockIdx.x * 2 + slot) * (size_t)TC_BM * args.l;
            ld = TC_BM;
          }
          // columns col0 .. col0+ncols-1 of this row, one pointer step per column
          int64_t* pt = dt + row + (int64_t)col0 * ld;
          float* pr = dr + row + (int64_t)col0 * ld;
          const int cmax = row_ok ? min(ncols, args.l - col0) : 0;   // columns written
#pragma unroll
          for (int cb = 0; cb < QC / 4; ++cb) {
            if (cb * 4 < ncols) {
              uint32_t r4[4], r5[4];
              tmem_ld4(lane_base + (uint32_t)(4 * W + col0 + cb * 4), r4);
              tmem_ld4(lane_base + (uint32_t)(5 * W + col0 + cb * 4), r5);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float R = __uint_as_float(r4[j]) + __uint_as_float(r5[j]) * 0.00390625f;
                if (cb * 4 + j < cmax) {
                  *pt = T[cb * 4 + j];
                  *pr = R;
                }
                pt += ld;
                pr += ld;
                T[cb * 4 + j] = 0;
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
        ++chunks;
      }
      g = gend;
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.status, 1 << RSVD_ERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// out (rows_out x l, ldo, FP64) = 2^(e_row + f_c - 14) (T 2^-24 + R 2^-32),
// with T, R summed over the tile's sources: the raw buffer for tiles one CTA
// wrote whole, the partial slots for split tiles (FixList).  Grid: (tile,
// column group of cpb columns); one thread per tile row.  Few tiles (a Gram's
// single tile split over many CTAs) take one column per block, so the sums
// over the partial slots spread over more SMs.
__global__ void f64tc_finalize_kernel(const int64_t* __restrict__ raw_t,
                                      const float* __restrict__ raw_r, int64_t rows_out, int l,
                                      const int64_t* __restrict__ part_t,
                                      const float* __restrict__ part_r,
                                      const int* __restrict__ rmax, const int* __restrict__ fexp,
                                      double* __restrict__ out, int64_t ldo, int cpb,
                                      const __grid_constant__ FixList fl) {
  const int t = blockIdx.x;
  __shared__ int s_idx;
  if (threadIdx.x == 0) {
    int idx = -1;
    for (int i = 0; i < fl.n; ++i)
      if (fl.tile[i] == t) { idx = i; break; }
    s_idx = idx;
  }
  __syncthreads();
  const int idx = s_idx;
  const int r = threadIdx.x;
  const int64_t row = (int64_t)t * TC_BM + r;
  if (row >= rows_out) return;
  const int per_tile = TC_BM * l;
  for (int cc = 0; cc < cpb; ++cc) {
    const int c = blockIdx.y * cpb + cc;
    if (c >= l) break;
    long long T = 0;
    double R = 0.0;
    if (idx < 0) {
      T = raw_t[row + (int64_t)c * rows_out];
      R = (double)raw_r[row + (int64_t)c * rows_out];
    } else {
      for (int j = fl.off[idx]; j < fl.off[idx + 1]; ++j) {
        const size_t o = (size_t)fl.src[j] * per_tile + (size_t)c * TC_BM + r;
        T += part_t[o];
        R += (double)part_r[o];
      }
    }
    const int e = (rmax ? rmax[row] - 1022 : 0) + fexp[c] - 14;
    double v;
    if (e - 32 >= -1022 && e - 24 <= 1023) {
      // 2^(e-24) and 2^(e-32) from their exponent fields: two FP64 operations
      const double s24 = __longlong_as_double((long long)(e - 24 + 1023) << 52);
      const double s32 = __longlong_as_double((long long)(e - 32 + 1023) << 52);
      v = fma((double)T, s24, R * s32);
    } else {
      v = ldexp((double)T * 0x1p-24 + R * 0x1p-32, e);
    }
    out[row + (int64_t)c * ldo] = v;
  }
}

// K-major BF16 map of the X slices: rows of `cols` elements (ld ldxs),
// 6 W of them; box 64 x W.
bool make_map_x(CUtensorMap* map, const void* base, int64_t kdim, int rows, int64_t ldxs, int W) {
  return make_map_bf16(map, base, kdim, rows, ldxs, 64, W);
}

}  // namespace

int f64tc_prepare_a(const double* A, int64_t m, int64_t n, int64_t lda, void* slices,
                    int64_t ldsl, int64_t ncol, int* rmax, int* status, int num_sms,
                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(int) * (size_t)m, st);
  if (e != cudaSuccess) return cuda_fail("row exponent reset", e);
  const int cpb = 256;
  dim3 g1((unsigned)((m + 255) / 256), (unsigned)((n + cpb - 1) / cpb));
  rowexp_kernel<<<g1, 256, 0, st>>>(A, m, n, lda, cpb, rmax, status);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("rowexp_kernel", e);
  if (lda % 2 == 0 && ldsl % 2 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)slices % 4 == 0) {
    const int64_t rb = (m + 511) / 512;
    const int64_t cy =
        std::max<int64_t>(1, std::min<int64_t>(ncol, ((int64_t)num_sms * 32 + rb - 1) / rb));
    slice_a2_kernel<<<dim3((unsigned)rb, (unsigned)std::min<int64_t>(cy, 65535)), 256, 0, st>>>(
        A, m, n, lda, rmax, (__nv_bfloat16*)slices, ldsl, ncol);
  } else {
    const int64_t rb = (m + 255) / 256;
    const int64_t cy =
        std::max<int64_t>(1, std::min<int64_t>(ncol, ((int64_t)num_sms * 32 + rb - 1) / rb));
    slice_a_kernel<<<dim3((unsigned)rb, (unsigned)std::min<int64_t>(cy, 65535)), 256, 0, st>>>(
        A, m, n, lda, rmax, (__nv_bfloat16*)slices, ldsl, ncol);
  }
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("slice_a_kernel", e);
  return RSVD_OK;
}

int launch_apass_f64tc(const F64tcCall& c, int num_sms, int* status, cudaStream_t st) {
  const int64_t rows_out = c.ax ? c.m : c.n;
  const int64_t kdim = c.ax ? c.n : c.m;
  if (c.ldsl % 8 || c.ldxs % 8 || c.ldxs < kdim || ((uintptr_t)c.slices % 16) ||
      ((uintptr_t)c.xslices % 16))
    return RSVD_ERR_UNSUPPORTED;
  const int64_t tiles = (rows_out + TC_BM - 1) / TC_BM;
  const int kt = (int)((kdim + TC_BK - 1) / TC_BK);
  const int64_t total = tiles * kt;
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(num_sms, total), tiles * 30);
  if ((int64_t)kt * grid / total + 2 > 32) return RSVD_ERR_UNSUPPORTED;
  CUtensorMap tmA;
  if (!make_map_bf16(&tmA, c.slices, c.m, TC_S * c.ncol, c.ldsl, 64, 64))
    return cuda_fail("A slice tensor map", cudaSuccess);
  cudaError_t e;
  static thread_local FixList fl;
  if (!build_fix_list(grid, total, kt, tiles, fl)) return RSVD_ERR_UNSUPPORTED;
  for (int c0 = 0; c0 < c.l; c0 += kF64tcMaxL) {
    const int lb = std::min(kF64tcMaxL, c.l - c0);
    const int W = (lb + 15) / 16 * 16;
    // X slices of this column block
    slice_x_kernel<<<W, 512, 0, st>>>(c.X + (int64_t)c0 * c.ldx, kdim, lb, c.ldx,
                                      c.ax ? nullptr : c.rmax, W, (__nv_bfloat16*)c.xslices,
                                      c.ldxs, c.fexp);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("slice_x_kernel", e);
    CUtensorMap tmX;
    if (!make_map_x(&tmX, c.xslices, kdim, TC_S * W, c.ldxs, W))
      return cuda_fail("X slice tensor map", cudaSuccess);
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rows_out = rows_out;
    a.total = total;
    a.kt = kt;
    a.l = lb;
    a.ncol = c.ncol;
    a.raw_t = c.raw_t;
    a.raw_r = c.raw_r;
    a.part_t = c.part_t;
    a.part_r = c.part_r;
    a.status = status;
    a.wait_cycles = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
    const size_t smem = 1024 + 256 + (size_t)2 * TC_S * W * 128 + (size_t)TC_S * A_SLAB;
#define RSVD_F64TC(AXV, WV, QV)                                                              \
  do {                                                                                      \
    cudaFuncSetAttribute(apass_f64tc_kernel<AXV, WV, QV>,                                   \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    apass_f64tc_kernel<AXV, WV, QV><<<grid, TC_THREADS, smem, st>>>(tmA, tmX, a);           \
  } while (0)
  // QC: columns per epilogue warp, a multiple of 4 with 3 QC >= W
#define RSVD_F64TC_W(AXV)                          \
  switch (W) {                                     \
    case 16: RSVD_F64TC(AXV, 16, 8); break;        \
    case 32: RSVD_F64TC(AXV, 32, 12); break;       \
    case 48: RSVD_F64TC(AXV, 48, 16); break;       \
    case 64: RSVD_F64TC(AXV, 64, 24); break;       \
    default: RSVD_F64TC(AXV, 80, 28); break;       \
  }
    if (c.ax) {
      RSVD_F64TC_W(true);
    } else {
      RSVD_F64TC_W(false);
    }
#undef RSVD_F64TC_W
#undef RSVD_F64TC
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("apass_f64tc_kernel", e);
    const int cpb = tiles * ((lb + 7) / 8) < 2 * num_sms ? 1 : 8;
    const dim3 fgrid((unsigned)tiles, (unsigned)((lb + cpb - 1) / cpb));
    f64tc_finalize_kernel<<<fgrid, TC_BM, 0, st>>>(c.raw_t, c.raw_r, rows_out, lb, c.part_t,
                                                   c.part_r, c.ax ? c.rmax : nullptr, c.fexp,
                                                   c.out + (int64_t)c0 * c.ldo, c.ldo, cpb, fl);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("f64tc_finalize_kernel", e);
  }
  return RSVD_OK;
}

}  // namespace rsvd
