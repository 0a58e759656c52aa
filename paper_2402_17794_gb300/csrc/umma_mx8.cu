// FP8 passes over A on the tcgen05 tensor cores with block-scaled MMA
// (tcgen05.mma kind::mxf8f6f4): the mixed path of Algorithm 4 (steps 2, 5
// and 6, Section 3.3) for A stored in E4M3 with one power-of-two scale per
// 128 x 128 tile.
//
//   kind AX  : Y = A X     (contracts n; A is MN-major for the MMA)
//   kind ATX : Z = A^T X   (contracts m; A is K-major)
//
// Both MMA operands are E4M3.  A comes straight from HBM by TMA, one byte per
// element, and its tile scale is applied by the tensor core as a UE8M0 block
// scale.  The FP32 operand X is split into S E4M3 slices
//   x_rc = 2^(d_c) sum_j 2^(e_k - 4 j) x_j,rc      (x_j E4M3, j = 0 .. S-1),
// d_c a power-of-two normalisation of column c (undone exactly in the
// epilogue, so columns of any magnitude keep their precision) and e_k one
// exponent per chunk k of the normalised X (BK rows, one stage), chosen so
// that the chunk's largest magnitude lands in [128, 256) in slice 0.  Each slice peels off
// the E4M3 rounding of what the earlier ones left, so S slices carry about
// 4 S significant bits of every element (E4M3: 4 significant bits).  The
// slice products of one output tile accumulate into one FP32 TMEM
// accumulator; each slice's power-of-two weight is its UE8M0 block scale.
// All scale factors are constant over a stage (A: per 128 x 128 tile; X: per
// chunk and slice), so every byte of a scale-factor region holds the
// same value and the MMA reads it wherever its layout places a row's or a
// column's scale.
//
// Shape and schedule follow the BF16 passes: persistent grid with stream-K
// ranges of (tile, k-block) iterations (tile = MT x 128 output rows,
// k-block = BK of the contraction), split tiles written as per-CTA partials
// and summed by the fixup kernel.  Warp roles: warp 0 TMA producer, warp 1
// MMA issuer (one lane), warps 2-5 epilogue (tcgen05.ld, FP32 stores), warps
// 6-9 write the scale factors of each stage into TMEM with tcgen05.st (one
// warp per TMEM lane quarter).  Every wait is bounded (plan wait limit or
// about one second); on expiry the CTA records RSVD_ERR_TIMEOUT, drains what
// it issued and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.h"
#include "umma.h"
#include "umma_ptx.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128;          // output rows per sub-tile (MMA M)
constexpr int THREADS = 320;     // 10 warps
constexpr int SFA_COLS = 4;      // TMEM columns of an A scale-factor region (M = 128)
// B scale-factor regions: 4 columns cover N <= 128, 8 columns N <= 256
__host__ __device__ constexpr int sfb_cols(int l16) { return l16 > 128 ? 8 : 4; }

// Shared-memory matrix descriptor with an explicit swizzle mode (bits 61-63:
// 2 = 128-byte, 4 = 64-byte swizzle); fields as in sdesc.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                             uint32_t mode) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)mode << 61;
  return d;
}

// Instruction descriptor of kind::mxf8f6f4: A and B E4M3 (format 0 in bits
// 7-9 and 10-12), A major in bit 15 (1: MN-major), B K-major, N >> 3 in bits
// 17-22, scale factors UE8M0 (bit 23 = 1), M >> 4 in bits 24-28; scale
// factor ids (bits 4-5 for B, 29-30 for A) zero.
__host__ __device__ constexpr uint32_t idesc_mx8(int M, int N, bool a_mn_major) {
  return ((a_mn_major ? 1u : 0u) << 15) | ((uint32_t)(N >> 3) << 17) | (1u << 23) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_mx8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X "
      "[%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

// Four TMEM columns of this warp's 32 lanes, every 32-bit cell = v.
__device__ __forceinline__ void tmem_st4_same(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(taddr),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// UE8M0 code of a power-of-two FP32 scale, replicated into four bytes; zero,
// non-finite or non-normal scales (an all-zero tile) give 2^0.
__device__ __forceinline__ uint32_t ue8m0x4_of_scale(float s) {
  const uint32_t b = __float_as_uint(s);
  uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu || (b & 0x80000000u)) e = 127u;
  return e * 0x01010101u;
}

__device__ __forceinline__ uint32_t ue8m0x4_of_exp(int e) {
  e = max(-126, min(127, e));
  return (uint32_t)(e + 127) * 0x01010101u;
}

struct Mx8Args {
  int sfb;                 // TMEM columns of a B scale-factor region
  int64_t rows_out;
  int64_t total;
  int kt;
  int l16;
  int l;
  int stages;
  uint32_t tmem_cols;
  uint32_t sf_col0;        // first scale-factor column (after the accumulators)
  float* out;
  int64_t ldo;
  float* part;
  int accumulate;
  int* status;
  const float* scales;     // A tile scales, tile (I, J) at scales[I + J * lds]
  int64_t lds;
  int sc_rows, sc_cols;
  const int* xexp;         // exponent e_k of each BK-row chunk of X
  const float* colscale;   // 2^(d_c) of each column of X
  long long wait_cycles;
};

// BK: contraction per stage, 128 (rows of 128 bytes, 128-byte swizzle) or 64
// (64-byte rows and swizzle for the K-major operands) where 128 leaves too
// little shared memory for two stages.
template <bool AX, int MT, int S, int BK>
__global__ void __launch_bounds__(THREADS, 1)
apass_mx8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                 const Mx8Args args) {
  constexpr int BMT = BM * MT;
  constexpr int SUB_BYTES = BM * BK;
  constexpr int A_BYTES = SUB_BYTES * MT;
  constexpr uint32_t KSW = BK == 128 ? 2 : 4;          // swizzle mode of K-major rows
  constexpr uint32_t KSBO = BK == 128 ? 1024 : 512;    // 8-row group stride of K-major rows
  const int sf_per_stage = MT * SFA_COLS + S * args.sfb;
  extern __shared__ uint8_t smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + args.stages;
  uint64_t* sf_full = empty + args.stages;
  uint64_t* acc_full = sf_full + args.stages;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t tiles_off = ((raw + 256 + 1023) & ~1023u) - raw;
  uint8_t* tiles = smem_raw + tiles_off;
  const int x_slice_bytes = args.l16 * BK;
  const int stage_bytes = A_BYTES + S * x_slice_bytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g0 = range_begin(args.total, blockIdx.x, gridDim.x);
  const int64_t g1 = range_begin(args.total, blockIdx.x + 1, gridDim.x);
  if (g0 >= g1) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < args.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&sf_full[s], 4);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int64_t t = g0 / args.kt;
      int kb = (int)(g0 - t * args.kt);
      int64_t issued = 0;
      for (int64_t g = g0; g < g1; ++g) {
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, args.wait_cycles)) break;
        uint8_t* a_s = tiles + (size_t)s * stage_bytes;
        uint8_t* x_s = a_s + A_BYTES;
        mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
#pragma unroll
        for (int q = 0; q < MT; ++q) {
          if (AX)   // box: 128 rows of A (128 bytes) x 64 columns
            tma_load_2d(&tmA, &full[s], a_s + q * SUB_BYTES, (int)(t * BMT + q * BM), kb * BK);
          else      // box: 64 rows of A (64 bytes) x 128 columns
            tma_load_2d(&tmA, &full[s], a_s + q * SUB_BYTES, kb * BK, (int)(t * BMT + q * BM));
        }
#pragma unroll
        for (int j = 0; j < S; ++j)
          tma_load_2d(&tmX, &full[s], x_s + j * x_slice_bytes, kb * BK, j * args.l16);
        ++issued;
        if (++s == args.stages) { s = 0; ph ^= 1u; }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      if (*abort_flag) {
        for (int64_t j = (issued > args.stages ? issued - args.stages : 0); j < issued; ++j) {
          long long t0 = clock64();
          while (!mbar_try_wait(&full[j % args.stages], (uint32_t)((j / args.stages) & 1)) &&
                 clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_mx8(BM, args.l16, AX);
      const uint32_t tiles_base = smem_u32(tiles);
      // descriptor start steps (16-byte units) per 32-deep K step: MN-major A
      // advances 32 rows of 128 bytes, K-major operands 32 bytes
      constexpr uint64_t a_kstep = AX ? (4096 >> 4) : (32 >> 4);
      constexpr uint64_t b_kstep = 32 >> 4;
      int s = 0;
      uint32_t ph = 0;
      int64_t t = g0 / args.kt;
      int kb = (int)(g0 - t * args.kt);
      int seg = 0;
      bool ok = true;
      for (int64_t g = g0; g < g1; ++g) {
        const bool seg_first = (g == g0) || kb == 0;
        const bool seg_last = (g == g1 - 1) || kb == args.kt - 1;
        if (seg_first && seg > 0) {
          if (!mbar_wait(acc_empty, (uint32_t)((seg - 1) & 1), abort_flag, args.wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], ph, abort_flag, args.wait_cycles) ||
            !mbar_wait(&sf_full[s], ph, abort_flag, args.wait_cycles)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = tiles_base + (uint32_t)s * (uint32_t)stage_bytes;
        const uint32_t x_base = a_base + A_BYTES;
        const uint32_t sf_base = tmem_base + args.sf_col0 + (uint32_t)(s * sf_per_stage);
#pragma unroll
        for (int j = 0; j < S; ++j) {
          // K-major slice: rows of BK bytes
          const uint64_t bd = sdesc_sw(x_base + j * x_slice_bytes, 16, KSBO, KSW);
#pragma unroll
          for (int h = 0; h < MT; ++h) {
            const uint32_t ah = a_base + h * SUB_BYTES;
            // MN-major A: one 128-byte atom across M, 8-row K groups 1024
            // bytes apart; K-major A: rows of BK bytes as the slices
            const uint64_t ad = AX ? sdesc_sw(ah, SUB_BYTES, 1024, 2) : sdesc_sw(ah, 16, KSBO, KSW);
#pragma unroll
            for (int kk = 0; kk < BK / 32; ++kk)
              umma_mx8(tmem_base + h * args.l16, ad + kk * a_kstep, bd + kk * b_kstep, idesc,
                       sf_base + h * SFA_COLS,
                       sf_base + MT * SFA_COLS + j * args.sfb,
                       (seg_first && kk == 0 && j == 0) ? 0u : 1u);
          }
        }
        umma_commit(&empty[s]);
        if (seg_last) {
          umma_commit(acc_full);
          ++seg;
        }
        if (++s == args.stages) { s = 0; ph ^= 1u; }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      if (!ok) {
        umma_commit(acc_full);
        long long t0 = clock64();
        while (!mbar_try_wait(acc_full, (uint32_t)(seg & 1)) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp >= 6) {
    // ---------------- scale factors (warps 6-9, one per TMEM lane quarter) ----------------
    const uint32_t lane_base = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + args.sf_col0;
    int s = 0;
    uint32_t ph = 0;
    int64_t t = g0 / args.kt;
    int kb = (int)(g0 - t * args.kt);
    for (int64_t g = g0; g < g1; ++g) {
      // the stage's scales, loaded before waiting for its regions to free up
      const int64_t kk = (int64_t)kb * BK / 128;   // tile of A along the contraction
      uint32_t sa[MT];
#pragma unroll
      for (int h = 0; h < MT; ++h) {
        const int64_t tt = t * MT + h;
        const int64_t I = AX ? tt : kk, J = AX ? kk : tt;
        sa[h] = ue8m0x4_of_scale((I < args.sc_rows && J < args.sc_cols)
                                     ? __ldg(&args.scales[I + J * args.lds])
                                     : 1.f);
      }
      const int e = __ldg(&args.xexp[kb]);
      // the stage's previous MMAs have read its regions (warp-uniform outcome:
      // tcgen05.st below is a warp-wide instruction)
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, abort_flag, args.wait_cycles)))
        break;
      tc_fence_after();
      const uint32_t col = lane_base + (uint32_t)(s * sf_per_stage);
#pragma unroll
      for (int h = 0; h < MT; ++h) tmem_st4_same(col + h * SFA_COLS, sa[h]);
#pragma unroll
      for (int j = 0; j < S; ++j)
        for (int c4 = 0; c4 < args.sfb; c4 += 4)
          tmem_st4_same(col + MT * SFA_COLS + j * args.sfb + c4, ue8m0x4_of_exp(e - 4 * j));
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sf_full[s]);
      if (++s == args.stages) { s = 0; ph ^= 1u; }
      if (++kb == args.kt) { kb = 0; ++t; }
    }
  } else {
    // ---------------- epilogue (warps 2-5) ----------------
    const int quad = warp & 3;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    int seg = 0;
    int64_t g = g0;
    while (g < g1) {
      const int64_t t = g / args.kt;
      const int kb0 = (int)(g - t * args.kt);
      const int64_t gend = (g1 < (t + 1) * args.kt) ? g1 : (t + 1) * args.kt;
      const bool full_tile = (kb0 == 0) && (gend - t * args.kt == args.kt);
      // warp-uniform outcome: tcgen05.ld below is a warp-wide instruction
      if (!__all_sync(0xffffffffu, mbar_wait(acc_full, (uint32_t)(seg & 1), abort_flag,
                                             args.wait_cycles)))
        break;
      tc_fence_after();
      float* dst;
      int64_t ld, row0;
      if (full_tile) {
        row0 = t * BMT;
        dst = args.out;
        ld = args.ldo;
      } else {
        const int slot = (g == g0) ? 0 : 1;
        row0 = 0;
        dst = args.part + ((size_t)blockIdx.x * 2 + slot) * (size_t)BMT * args.l;
        ld = BMT;
      }
#pragma unroll
      for (int h = 0; h < MT; ++h) {
        const int64_t row = row0 + h * BM + quad * 32 + lane;
        const bool row_ok = full_tile ? (row < args.rows_out) : true;
        const bool acc_out = full_tile && args.accumulate;
        for (int c0 = 0; c0 < args.l; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(lane_base + (uint32_t)(h * args.l16 + c0), r);
          tmem_wait_ld();
          if (row_ok) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < args.l) {
                const float v = __uint_as_float(r[j]) * __ldg(&args.colscale[c0 + j]);
                float* d = dst + row + (int64_t)(c0 + j) * ld;
                *d = acc_out ? *d + v : v;
              }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      ++seg;
      g = gend;
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.status, 1 << RSVD_ERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, args.tmem_cols);
  }
}

// Column maxima of |X| as FP32 bit patterns (order-preserving for
// non-negative values): colbits[c] = max over rows (colbits zeroed first).
__global__ void colmax_kernel(const float* __restrict__ X, int64_t rows, int64_t ldx,
                              unsigned* __restrict__ colbits) {
  const int c = blockIdx.y;
  float mx = 0.f;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    mx = fmaxf(mx, fabsf(X[r + (int64_t)c * ldx]));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(&colbits[c], __float_as_uint(mx));
}

// Power-of-two exponent d with 2^d <= v < 2^(d+1) of a positive finite FP32
// bit pattern (0 for zero, subnormal or non-finite).
__device__ __forceinline__ int pow2_floor_exp(unsigned bits) {
  const int e = (int)((bits >> 23) & 0xFFu);
  return (e == 0 || e == 0xFF) ? 0 : e - 127;
}

// 2^k as an FP32 (k in [-126, 127]): exact power-of-two scaling by a multiply.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// X (FP32, rows x l, ld ldx) -> S E4M3 slices of the column-normalised
// x 2^-d_c (d_c from the column maxima), slice j column c at
// out[(j * l16 + c) * ldo + r] (columns l .. l16 zero), and the exponent of
// each chunk of `chunk` rows (64 or 128, the pass's stage depth):
// e_k = floor(log2 max |x 2^-d_c|) - 7 over the chunk (0 for an all-zero
// chunk), so slice 0 holds magnitudes below 256.  Block 0 also writes
// colscale[c] = 2^d_c.  One block per chunk; each thread takes four
// consecutive rows of a column and stores each slice's four codes as one
// 32-bit word.  Every scaling is by a power of two (exact), and each
// residual is exact: v minus its E4M3 rounding.
__global__ void __launch_bounds__(256) split_e4m3_kernel(const float* __restrict__ X, int64_t rows,
                                                         int l, int64_t ldx, int l16, int S,
                                                         int chunk,
                                                         const unsigned* __restrict__ colbits,
                                                         uint8_t* __restrict__ out, int64_t ldo,
                                                         int* __restrict__ xexp,
                                                         float* __restrict__ colscale) {
  __shared__ float s_mx[8];
  __shared__ float s_inv[256];   // 2^-d_c
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int tid = threadIdx.x;
  for (int c = tid; c < l16; c += 256) {
    const int d = c < l ? max(-120, min(120, pow2_floor_exp(colbits[c]))) : 0;
    s_inv[c] = pow2f(-d);
    if (blockIdx.x == 0) colscale[c] = pow2f(d);
  }
  __syncthreads();
  const int quads = chunk / 4, phases = 256 / quads;
  const int qd = tid % quads, cq = tid / quads;   // row quad in the chunk, column phase
  const int64_t r = r0 + 4 * qd;
  const int64_t left = rows - r;
  const int nr = left <= 0 ? 0 : (left >= 4 ? 4 : (int)left);   // rows of this quad
  float mx = 0.f;
  for (int c = cq; c < l; c += phases) {
    const float* x = X + r + (int64_t)c * ldx;
    const float sc = s_inv[c];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < nr) mx = fmaxf(mx, fabsf(x[k] * sc));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) s_mx[tid >> 5] = mx;
  __syncthreads();
  mx = s_mx[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) mx = fmaxf(mx, s_mx[i]);
  int e = 0;
  if (mx > 0.f && isfinite(mx)) e = (int)((__float_as_uint(mx) >> 23) & 0xFF) - 127 - 7;
  e = max(-100, min(100, e));
  if (tid == 0) xexp[blockIdx.x] = e;
  if (nr == 0) return;
  for (int c = cq; c < l16; c += phases) {
    float v[4];
    const float sc = s_inv[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (c < l && k < nr) ? X[r + k + (int64_t)c * ldx] * sc : 0.f;
    uint8_t* o = out + (int64_t)c * ldo + r;
    for (int j = 0; j < S; ++j) {
      const float down = pow2f(-(e - 4 * j)), up = pow2f(e - 4 * j);
      uint32_t word = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const __nv_fp8_e4m3 q(v[k] * down);   // round to nearest, saturating
        word |= (uint32_t)q.__x << (8 * k);
        v[k] -= float(q) * up;                // exact: the rounding error of v
      }
      uint8_t* oj = o + (int64_t)j * l16 * ldo;
      if (nr == 4) {
        *reinterpret_cast<uint32_t*>(oj) = word;
      } else {
        for (int k = 0; k < nr; ++k) oj[k] = (uint8_t)(word >> (8 * k));
      }
    }
  }
}

// E4M3 tensor map (uint8 elements) with the given swizzle.
bool make_map_e4m3(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                   int box_rows, int box_cols, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int64_t mx8_xexp_count(int64_t rows) { return (rows + 63) / 64; }

namespace {
// Launch shape of a pass: sub-tiles per CTA tile, stage depth, stages.  The
// deeper 128-row stages (128-byte TMA rows) when two of them fit shared
// memory and TMEM, else 64-row stages.
struct Mx8Shape {
  int mt = 0, bk = 0, stages = 0, sfb = 0;
};
Mx8Shape mx8_shape(int64_t rows_out, int l, int S) {
  const int l16 = (l + 15) / 16 * 16;
  Mx8Shape sh;
  sh.sfb = sfb_cols(l16);
  for (int bk : {128, 64}) {
    for (int mt = (rows_out > BM) ? 2 : 1; mt >= 1; --mt) {
      const int stage_bytes = BM * bk * mt + S * l16 * bk;
      int stages = std::min((227 * 1024 - 2048) / stage_bytes, 8);
      const int sf_per_stage = mt * SFA_COLS + S * sh.sfb;
      const int acc = (mt * l16 + 3) / 4 * 4;
      while (stages >= 2 && acc + stages * sf_per_stage > 512) --stages;
      if (stages >= 2) {
        sh.mt = mt;
        sh.bk = bk;
        sh.stages = stages;
        return sh;
      }
    }
  }
  return sh;
}
}  // namespace

int mx8_chunk_rows(bool ax, int64_t m, int64_t n, int l, int slices) {
  return mx8_shape(ax ? m : n, l, slices).bk;
}

int launch_split_e4m3(const float* X, int64_t rows, int l, int64_t ldx, int slices, int chunk,
                      uint8_t* out, int64_t ldo, int* xexp, float* colscale, unsigned* colbits,
                      cudaStream_t st) {
  const int l16 = (l + 15) / 16 * 16;
  if (rows < 1 || l < 1 || l16 > 256 || slices < 1 || ldo < rows || (chunk != 64 && chunk != 128))
    return RSVD_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(colbits, 0, sizeof(unsigned) * (size_t)l, st) != cudaSuccess)
    return RSVD_ERR_CUDA;
  const int bx = (int)std::min<int64_t>((rows + 255) / 256, 32);
  colmax_kernel<<<dim3((unsigned)bx, (unsigned)l), 256, 0, st>>>(X, rows, ldx, colbits);
  note_launch();
  split_e4m3_kernel<<<(unsigned)((rows + chunk - 1) / chunk), 256, 0, st>>>(
      X, rows, l, ldx, l16, slices, chunk, colbits, out, ldo, xexp, colscale);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

int launch_apass_mx8(const Mx8Call& c, int num_sms, int* status, cudaStream_t st) {
  if (c.lda % 16 || c.ldx % 16 || ((uintptr_t)c.A % 16) || ((uintptr_t)c.X % 16) || !c.scales ||
      !c.xexp || !c.colscale || c.lds < (c.m + 127) / 128)
    return RSVD_ERR_UNSUPPORTED;
  const int64_t rows_out = c.ax ? c.m : c.n;
  const int64_t kdim = c.ax ? c.n : c.m;
  const int l16 = (c.l + 15) / 16 * 16;
  if (c.l < 1 || c.l > 256) return RSVD_ERR_UNSUPPORTED;
  const int S = c.slices;
  if (S != 2 && S != 4 && S != 6) return RSVD_ERR_UNSUPPORTED;
  const Mx8Shape sh = mx8_shape(rows_out, c.l, S);
  if (sh.stages < 2 || sh.bk != c.chunk) return RSVD_ERR_UNSUPPORTED;
  const int mt = sh.mt, bk = sh.bk, stages = sh.stages;
  const int kt = (int)((kdim + bk - 1) / bk);
  const int stage_bytes = BM * bk * mt + S * l16 * bk;
  const int bmt = BM * mt;
  const int64_t tiles = (rows_out + bmt - 1) / bmt;
  const int64_t total = tiles * kt;
  const size_t smem = 2048 + (size_t)stages * stage_bytes;
  const uint32_t tmem_cols = 512;

  CUtensorMap tmA, tmX;
  const CUtensorMapSwizzle ksw = bk == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const bool okA = c.ax ? make_map_e4m3(&tmA, c.A, c.m, c.n, c.lda, 128, bk,
                                        CU_TENSOR_MAP_SWIZZLE_128B)
                        : make_map_e4m3(&tmA, c.A, c.m, c.n, c.lda, bk, 128, ksw);
  if (!okA) return RSVD_ERR_CUDA;
  if (!make_map_e4m3(&tmX, c.X, kdim, (int64_t)S * l16, c.ldx, bk, l16, ksw)) return RSVD_ERR_CUDA;

  int grid = (int)std::min<int64_t>(std::min<int64_t>(num_sms, total), tiles * 30);
  Mx8Args a;
  a.sfb = sh.sfb;
  a.rows_out = rows_out;
  a.total = total;
  a.kt = kt;
  a.l16 = l16;
  a.l = c.l;
  a.stages = stages;
  a.tmem_cols = tmem_cols;
  a.sf_col0 = (uint32_t)(mt * l16 + 3) / 4 * 4;
  a.out = c.out;
  a.ldo = c.ldo;
  a.part = c.part;
  a.accumulate = c.accumulate ? 1 : 0;
  a.status = status;
  a.scales = c.scales;
  a.lds = c.lds;
  a.sc_rows = (int)((c.m + 127) / 128);
  a.sc_cols = (int)((c.n + 127) / 128);
  a.xexp = c.xexp;
  a.colscale = c.colscale;
  a.wait_cycles = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
  if (a.sf_col0 + (uint32_t)(stages * (mt * SFA_COLS + S * sh.sfb)) > tmem_cols)
    return RSVD_ERR_UNSUPPORTED;
  if (c.part_floats < (size_t)grid * 2 * bmt * c.l) return RSVD_ERR_WORKSPACE;
  if ((int64_t)kt * grid / total + 2 > 32) return RSVD_ERR_UNSUPPORTED;
#define RSVD_LAUNCH_MX8(AXV, MTV, SV, BKV)                                                 \
  do {                                                                                     \
    cudaFuncSetAttribute(apass_mx8_kernel<AXV, MTV, SV, BKV>,                              \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    apass_mx8_kernel<AXV, MTV, SV, BKV><<<grid, THREADS, smem, st>>>(tmA, tmX, a);         \
  } while (0)
#define RSVD_LAUNCH_MX8_B(AXV, MTV, SV)              \
  do {                                               \
    if (bk == 128) RSVD_LAUNCH_MX8(AXV, MTV, SV, 128); \
    else RSVD_LAUNCH_MX8(AXV, MTV, SV, 64);           \
  } while (0)
#define RSVD_LAUNCH_MX8_S(AXV, MTV)                  \
  do {                                               \
    if (S == 2) RSVD_LAUNCH_MX8_B(AXV, MTV, 2);      \
    else if (S == 4) RSVD_LAUNCH_MX8_B(AXV, MTV, 4); \
    else RSVD_LAUNCH_MX8_B(AXV, MTV, 6);             \
  } while (0)
  if (c.ax) {
    if (mt == 2) RSVD_LAUNCH_MX8_S(true, 2);
    else RSVD_LAUNCH_MX8_S(true, 1);
  } else {
    if (mt == 2) RSVD_LAUNCH_MX8_S(false, 2);
    else RSVD_LAUNCH_MX8_S(false, 1);
  }
#undef RSVD_LAUNCH_MX8_S
#undef RSVD_LAUNCH_MX8_B
#undef RSVD_LAUNCH_MX8
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return RSVD_ERR_CUDA;
  return launch_apass_fixup(c.part, grid, total, kt, bmt, c.l, rows_out, tiles, c.out, c.ldo,
                            a.accumulate, st);
}

}  // namespace rsvd
