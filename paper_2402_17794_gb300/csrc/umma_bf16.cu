// BF16 passes over A on the tcgen05 tensor cores (mixed path of Algorithm 4,
// steps 2, 5 and 6, Section 3.3):
//
//   kind AX  : Y = A X     (m x n times n x N, contracts the long n; A is
//              MN-major for the MMA because its columns are contiguous)
//   kind ATX : Z = A^T X   (n x m times m x N, contracts the long m; A is
//              K-major)
//
// A is read exactly once from HBM per pass; X (l <= 256 columns, BF16,
// column-major) is small and is re-read from L2.  X may hold up to three BF16
// "slices" side by side (x = x_1 + x_2 + x_3, the bf16x2 / bf16x3 split of an
// FP32 operand); the MMAs of every slice accumulate into the same TMEM
// accumulator, so D = A (x_1 + x_2 + x_3) in FP32.  Design:
//
//  * Persistent grid, one CTA per SM.  The (tile, k-block) iteration space
//    (tile = 128 output rows, k-block = 64 of the contraction) is cut into
//    equal contiguous ranges, one per CTA ("stream-K"), so every SM streams
//    the same number of bytes of A.  A tile whose k-range is split between
//    CTAs is written as per-CTA partials and summed by a second kernel in
//    CTA order (deterministic).
//  * Warp roles: warp 0 issues TMA (cp.async.bulk.tensor, 128-byte swizzle)
//    into a ring of shared-memory stages guarded by mbarriers; warp 1 owns
//    the TMEM accumulator and one lane issues tcgen05.mma (M=128, N<=256 per
//    instruction, K=16, FP32 accumulate in TMEM) and tcgen05.commit; warps
//    2-5 drain the accumulator with tcgen05.ld and store FP32 results.
//  * Every mbarrier wait is bounded (about one second of clock64 by default,
//    the plan's wait limit if set); on expiry the CTA records
//    RSVD_ERR_TIMEOUT, stops issuing, drains what it issued (those waits keep
//    the one-second bound) and frees its TMEM before returning.
//  * FP8 A (E4M3, one power-of-two scale per 128 x 128 tile): TMA brings the
//    raw 8-bit tile into a staging buffer of the stage; eight more warps turn
//    it into the same swizzled BF16 operand the TMA would have written, with
//    the tile's scale folded in (exact: an E4M3 value times a power of two is
//    a BF16 value), and release the stage to the MMA issuer.  HBM traffic is
//    one byte per element of A.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "umma.h"
#include "umma_ptx.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128;               // output rows per tile (MMA M)
constexpr int BK = 64;                // contraction per stage (one 128-byte swizzle row)
constexpr int A_STAGE_BYTES = BM * BK * 2;
constexpr int THREADS = 192;          // 6 warps
constexpr int THREADS_F8 = 448;       // + 8 converter warps for FP8 A
constexpr int CONV_WARPS = 8;

// 16 E4M3 values (one 16-byte chunk) times a power-of-two scale -> 16 BF16
// values (two 16-byte chunks), element order kept.  Every step is exact:
// E4M3 -> FP16 (a superset), FP16 -> FP32, the scaling, FP32 -> BF16.
__device__ __forceinline__ void e4m3x16_to_bf16(const uint4 v, float sc, uint4& lo, uint4& hi) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint16_t pair = (uint16_t)(w[q] >> (16 * h));
      uint32_t h2;
      asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(pair));
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h2));
      uint32_t b;
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(b) : "f"(f.y * sc), "f"(f.x * sc));
      o[2 * q + h] = b;
    }
  }
  lo = make_uint4(o[0], o[1], o[2], o[3]);
  hi = make_uint4(o[4], o[5], o[6], o[7]);
}

// Fast path of the same conversion for chunks whose 16 codes are all normal
// numbers (exponent field 1..15, not NaN), with integer operations only (the
// floating-point conversions run at a fraction of the ALU rate): an E4M3
// normal (-1)^s 2^(e-7) (1 + m/8) times 2^se is the BF16 number with sign s,
// exponent field e + 120 + se and mantissa m followed by four zero bits.
// Each code is moved into bits 8..15 of a 16-bit half (its sign lands on the
// BF16 sign bit), the magnitude shifted down by 4 and the exponent bias added.
// Needs -120 <= se <= 119.  Returns false (outputs untouched) if a code is
// zero, subnormal or NaN: bytes whose exponent field is 0 are the ones that
// do not carry into bit 7 when 0x78 is added to (code & 0x78); NaN magnitudes
// 0x7F are the ones that do carry when 1 is added to (code & 0x7F).
__device__ __forceinline__ bool e4m3x16_to_bf16_normal(const uint4 v, uint32_t C, uint4& lo,
                                                       uint4& hi) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t normal = 0x80808080u, nan = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    normal &= (w[q] & 0x78787878u) + 0x78787878u;
    nan |= (w[q] & 0x7F7F7F7Fu) + 0x01010101u;
  }
  if (((normal & 0x80808080u) != 0x80808080u) | ((nan & 0x80808080u) != 0)) return false;
  uint32_t o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t xl = __byte_perm(w[q], 0, 0x1404);   // codes 0, 1 in bits 8..15 of the halves
    const uint32_t xh = __byte_perm(w[q], 0, 0x3424);   // codes 2, 3
    o[2 * q] = (((xl >> 4) & 0x07F007F0u) + C) | (xl & 0x80008000u);
    o[2 * q + 1] = (((xh >> 4) & 0x07F007F0u) + C) | (xh & 0x80008000u);
  }
  lo = make_uint4(o[0], o[1], o[2], o[3]);
  hi = make_uint4(o[4], o[5], o[6], o[7]);
  return true;
}

// ---------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------

struct ApassArgs {
  int64_t rows_out;   // output rows (m for AX, n for ATX)
  int64_t total;      // tiles * kt iterations
  int kt;             // k-blocks per tile
  int slices;         // operand slices accumulated into D
  int slice_stride;   // columns between slices in the operand
  int l16;            // MMA N: output columns rounded up to 16 (<= 256)
  int l;              // output columns
  int stages;
  uint32_t tmem_cols;
  float* out;
  int64_t ldo;
  float* part;        // partial slots, gridDim.x * 2 * (MT*128) * l floats
  int accumulate;     // 1: out += result, 0: out = result
  int* status;
  const float* scales;  // FP8 A: tile scales, tile (I, J) at scales[I + J * lds]
  int64_t lds;
  int sc_rows, sc_cols; // tiles of A along m and n
  long long wait_cycles;  // bound of every pipeline wait (the drain waits keep kWaitCycles)
};


// MT: 128-row M sub-tiles per CTA tile (each with its own TMEM accumulator of
// l16 columns); they share every X stage, so X is fetched once per MT*128
// rows of A.
template <bool AX, int MT, bool F8>
__global__ void __launch_bounds__(F8 ? THREADS_F8 : THREADS, 1)
apass_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                  const ApassArgs args) {
  constexpr int BMT = BM * MT;
  constexpr int A_BYTES = A_STAGE_BYTES * MT;
  constexpr int STG_BYTES = F8 ? A_BYTES / 2 : 0;   // raw FP8 tile of the stage
  extern __shared__ uint8_t smem_raw[];
  // carve: barriers first, then 1024-aligned stages [A BF16 | X | FP8 staging]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + args.stages;
  uint64_t* conv = empty + args.stages;           // FP8: converted A ready
  uint64_t* acc_full = conv + args.stages;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t tiles_off = ((raw + 256 + 1023) & ~1023u) - raw;
  uint8_t* tiles = smem_raw + tiles_off;
  const int x_stage_bytes = args.slices * args.l16 * 128;
  const int stage_bytes = A_BYTES + x_stage_bytes + STG_BYTES;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g0 = range_begin(args.total, blockIdx.x, gridDim.x);
  const int64_t g1 = range_begin(args.total, blockIdx.x + 1, gridDim.x);
  if (g0 >= g1) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < args.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], CONV_WARPS);
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
        mbar_expect_tx(&full[s], (uint32_t)(STG_BYTES + (F8 ? x_stage_bytes : stage_bytes)));
        if constexpr (F8) {
          uint8_t* stg = x_s + x_stage_bytes;
          if (AX) {   // boxes of 128 rows (m, 128 bytes) x 64 columns
#pragma unroll
            for (int q = 0; q < MT; ++q)
              tma_load_2d(&tmA, &full[s], stg + q * 8192, (int)(t * BMT + q * 128), kb * BK);
          } else {    // one box of 64 rows (m, 64 bytes) x BMT columns
            tma_load_2d(&tmA, &full[s], stg, kb * BK, (int)(t * BMT));
          }
        } else {
#pragma unroll
          for (int h = 0; h < 2 * MT; ++h) {  // 64-row boxes of the A tile
            if (AX)
              tma_load_2d(&tmA, &full[s], a_s + h * (A_STAGE_BYTES / 2), (int)(t * BMT + h * 64),
                          kb * BK);
            else
              tma_load_2d(&tmA, &full[s], a_s + h * (A_STAGE_BYTES / 2), kb * BK,
                          (int)(t * BMT + h * 64));
          }
        }
        for (int sl = 0; sl < args.slices; ++sl)
          tma_load_2d(&tmX, &full[s], x_s + sl * args.l16 * 128, kb * BK, sl * args.slice_stride);
        ++issued;
        if (++s == args.stages) { s = 0; ph ^= 1u; }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      // on abort: wait (bounded) for the loads already issued to land
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
      const uint32_t idesc = idesc_bf16(BM, args.l16, AX);
      const uint32_t tiles_base = smem_u32(tiles);
      // descriptor start-address steps (in 16-byte units) per 16-wide K step
      constexpr uint64_t a_kstep = AX ? (2048 >> 4) : (32 >> 4);
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
          // the epilogue must have drained the previous segment
          if (!mbar_wait(acc_empty, (uint32_t)((seg - 1) & 1), abort_flag, args.wait_cycles)) { ok = false; break; }
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], ph, abort_flag, args.wait_cycles)) { ok = false; break; }
        if (F8 && !mbar_wait(&conv[s], ph, abort_flag, args.wait_cycles)) { ok = false; break; }
        tc_fence_after();
        const uint32_t a_base = tiles_base + (uint32_t)s * (uint32_t)stage_bytes;
        const uint32_t x_base = a_base + A_BYTES;
        // MN-major A (AX): two 64-element MN atoms per sub-tile, 64 K-rows of
        // 128 bytes each: leading offset BK*128 bytes, 8-row K groups 1024 apart.
        // K-major A (ATX): rows of 128 bytes, 8-row groups 1024 bytes apart.
        const uint64_t bd0 = sdesc(x_base, 16, 1024);
        for (int sl = 0; sl < args.slices; ++sl) {
          const uint64_t bd = bd0 + (uint64_t)((sl * args.l16 * 128) >> 4);
#pragma unroll
          for (int h = 0; h < MT; ++h) {
            const uint32_t ah = a_base + h * A_STAGE_BYTES;
            const uint64_t ad = AX ? sdesc(ah, BK * 128, 1024) : sdesc(ah, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              umma_bf16(tmem_base + h * args.l16, ad + kk * a_kstep, bd + kk * b_kstep, idesc,
                        (seg_first && kk == 0 && sl == 0) ? 0u : 1u);
          }
        }
        umma_commit(&empty[s]);           // stage reusable once these MMAs finish
        if (seg_last) {
          umma_commit(acc_full);          // accumulators ready for the epilogue
          ++seg;
        }
        if (++s == args.stages) { s = 0; ph ^= 1u; }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
      if (!ok) {
        // drain: one more commit tracks every MMA issued so far; wait for it
        // (bounded) so TMEM is idle before it is freed
        umma_commit(acc_full);
        long long t0 = clock64();
        while (!mbar_try_wait(acc_full, (uint32_t)(seg & 1)) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp >= 6) {
    // ---------------- FP8 converter (warps 6 .. 6 + CONV_WARPS - 1) ----------------
    if constexpr (F8) {
      constexpr int TASKS = 4 * MT * 4 / CONV_WARPS;   // 16-code chunks per thread per stage
      const int ct = threadIdx.x - 192;
      // the chunk -> (staging offset, operand offsets, tile) map is the same every stage
      int src_off[TASKS], dst_lo[TASKS], dst_hi[TASKS], tq[TASKS];
#pragma unroll
      for (int i = 0; i < TASKS; ++i) {
        const int task = ct + 32 * CONV_WARPS * i;
        int row, ch0, sw;
        if (AX) {   // task = (q, k, 16-code chunk of the 128 m of box q)
          const int q = task >> 9, k = (task >> 3) & 63, c16 = task & 7;
          src_off[i] = q * 8192 + k * 128 + c16 * 16;
          row = (2 * q + (c16 >> 2)) * 8192 + k * 128;
          ch0 = 2 * (c16 & 3);
          sw = k & 7;
          tq[i] = q;
        } else {    // task = (n, 16-code chunk of the 64 k)
          const int n = task >> 2, c16 = task & 3;
          src_off[i] = n * 64 + c16 * 16;
          row = (n >> 6) * 8192 + (n & 63) * 128;
          ch0 = 2 * c16;
          sw = n & 7;
          tq[i] = n >> 7;
        }
        dst_lo[i] = row + ((ch0 ^ sw) << 4);
        dst_hi[i] = row + (((ch0 + 1) ^ sw) << 4);
      }
      int s = 0;
      uint32_t ph = 0;
      int64_t t = g0 / args.kt;
      int kb = (int)(g0 - t * args.kt);
      for (int64_t g = g0; g < g1; ++g) {
        // warp-uniform outcome: the lanes meet again at __syncwarp below
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, abort_flag, args.wait_cycles))) break;
        uint8_t* a_s = tiles + (size_t)s * stage_bytes;
        const uint8_t* stg = a_s + A_BYTES + x_stage_bytes;
        // scales of the stage's MT tiles: AX walks 128-row tiles I of A at
        // column tile J = k / 128; A^T X walks column tiles at row tile k / 128
        float sc[MT];
        uint32_t cb[MT];
        bool fast[MT];
#pragma unroll
        for (int q = 0; q < MT; ++q) {
          const int64_t tt = t * MT + q, kk = (int64_t)kb * BK / 128;
          const int64_t I = AX ? tt : kk, J = AX ? kk : tt;
          sc[q] = (I < args.sc_rows && J < args.sc_cols) ? __ldg(&args.scales[I + J * args.lds])
                                                         : 0.f;
          // a power-of-two scale's exponent, when the integer path covers it
          const int e = (int)((__float_as_uint(sc[q]) >> 23) & 0xFF) - 127;
          fast[q] = sc[q] > 0.f && e >= -120 && e <= 119;
          cb[q] = (uint32_t)((120 + e) << 7) * 0x00010001u;
        }
#pragma unroll
        for (int i = 0; i < TASKS; ++i) {
          const bool second = MT > 1 && tq[i] != 0;   // selects, not a register-array index
          const float scq = second ? sc[MT - 1] : sc[0];
          const uint32_t cbq = second ? cb[MT - 1] : cb[0];
          const bool fq = second ? fast[MT - 1] : fast[0];
          uint4 lo, hi;
          const uint4 raw = *reinterpret_cast<const uint4*>(stg + src_off[i]);
          if (!fq || !e4m3x16_to_bf16_normal(raw, cbq, lo, hi)) e4m3x16_to_bf16(raw, scq, lo, hi);
          *reinterpret_cast<uint4*>(a_s + dst_lo[i]) = lo;
          *reinterpret_cast<uint4*>(a_s + dst_hi[i]) = hi;
        }
        fence_async_shared();   // the converted tile is read by the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
        if (++s == args.stages) { s = 0; ph ^= 1u; }
        if (++kb == args.kt) { kb = 0; ++t; }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quad = warp & 3;            // TMEM lane quadrant this warp may access
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
      int64_t ld;
      int64_t row0;
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
                float* d = dst + row + (int64_t)(c0 + j) * ld;
                *d = acc_out ? *d + __uint_as_float(r[j]) : __uint_as_float(r[j]);
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// FP8 A as raw bytes: no swizzle (the converter warps read the staging tile
// row by row and write the swizzled BF16 operand themselves).
bool make_map_u8(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_rows, int box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}


}  // namespace

size_t apass_partial_floats(int num_sms, int l) { return (size_t)num_sms * 2 * (2 * BM) * l; }

int launch_apass_bf16(const ApassCall& c, int num_sms, int* status, cudaStream_t st) {
  // shape checks (host-side; the kernel assumes them)
  if (c.lda % 8 || c.ldx % 8 || ((uintptr_t)c.A % 16) || ((uintptr_t)c.X % 16))
    return RSVD_ERR_UNSUPPORTED;
  if (c.fp8 && (c.lda % 16 || !c.scales || c.lds < (c.m + 127) / 128)) return RSVD_ERR_UNSUPPORTED;
  const int64_t rows_out = c.ax ? c.m : c.n;
  const int64_t kdim = c.ax ? c.n : c.m;
  const int l16 = (c.l + 15) / 16 * 16;
  if (c.l < 1 || c.l > 256 || c.slices < 1 || c.slices > 3) return RSVD_ERR_UNSUPPORTED;
  if (c.slice_stride < l16 && c.slices > 1) return RSVD_ERR_UNSUPPORTED;
  // two 128-row sub-tiles per CTA tile when the output has the rows and TMEM
  // holds both accumulators
  const int mt = (rows_out > BM && 2 * l16 <= 512) ? 2 : 1;
  const int bmt = BM * mt;
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(mt * l16)) tmem_cols <<= 1;
  const int64_t tiles = (rows_out + bmt - 1) / bmt;
  const int kt = (int)((kdim + BK - 1) / BK);
  const int64_t total = tiles * kt;
  const int stage_bytes =
      A_STAGE_BYTES * mt + c.slices * l16 * 128 + (c.fp8 ? A_STAGE_BYTES * mt / 2 : 0);
  const int smem_cap = 227 * 1024;
  int stages = (smem_cap - 2048) / stage_bytes;
  stages = std::min(stages, 8);
  if (stages < 2) return RSVD_ERR_UNSUPPORTED;
  const size_t smem = 2048 + (size_t)stages * stage_bytes;

  CUtensorMap tmA, tmX;
  // A: rows x cols = m x n; X: (kdim) x (operand columns) with ld ldx
  if (c.fp8) {
    const bool ok = c.ax ? make_map_u8(&tmA, c.A, c.m, c.n, c.lda, 128, 64)
                         : make_map_u8(&tmA, c.A, c.m, c.n, c.lda, 64, bmt);
    if (!ok) return RSVD_ERR_CUDA;
  } else if (!make_map_bf16(&tmA, c.A, c.m, c.n, c.lda, 64, 64)) {
    return RSVD_ERR_CUDA;
  }
  if (!make_map_bf16(&tmX, c.X, kdim, c.x_cols, c.ldx, 64, l16)) return RSVD_ERR_CUDA;

  // every CTA gets a non-empty range, and no tile is shared by more CTAs than
  // the fixup kernel resolves
  int grid = (int)std::min<int64_t>(std::min<int64_t>(num_sms, total), tiles * 30);
  ApassArgs a;
  a.rows_out = rows_out;
  a.total = total;
  a.kt = kt;
  a.slices = c.slices;
  a.slice_stride = c.slice_stride;
  a.l16 = l16;
  a.l = c.l;
  a.stages = stages;
  a.tmem_cols = tmem_cols;
  a.out = c.out;
  a.ldo = c.ldo;
  a.part = c.part;
  a.accumulate = c.accumulate ? 1 : 0;
  a.status = status;
  a.scales = c.scales;
  a.lds = c.lds;
  a.sc_rows = (int)((c.m + 127) / 128);
  a.sc_cols = (int)((c.n + 127) / 128);
  a.wait_cycles = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
  if (c.part_floats < (size_t)grid * 2 * bmt * c.l) return RSVD_ERR_WORKSPACE;
  if ((int64_t)kt * grid / total + 2 > 32) return RSVD_ERR_UNSUPPORTED;
#define RSVD_LAUNCH_APASS(AXV, MTV, F8V)                                                     \
  do {                                                                                       \
    cudaFuncSetAttribute(apass_bf16_kernel<AXV, MTV, F8V>,                                   \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
    apass_bf16_kernel<AXV, MTV, F8V><<<grid, F8V ? THREADS_F8 : THREADS, smem, st>>>(tmA, tmX, \
                                                                                   a);       \
  } while (0)
#define RSVD_LAUNCH_APASS_T(F8V)                   \
  do {                                             \
    if (c.ax) {                                    \
      if (mt == 2) RSVD_LAUNCH_APASS(true, 2, F8V); \
      else RSVD_LAUNCH_APASS(true, 1, F8V);         \
    } else {                                       \
      if (mt == 2) RSVD_LAUNCH_APASS(false, 2, F8V); \
      else RSVD_LAUNCH_APASS(false, 1, F8V);         \
    }                                              \
  } while (0)
  if (c.fp8) RSVD_LAUNCH_APASS_T(true);
  else RSVD_LAUNCH_APASS_T(false);
#undef RSVD_LAUNCH_APASS_T
#undef RSVD_LAUNCH_APASS
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return RSVD_ERR_CUDA;
  return launch_apass_fixup(c.part, grid, total, kt, bmt, c.l, rows_out, tiles, c.out, c.ldo,
                            a.accumulate, st);
}

}  // namespace rsvd

