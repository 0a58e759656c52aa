// Grouped FP32 products on the tcgen05 tensor cores (the batched form of
// Algorithm 4, Section 3.3: every problem's passes over A, its Gram products
// and its products with R^-1 and the small SVD's factors).
//
// FP32 accuracy from BF16 tensor cores.  An FP32 value v splits into three
// BF16 values v = v1 + v2 + v3 (v1 = bf16(v), v2 = bf16(v - v1),
// v3 = v - v1 - v2; each remainder is exact in FP32 and the last one fits
// eight bits), exactly for |v| >= 2^-110 and to within 2^-134 below that
// (BF16's subnormal step).  A product a x is then the sum of the nine slice products, of
// which the six with i + j <= 4 are kept:
//   a x ~ a1 (x1 + x2 + x3) + a2 (x1 + x2) + a3 x1,
// dropping terms of relative size 2^-24 and below, with FP32 accumulation --
// the accuracy of an FP32 product.
//
// One persistent CTA per SM walks its list of work units (a 128-row x t
// column output tile of one product over a range of 64-deep contraction
// blocks).  Roles (416 threads):
//  * warps 0-7 load A with plain coalesced loads (any lda, any alignment),
//    two blocks ahead in registers, split each value into its three slices
//    and store them in the 128-byte-swizzled layout the MMA reads (MN-major
//    for the AX form, where A's columns are contiguous; K-major for ATX);
//    one of them issues the block's X image (written pre-swizzled by the
//    split kernel) as a single bulk copy; the stage goes to the MMA issuer
//    once the stores (after a proxy fence) and the copy have landed;
//  * warp 8: one lane issues tcgen05.mma (kind::f16, BF16 in, FP32 in TMEM)
//    and tcgen05.commit: five MMAs per 16-deep step, the leading products
//    (a1 x1, a2 x1, a3 x1) into D1 and the rest into D2 | D3, issued
//    alternately; D1 starts from zero every group of DRAIN (2) contraction
//    blocks, two buffers alternating, so the drain of one group overlaps the
//    next group's MMAs;
//  * warps 9-12 drain each group's D1 (tcgen05.ld) into per-row running sums
//    with round-to-nearest FP32 adds (the tensor cores' internal
//    accumulation rounds toward zero; over a long contraction that would
//    bias every sum toward zero), and after the unit's last group add D2 and
//    D3 and store C, or the partial slot of a split tile.
// Every mbarrier wait is bounded; on expiry the CTA records RSVD_ERR_TIMEOUT,
// drains what it issued and frees its TMEM.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <queue>

#include "grouped_tc.h"
#include "umma_ptx.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128;
constexpr int BK = kGtcBlockK;
constexpr int A_SLICE_BYTES = BM * BK * 2;       // one BF16 slice of the A tile (16 KB)
constexpr int A_BYTES = 3 * A_SLICE_BYTES;
constexpr int PROD_WARPS = 8;
constexpr int PROD_THREADS = PROD_WARPS * 32;
constexpr int MMA_WARP = PROD_WARPS;
constexpr int THREADS = (PROD_WARPS + 1 + 4) * 32;
constexpr int EPT = BM * BK / PROD_THREADS;      // A elements per producer thread per block (32)
constexpr int DRAIN = 2;                         // contraction blocks per drained accumulator

__host__ __device__ inline int stage_bytes_of(int t) { return A_BYTES + 3 * t * 128; }

struct GtcArgs {
  const GtcGemm* gemm;
  const GtcUnit* units;
  const int* cta_off;
  float* part;
  int tmax;
  int stages;
  uint32_t tmem_cols;
  int* status;
  long long wait_cycles;
};

// Contiguous global -> shared copy (16-byte aligned, size a multiple of 16),
// completed on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// v -> three BF16 slices (bits), v = f(s1) + f(s2) + f(s3) (exact for
// |v| >= 2^-110).
__device__ __forceinline__ void split3(float v, uint16_t& s1, uint16_t& s2, uint16_t& s3) {
  uint16_t b;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(b) : "f"(v));
  s1 = b;
  const float r1 = v - __uint_as_float((uint32_t)b << 16);
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(b) : "f"(r1));
  s2 = b;
  const float r2 = r1 - __uint_as_float((uint32_t)b << 16);
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(b) : "f"(r2));
  s3 = b;
}

// v0, v1 -> three packed BF16 slice pairs (v0 in the low half), each value
// the sum of its three slices (exact for |v| >= 2^-110).
__device__ __forceinline__ void split3x2(float v0, float v1, uint32_t& s1, uint32_t& s2,
                                         uint32_t& s3) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(s1) : "f"(v1), "f"(v0));
  const float r0 = v0 - __uint_as_float(s1 << 16);
  const float r1 = v1 - __uint_as_float(s1 & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(s2) : "f"(r1), "f"(r0));
  const float q0 = r0 - __uint_as_float(s2 << 16);
  const float q1 = r1 - __uint_as_float(s2 & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(s3) : "f"(q1), "f"(q0));
}
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// The producer's copies of a unit and its product, read from global memory
// once per unit (not once per block): what the A loads need (LUnit) and what
// the X copy needs (XUnit).
struct LUnit {
  const float* A;
  int64_t lda;
  int M, K, row0, kb0, kb1;
};
struct XUnit {
  const uint16_t* xs;
  int col0, kb0, kb1, t, kpad;
};
__device__ __forceinline__ void fetch_unit(const GtcArgs& a, int u, LUnit& p) {
  const GtcUnit un = a.units[u];
  const GtcGemm& G = a.gemm[un.prob];
  p.A = G.A;
  p.lda = G.lda;
  p.M = G.M;
  p.K = G.K;
  p.row0 = un.row0;
  p.kb0 = un.kb0;
  p.kb1 = un.kb1;
}
__device__ __forceinline__ void fetch_unit(const GtcArgs& a, int u, XUnit& p) {
  const GtcUnit un = a.units[u];
  const GtcGemm& G = a.gemm[un.prob];
  p.xs = G.xs;
  p.kpad = G.kpad;
  p.col0 = un.col0;
  p.kb0 = un.kb0;
  p.kb1 = un.kb1;
  p.t = un.t;
}

// A block is 128 tile rows x 64 contraction entries, taken as 4096 pairs of
// neighbours in the swizzled slice layout, PPT per producer thread (index q):
//   AX  (MN-major: neighbours are rows i, i + 1 of one column kk):
//       i = 2 (pt % 64), kk = pt / 64 + SK q -- a warp covers 64 rows of a
//       column, 256 contiguous bytes of A;
//   ATX (K-major: neighbours are kk, kk + 1 of one tile row i):
//       kk = 2 (pt % 32), i = pt / 32 + SI q -- a warp covers 64 entries of
//       one of A's columns.
// Loads walk a per-thread pointer by a fixed stride (SK lda or SI lda).
constexpr int PPT = EPT / 2;                 // pairs per producer thread
constexpr int SK = PROD_THREADS / 64;        // AX: contraction step between a thread's pairs
constexpr int SI = PROD_THREADS / 32;        // ATX: row step between a thread's pairs
static_assert(SI % 8 == 0, "ATX pairs of a thread share their swizzle phase");

template <bool AX>
__device__ __forceinline__ void load_block(const LUnit& U, int kb, int pt, float (&r)[EPT]) {
  const int k0 = kb * BK;
  const float* p;
  int64_t stride;
  bool ok0, ok1;
  int qmax;
  if (AX) {
    const int row = U.row0 + 2 * (pt & 63), k = k0 + (pt >> 6);
    ok0 = row < U.M;
    ok1 = row + 1 < U.M;
    qmax = k < U.K ? (U.K - k + SK - 1) / SK : 0;
    p = U.A + row + (int64_t)k * U.lda;
    stride = SK * U.lda;
  } else {
    const int k = k0 + 2 * (pt & 31), row = U.row0 + (pt >> 5);
    ok0 = k < U.K;
    ok1 = k + 1 < U.K;
    qmax = row < U.M ? (U.M - row + SI - 1) / SI : 0;
    p = U.A + k + (int64_t)row * U.lda;
    stride = SI * U.lda;
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const bool in = q < qmax;
    r[2 * q] = (in && ok0) ? __ldg(p) : 0.f;
    r[2 * q + 1] = (in && ok1) ? __ldg(p + 1) : 0.f;
    p += stride;
  }
}

template <bool AX>
__device__ __forceinline__ void store_block(uint32_t a_s, int pt, const float (&r)[EPT]) {
  if (AX) {
    const int i2 = pt & 63, k0t = pt >> 6;
    const int m = (2 * i2) & 63, c = m >> 3;
    const uint32_t base = (uint32_t)((i2 >> 5) * 8192 + (m & 7) * 2);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      uint32_t s1, s2, s3;
      split3x2(r[2 * q], r[2 * q + 1], s1, s2, s3);
      const int kk = k0t + SK * q;
      const uint32_t o = a_s + base + (uint32_t)(kk * 128 + ((c ^ (kk & 7)) << 4));
      st_shared_u32(o, s1);
      st_shared_u32(o + A_SLICE_BYTES, s2);
      st_shared_u32(o + 2 * A_SLICE_BYTES, s3);
    }
  } else {
    const int kk2 = pt & 31, i0t = pt >> 5;
    const uint32_t base = (uint32_t)((i0t >> 3) * 1024 + (i0t & 7) * 128 +
                                     (((kk2 >> 2) ^ (i0t & 7)) << 4) + ((2 * kk2) & 7) * 2);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      uint32_t s1, s2, s3;
      split3x2(r[2 * q], r[2 * q + 1], s1, s2, s3);
      const uint32_t o = a_s + base + (uint32_t)q * (SI / 8) * 1024;
      st_shared_u32(o, s1);
      st_shared_u32(o + A_SLICE_BYTES, s2);
      st_shared_u32(o + 2 * A_SLICE_BYTES, s3);
    }
  }
}

// The block's X image (3t rows of 128 bytes, already swizzled) as one bulk
// copy completing on the stage's X barrier.
__device__ __forceinline__ void load_x(const XUnit& U, int kb, uint32_t x_s, uint64_t* bar) {
  const uint32_t bytes = (uint32_t)(3 * U.t * 128);
  const int64_t img = (int64_t)(U.col0 / U.t) * (U.kpad / BK) + kb;
  mbar_expect_tx(bar, bytes);
  bulk_g2s(x_s, U.xs + img * (3 * U.t * 64), bytes, bar);
}

template <bool AX>
__global__ void __launch_bounds__(THREADS, 1) gtc_kernel(const GtcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  const int S = args.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);   // producer warps' stores
  uint64_t* xfull = full + S;                                  // the X image's bulk copy
  uint64_t* empty = xfull + S;
  uint64_t* acc_full = empty + S;       // [2] D1 buffer of a group ready
  uint64_t* acc_empty = acc_full + 2;   // [2] D1 buffer drained
  uint64_t* unit_empty = acc_empty + 2; // [2] D2|D3 pair of a unit read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(unit_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t tiles = (raw + 256 + 1023) & ~1023u;   // 1024-aligned stages
  const int tmax = args.tmax;
  const uint32_t stage_bytes = (uint32_t)stage_bytes_of(tmax);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ubeg = args.cta_off[blockIdx.x], uend = args.cta_off[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], PROD_WARPS);
      mbar_init(&xfull[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
      mbar_init(&unit_empty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    tmem_alloc(tmem_slot, args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // the same unit sequence for every role: units of skipped products are
  // passed over by all of them
  auto live = [&](int u) { return args.gemm[args.units[u].prob].M > 0; };

  if (warp < PROD_WARPS) {
    // ---------------- producers ----------------
    const int pt = threadIdx.x;
    int s = 0;
    uint32_t ph = 0;
    // cursors: the block being stored (cs) and the block being loaded (cl,
    // two ahead), each with its unit's descriptor in registers
    auto first_live = [&](int u) {
      while (u < uend && !live(u)) ++u;
      return u;
    };
    auto start = [&](auto& c, int u) {
      c.u = first_live(u);
      if (c.u < uend) {
        fetch_unit(args, c.u, c.p);
        c.kb = c.p.kb0;
      }
    };
    auto advance = [&](auto& c) {
      if (c.u >= uend) return;
      if (++c.kb < c.p.kb1) return;
      start(c, c.u + 1);
    };
    struct {
      int u, kb;
      XUnit p;
    } cs;
    struct {
      int u, kb;
      LUnit p;
    } cl;
    start(cs, ubeg);
    start(cl, ubeg);
    // two blocks of A in flight per thread (register buffers ra, rb)
    float ra[EPT], rb[EPT];
    if (cl.u < uend) load_block<AX>(cl.p, cl.kb, pt, ra);
    advance(cl);
    if (cl.u < uend) load_block<AX>(cl.p, cl.kb, pt, rb);
    bool ok = true;
    int xcount[4] = {0, 0, 0, 0};   // thread 0: X copies issued per stage
    // one stage: the X copy and the slices of the block in r (cs), then the
    // block two ahead into r
    auto step = [&](float (&r)[EPT]) {
      // warp-uniform outcome: the warp's lanes must stay together for
      // __syncwarp below even when a bounded wait expires in some of them
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, abort_flag, args.wait_cycles))) {
        ok = false;
        return;
      }
      const uint32_t a_s = tiles + (uint32_t)s * stage_bytes;
      if (pt == 0) {
        load_x(cs.p, cs.kb, a_s + A_BYTES, &xfull[s]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q == s) ++xcount[q];
      }
      store_block<AX>(a_s, pt, r);
      advance(cl);
      if (cl.u < uend) load_block<AX>(cl.p, cl.kb, pt, r);
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
      advance(cs);
    };
    while (ok && cs.u < uend) {
      step(ra);
      if (!ok || cs.u >= uend) break;
      step(rb);
    }
    // after an abort, the bulk copies still in flight must land before the
    // CTA's shared memory goes away (each wait bounded)
    if (pt == 0 && *abort_flag) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q >= S || xcount[q] == 0) continue;
        const long long t0 = clock64();
        while (!mbar_try_wait(&xfull[q], (uint32_t)((xcount[q] - 1) & 1)) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    // TMEM: D1 (a1 x1 + a2 x1 + a3 x1, the leading part) in two buffers of
    // tmax columns that alternate per group of DRAIN blocks; [D2 | D3]
    // (a1 x2 + a2 x2 | a1 x3, 2^-8 and 2^-16 of D1) in two pairs that
    // alternate per unit.  D1 restarts from zero every group, so the tensor
    // cores' rounding toward zero only spans one group of it; D2 and D3 are
    // small enough to run over the whole unit.
    if (lane == 0) {
      constexpr uint64_t a_kstep = AX ? (2048 >> 4) : (32 >> 4);
      constexpr uint64_t b_kstep = 32 >> 4;
      int s = 0;
      uint32_t ph = 0;
      int g = 0, nu = 0;
      bool ok = true;
      for (int u = ubeg; u < uend && ok; ++u, ++nu) {
        if (!live(u)) {
          --nu;
          continue;
        }
        const GtcUnit un = args.units[u];
        const int t = un.t;
        const uint32_t id1 = idesc_bf16(BM, t, AX);
        const uint32_t id2 = idesc_bf16(BM, 2 * t, AX);
        const int c = nu & 1;
        if (nu >= 2) {
          if (!mbar_wait(&unit_empty[c], (uint32_t)(((nu >> 1) - 1) & 1), abort_flag,
                         args.wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const uint32_t d23 = tmem_base + (uint32_t)(2 * tmax + c * 2 * tmax);
        for (int kg = un.kb0; kg < un.kb1 && ok; kg += DRAIN, ++g) {
          const int b = g & 1;
          if (g >= 2) {
            if (!mbar_wait(&acc_empty[b], (uint32_t)(((g >> 1) - 1) & 1), abort_flag,
                           args.wait_cycles)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t d1 = tmem_base + (uint32_t)(b * tmax);
          const int kend = min(kg + DRAIN, un.kb1);
          for (int kb = kg; kb < kend; ++kb) {
            if (!mbar_wait(&full[s], ph, abort_flag, args.wait_cycles) ||
                !mbar_wait(&xfull[s], ph, abort_flag, args.wait_cycles)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_base = tiles + (uint32_t)s * stage_bytes;
            const uint64_t bd = sdesc(a_base + A_BYTES, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t a1 =
                  (AX ? sdesc(a_base, BK * 128, 1024) : sdesc(a_base, 16, 1024)) + kk * a_kstep;
              const uint64_t a2 = a1 + (A_SLICE_BYTES >> 4);
              const uint64_t a3 = a2 + (A_SLICE_BYTES >> 4);
              const uint64_t x1 = bd + kk * b_kstep;
              const uint64_t x2 = x1 + (uint64_t)((t * 128) >> 4);   // rows t .. 3t-1: x2, x3
              // consecutive MMAs alternate between D1 and D2 | D3
              umma_bf16(d1, a1, x1, id1, (kb > kg || kk > 0) ? 1u : 0u);
              umma_bf16(d23, a1, x2, id2, (kb > un.kb0 || kk > 0) ? 1u : 0u);
              umma_bf16(d1, a2, x1, id1, 1u);
              umma_bf16(d23, a2, x2, id1, 1u);   // N = t: a2 x2 into D2 only
              umma_bf16(d1, a3, x1, id1, 1u);
            }
            umma_commit(&empty[s]);       // stage reusable once these MMAs finish
            if (++s == S) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit(&acc_full[b]);      // D1 of the group (and, after a unit's
                                          // last group, its D2 and D3) ready
        }
      }
      if (!ok) {
        // one more commit tracks every MMA issued; wait (bounded) for it so
        // TMEM is idle before it is freed
        umma_commit(&acc_full[g & 1]);
        const long long t0 = clock64();
        while (!mbar_try_wait(&acc_full[g & 1], (uint32_t)((g >> 1) & 1)) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 9..12) ----------------
    // Thread r owns tile row r.  Each group's D1 goes into the row's running
    // sums (shared memory, column-major 128 x t) with round-to-nearest FP32
    // adds; after the unit's last group the result is
    // (sums + D1) + (D2 + D3), stored to C or to the unit's partial slot.
    const int quad = warp & 3;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    const int r = quad * 32 + lane;
    float* sums = reinterpret_cast<float*>(smem_raw + (tiles - raw) + (size_t)S * stage_bytes);
    int g = 0, nu = 0;
    bool ok = true;
    for (int u = ubeg; u < uend && ok; ++u) {
      if (!live(u)) continue;
      const GtcUnit un = args.units[u];
      const GtcGemm& G = args.gemm[un.prob];
      const int t = un.t;
      const int row = un.row0 + r;
      const int cols = min(t, G.N - un.col0);
      const uint32_t d23 = lane_base + (uint32_t)(2 * tmax + (nu & 1) * 2 * tmax);
      for (int kg = un.kb0; kg < un.kb1; kg += DRAIN, ++g) {
        const int b = g & 1;
        // warp-uniform outcome: tcgen05.ld below is a warp-wide instruction
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)((g >> 1) & 1), abort_flag,
                                               args.wait_cycles))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool first = kg == un.kb0, last = kg + DRAIN >= un.kb1;
        const uint32_t d1 = lane_base + (uint32_t)(b * tmax);
        if (!last) {
          // the group's D1, 16 columns per round trip, into the sums
#pragma unroll
          for (int ch = 0; ch < kGtcMaxTile / 16; ++ch) {
            if (ch * 16 >= t) continue;
            uint32_t v[16];
            tmem_ld16(d1 + (uint32_t)(ch * 16), v);
            tmem_wait_ld();
            float* sp = sums + r + (size_t)ch * 16 * BM;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              sp[j * BM] = first ? __uint_as_float(v[j]) : sp[j * BM] + __uint_as_float(v[j]);
          }
        } else {
#pragma unroll
          for (int ch = 0; ch < kGtcMaxTile / 16; ++ch) {
            if (ch * 16 >= t) continue;
            uint32_t v[16], w[16];
            tmem_ld16(d23 + (uint32_t)(ch * 16), v);
            tmem_ld16(d23 + (uint32_t)(t + ch * 16), w);
            tmem_wait_ld();
            float tail[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) tail[j] = __uint_as_float(v[j]) + __uint_as_float(w[j]);
            tmem_ld16(d1 + (uint32_t)(ch * 16), v);
            tmem_wait_ld();
            const float* sp = sums + r + (size_t)ch * 16 * BM;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float lead = first ? __uint_as_float(v[j]) : sp[j * BM] + __uint_as_float(v[j]);
              const float tot = lead + tail[j];
              const int c = ch * 16 + j;
              if (un.slot >= 0)
                args.part[(size_t)un.slot * BM * tmax + r + (size_t)c * BM] = tot;
              else if (row < G.M && c < cols)
                G.C[row + (int64_t)(un.col0 + c) * G.ldc] = tot;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&acc_empty[b]);
          if (last) mbar_arrive(&unit_empty[nu & 1]);
        }
      }
      ++nu;
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.status, 1 << RSVD_ERR_TIMEOUT);
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem_base, args.tmem_cols);
  }
}

// Split tiles: C tile = sum of its partial slots in slot order (the order of
// the contraction chunks), so the result does not depend on scheduling.
__global__ void gtc_fix_kernel(const GtcGemm* __restrict__ gemm, const GtcFix* __restrict__ fix,
                               const float* __restrict__ part, int tmax) {
  const GtcFix f = fix[blockIdx.x];
  const GtcGemm& G = gemm[f.prob];
  if (G.M <= 0) return;
  const int r = threadIdx.x;   // 128 threads: one per tile row
  const int row = f.row0 + r;
  if (row >= G.M) return;
  const int cols = min(f.t, G.N - f.col0);
  for (int c = 0; c < cols; ++c) {
    float s = 0.f;
    for (int q = 0; q < f.nslot; ++q)
      s += part[(size_t)(f.slot0 + q) * BM * tmax + r + (size_t)c * BM];
    G.C[row + (int64_t)(f.col0 + c) * G.ldc] = s;
  }
}

// Every product's X as its MMA images (see GtcGemm).  Thread e takes 8
// consecutive contraction entries (logical chunk lc) of one column of one
// image, splits each entry once and writes the chunk of all three slices:
// row j = s t + cc of the image, physical chunk lc ^ (j % 8).
__global__ void gtc_split_kernel(const GtcGemm* __restrict__ gemm) {
  const GtcGemm& G = gemm[blockIdx.y];
  if (G.M <= 0) return;
  const int t = G.t, nkb = G.kpad / BK;
  const int nimg = (G.ncols / t) * nkb;
  const int tasks = nimg * t * 8;
  uint4* out = reinterpret_cast<uint4*>(G.xs);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tasks; e += gridDim.x * blockDim.x) {
    const int lc = e & 7, rest = e >> 3;
    const int img = rest / t, cc = rest - img * t;
    const int ct = img / nkb, kb = img - ct * nkb;
    const int c = ct * t + cc, k0 = kb * BK + lc * 8;
    uint32_t w[3][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      uint16_t sl[2][3];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = k0 + 2 * h + q;
        float v = 0.f;
        if (k < G.K && c < G.N && (!G.x_upper || k <= c)) v = G.X[k + (int64_t)c * G.ldx];
        split3(v, sl[q][0], sl[q][1], sl[q][2]);
      }
#pragma unroll
      for (int z = 0; z < 3; ++z) w[z][h] = (uint32_t)sl[0][z] | ((uint32_t)sl[1][z] << 16);
    }
#pragma unroll
    for (int z = 0; z < 3; ++z) {
      const int j = z * t + cc;
      const int64_t row = (int64_t)img * 3 * t + j;
      out[row * 8 + (lc ^ (j & 7))] = make_uint4(w[z][0], w[z][1], w[z][2], w[z][3]);
    }
  }
}

std::mutex g_tune_mu;
int g_chunk[2][2][32];   // [form][one row tile][K bucket] -> blocks per unit (0: not tuned)
int g_tile[32];       // [N bucket] -> column tile limit (0: not tuned)
int g_generation = 0;

}  // namespace

// the running sums of the epilogue (128 x t floats) follow the stages
int gtc_stages(int t) {
  const int cap = 227 * 1024 - 1024 - 256 - BM * t * 4;
  return std::min(4, cap / stage_bytes_of(t));
}

bool gtc_chunk_tuned(bool ax, int K, int M) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  return g_chunk[ax ? 1 : 0][M <= BM ? 1 : 0][gtc_bucket(K)] != 0;
}
int gtc_chunk(bool ax, int K, int M) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const int c = g_chunk[ax ? 1 : 0][M <= BM ? 1 : 0][gtc_bucket(K)];
  return c > 0 ? c : kGtcDefaultChunk;
}
void gtc_set_chunk(bool ax, int K, int M, int chunk_kb) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  int& c = g_chunk[ax ? 1 : 0][M <= BM ? 1 : 0][gtc_bucket(K)];
  if (c == 0 && chunk_kb > 0) {
    c = chunk_kb;
    ++g_generation;
  }
}
int gtc_generation() {
  std::lock_guard<std::mutex> g(g_tune_mu);
  return g_generation;
}
bool gtc_tile_tuned(int N) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  return g_tile[gtc_bucket(N)] != 0;
}
void gtc_set_tile_cap(int N, int cap) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  int& c = g_tile[gtc_bucket(N)];
  if (c == 0 && cap >= 16 && cap <= kGtcMaxTile && cap % 16 == 0) {
    c = cap;
    ++g_generation;
  }
}
int gtc_tile(int N) {
  int cap;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    cap = g_tile[gtc_bucket(N)];
  }
  return gtc_tile_rule(N, cap);
}
void gtc_caps(GtcCaps& c) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (int i = 0; i < 32; ++i) c.cap[i] = g_tile[i];
}

void gtc_schedule(const GtcShape* shapes, int count, bool ax, int num_sms, GtcSchedule& out,
                  int force_chunk, const GtcCaps* caps) {
  out.units.clear();
  out.fix.clear();
  out.slots = 0;
  out.tmax = 16;
  std::vector<GtcUnit> all;
  std::vector<int> cost;
  for (int p = 0; p < count; ++p) {
    const GtcShape& s = shapes[p];
    if (s.M <= 0 || s.N <= 0) continue;
    const int t = caps ? gtc_tile_rule(s.N, caps->cap[gtc_bucket(s.N)]) : gtc_tile(s.N);
    out.tmax = std::max(out.tmax, t);
    const int kbs = std::max(1, (s.K + BK - 1) / BK);
    const int chunk = force_chunk > 0 ? force_chunk : gtc_chunk(ax, s.K, s.M);
    const int nchunk = (kbs + chunk - 1) / chunk;
    for (int r0 = 0; r0 < s.M; r0 += BM)
      for (int c0 = 0; c0 < s.N; c0 += t) {
        if (nchunk == 1) {
          all.push_back({p, r0, c0, 0, kbs, -1, t, 0});
          cost.push_back(kbs + 2);
        } else {
          out.fix.push_back({p, r0, c0, out.slots, nchunk, t});
          for (int q = 0; q < nchunk; ++q) {
            const int k0 = q * kbs / nchunk, k1 = (q + 1) * kbs / nchunk;
            all.push_back({p, r0, c0, k0, k1, out.slots + q, t, 0});
            cost.push_back(k1 - k0 + 2);
          }
          out.slots += nchunk;
        }
      }
  }
  const int n = (int)all.size();
  const int grid = std::max(1, std::min(num_sms, n));
  out.grid = grid;
  // longest first to the least loaded CTA; ties by index (deterministic)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  using Load = std::pair<long long, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < grid; ++c) heap.push({0, c});
  std::vector<std::vector<int>> per(grid);
  for (int i : order) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(i);
    l.first += cost[i];
    heap.push(l);
  }
  out.cta_off.assign(grid + 1, 0);
  out.units.reserve(n);
  for (int c = 0; c < grid; ++c) {
    // within a CTA: by product and tile, so neighbouring units share X in L2
    std::sort(per[c].begin(), per[c].end());
    for (int i : per[c]) out.units.push_back(all[i]);
    out.cta_off[c + 1] = (int)out.units.size();
  }
}

int launch_gtc_split(const GtcGemm* gemm, int count, int max_kpad, int max_ncols,
                     cudaStream_t st) {
  if (count < 1) return RSVD_OK;
  const int64_t chunks = (int64_t)3 * max_kpad * max_ncols / 8;   // 16-byte chunks of the largest
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>(64, (chunks + 255) / 256));
  gtc_split_kernel<<<dim3(bx, count), 256, 0, st>>>(gemm);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

int launch_gtc(const GtcLaunch& L, cudaStream_t st) {
  if (L.tmax < 16 || L.tmax > kGtcMaxTile || L.tmax % 16) return RSVD_ERR_UNSUPPORTED;
  if (L.grid < 1) return RSVD_OK;
  const int stages = gtc_stages(L.tmax);
  if (stages < 2) return RSVD_ERR_UNSUPPORTED;
  GtcArgs a;
  a.gemm = L.gemm;
  a.units = L.units;
  a.cta_off = L.cta_off;
  a.part = L.part;
  a.tmax = L.tmax;
  a.stages = stages;
  uint32_t cols = 32;
  while (cols < (uint32_t)(6 * L.tmax)) cols <<= 1;
  a.tmem_cols = cols;
  a.status = L.status;
  a.wait_cycles = L.wait_cycles > 0 ? L.wait_cycles : kWaitCycles;
  const size_t smem = 1024 + 256 + (size_t)stages * stage_bytes_of(L.tmax) + (size_t)BM * L.tmax * 4;
  if (L.ax) {
    cudaFuncSetAttribute(gtc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gtc_kernel<true><<<L.grid, THREADS, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(gtc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gtc_kernel<false><<<L.grid, THREADS, smem, st>>>(a);
  }
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return RSVD_ERR_CUDA;
  if (L.nfix > 0) {
    gtc_fix_kernel<<<L.nfix, BM, 0, st>>>(L.gemm, L.fix, L.part, L.tmax);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RSVD_ERR_CUDA;
  }
  return RSVD_OK;
}

}  // namespace rsvd
