// FP32-accurate tensor-core GEMMs on tcgen05/TMEM (sm_103a) for the mixed path, built
// from exact TF32 splits: x = hi + lo with hi = x with its 13 low mantissa bits cleared
// (exactly representable in TF32) and lo = x - hi (exact in FP32; its own TF32 rounding
// costs ~2^-22 of x). D (M x N, FP32 accumulation in TMEM) = A (M x K) * B (N x K)^T:
//
//   MODE_Y2  Y = A G (step 2): A row-major (K-major), split on chip; G not split (rounding
//            G only changes the Gaussian test matrix). Products hi(A) G + lo(A) G.
//   MODE_C3  C^T = A^T L~ (step 5): the A tile arrives n-contiguous (MN-major) and is
//            transposed and split on chip; L~ comes pre-split (hi, lo). Products
//            Ahi Lhi + Alo Lhi + Ahi Llo. Also the LUs' large trailing updates
//            (umma3_trail: X's multiplier columns as A, with an epilogue that subtracts the
//            product from the rows still to be eliminated) and two plane products of the
//            fast randomized LU.
//   MODE_G3  Gram L~^T L~ (step 5): both operands pre-split, three products.
//   MODE_Y3  Y = A Z (the power iterations of Section 5): A split on chip as in MODE_Y2, Z
//            pre-split (hi, lo); products hi(A) Zhi + lo(A) Zhi + hi(A) Zlo.
//
// Warp roles: warp 0 TMA producer (ring of STAGES slots, full/empty mbarriers), warp 1
// TMEM allocation and MMA issue, warps 2..5 epilogue (tcgen05.ld), warps 6..9 converter
// (MODE_Y2 / MODE_Y3 / MODE_C3): one thread per tile row. In the one-tile kernel, and in
// the persistent batched kernel with one CTA per SM, the converter stores the row's hi and
// lo parts into tensor memory (tcgen05.st, the thread's own TMEM lane) and the MMAs take A
// from there, so shared memory carries only what TMA brings and what the MMAs read of B;
// in the persistent kernel with two CTAs per SM it writes 128-byte-swizzled K-major hi/lo
// tiles to shared memory and fences them to the async proxy. Either way it arrives on a
// per-slot mbarrier. Every wait is bounded (~1 s) and records an error instead of hanging.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "umma.cuh"

namespace rlu {

static constexpr int U3_BM = 128;
static constexpr int U3_BK = 32;
static constexpr int U3_THREADS = 320;
static constexpr int U3_MAXST = 4;       // ring slots of the persistent batched kernel
static constexpr int U3_MAXST_TILE = 6;  // ring slots of the one-tile kernel
// TMEM of the one-tile kernel: the FP32 accumulator in columns 0..255; for the modes that
// split A on chip, U3_NA buffers of 64 columns (hi(A) in 32, lo(A) in 32; lane = tile row,
// column = K index) at 256 + 64 b
static constexpr int U3_NA = 4;
static constexpr uint32_t U3_ACOL = 256;

struct U3Smem {
  uint64_t full[U3_MAXST_TILE];
  uint64_t conv[U3_MAXST_TILE];
  uint64_t empty[U3_MAXST_TILE];
  uint64_t afree[U3_NA];  // TMEM A buffer b no longer read by the MMAs
  uint64_t accum;
  uint64_t drain;  // final commit of the MMA issuer when a wait gave up
  uint32_t tmem_base;
  int32_t err;
};

namespace u3 {
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mb_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n"
               ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mb_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity) {
  if (mb_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mb_try(bar, parity))
    if (now_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                      uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// the same load with an L2 eviction-priority policy (from evict_first_policy)
__device__ __forceinline__ void tma2d_hint(uint32_t dst, const CUtensorMap* map, int x, int y,
                                           uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}
// L2 policy for data read once (A streamed past operands that other tiles read again)
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}
// A from tensor memory (M rows in lanes 0..M-1, the 8 K values of this MMA in 8 columns
// from tmem_a), B from shared memory
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem, uint32_t tmem_a, uint64_t db,
                                            uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
               ::"r"(tmem), "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc) : "memory");
}
// 32 consecutive columns of this thread's TMEM lane (the warp's 32-lane quarter)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31, %32};\n"
      ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
        "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
        "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]),
        "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]),
        "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               ::"r"(bar) : "memory");
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}
}  // namespace u3

__host__ __device__ constexpr uint32_t u3_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Shared-memory plan of one ring slot (bytes, all multiples of 1024).
struct U3Layout {
  uint32_t a0, a1, a2, b0, b1, stage;
};
__host__ __device__ inline U3Layout u3_layout(int mode, int BN) {
  U3Layout L{};
  const uint32_t at = U3_BM * 128, bt = (uint32_t)BN * 128;
  if (mode == U3_MODE_Y2) {         // a0: TMA A -> hi in place, a1: lo, b0: G
    L.a0 = 0; L.a1 = at; L.b0 = 2 * at; L.b1 = L.b0; L.a2 = 0; L.stage = 2 * at + bt;
  } else if (mode == U3_MODE_Y3) {  // a0: TMA A -> hi in place, a1: lo, b0 Zhi, b1 Zlo
    L.a0 = 0; L.a1 = at; L.b0 = 2 * at; L.b1 = 2 * at + bt; L.a2 = 0; L.stage = 2 * at + 2 * bt;
  } else if (mode == U3_MODE_C3) {  // a2: raw A (n-contiguous), a0 hi, a1 lo, b0 Lhi, b1 Llo
    L.a2 = 0; L.a0 = at; L.a1 = 2 * at; L.b0 = 3 * at; L.b1 = 3 * at + bt; L.stage = 3 * at + 2 * bt;
  } else {                          // G3: a0 hi, a1 lo, b0 hi, b1 lo (all TMA)
    L.a0 = 0; L.a1 = at; L.b0 = 2 * at; L.b1 = 2 * at + bt; L.a2 = 0; L.stage = 2 * at + 2 * bt;
  }
  L.stage = (L.stage + 1023u) & ~1023u;
  return L;
}

// Ring slot of the one-tile kernel: only what TMA brings, since the converter's hi / lo
// parts of A go to tensor memory. Y2: A (a0), G (b0); Y3: A (a0), Zhi (b0), Zlo (b1); C3:
// raw n-contiguous A (a2), Lhi (b0), Llo (b1); G3 as in the batched layout.
__host__ __device__ inline U3Layout u3_tile_layout(int mode, int BN) {
  U3Layout L = u3_layout(mode, BN);
  const uint32_t at = U3_BM * 128, bt = (uint32_t)BN * 128;
  if (mode == U3_MODE_Y2) {
    L.a0 = 0; L.a1 = 0; L.b0 = at; L.b1 = at; L.a2 = 0; L.stage = at + bt;
  } else if (mode == U3_MODE_Y3) {
    L.a0 = 0; L.a1 = 0; L.b0 = at; L.b1 = at + bt; L.a2 = 0; L.stage = at + 2 * bt;
  } else if (mode == U3_MODE_C3) {
    L.a2 = 0; L.a0 = 0; L.a1 = 0; L.b0 = at; L.b1 = at + bt; L.stage = at + 2 * bt;
  }
  L.stage = (L.stage + 1023u) & ~1023u;
  return L;
}

// One 128-row tile (mt) of N tile nt over K slice kz; the tensor maps are read by address
// (kernel parameters or, for the batched form, records in global memory).
template <int MODE>
__device__ __forceinline__ void umma3_tile(const CUtensorMap& mA0, const CUtensorMap& mA1,
                                           const CUtensorMap& mB0, const CUtensorMap& mB1,
                                           const Umma3Args& a, int mt, int kz, int nt) {
  using namespace u3;
  extern __shared__ __align__(1024) unsigned char u3_smem[];
  U3Smem& sh = *reinterpret_cast<U3Smem*>(u3_smem);
  const uint32_t tiles = (su32(u3_smem) + sizeof(U3Smem) + 1023u) & ~1023u;
  const U3Layout lay = u3_tile_layout(MODE, a.BN);
  const int S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = mt * U3_BM;
  const int nb0 = nt * a.BN;  // first column of this CTA's N tile
  const int k_begin = kz * a.kchunk;
  const int k_end = min(a.K, k_begin + a.kchunk);
  const int nk = (k_end - k_begin + U3_BK - 1) / U3_BK;
  constexpr bool CONV = (MODE != U3_MODE_G3);
  constexpr uint32_t TCOLS = CONV ? 512u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(su32(&sh.full[s]), 1);
      mb_init(su32(&sh.conv[s]), 128);
      mb_init(su32(&sh.empty[s]), 1);
    }
    mb_init(su32(&sh.accum), 1);
    mb_init(su32(&sh.drain), 1);
    for (int b = 0; b < U3_NA; ++b) mb_init(su32(&sh.afree[b]), 1);
    sh.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(su32(&sh.tmem_base)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sh.tmem_base;
  int issued = 0;  // k-steps whose loads the producer started

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ------------------------------------------------------------------
    uint32_t tx = lay.stage;
    if (MODE == U3_MODE_Y2) tx = 2 * 0 + U3_BM * 128 + (uint32_t)a.BN * 128;
    if (MODE == U3_MODE_C3) tx = U3_BM * 128 + 2 * (uint32_t)a.BN * 128;
    if (MODE == U3_MODE_G3) tx = 2 * U3_BM * 128 + 2 * (uint32_t)a.BN * 128;
    if (MODE == U3_MODE_Y3) tx = U3_BM * 128 + 2 * (uint32_t)a.BN * 128;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      if (kt >= S && !mb_wait(su32(&sh.empty[s]), (uint32_t)(((kt / S) - 1) & 1))) {
        sh.err = 1;
        break;
      }
      const uint32_t base = tiles + s * lay.stage;
      const uint32_t bar = su32(&sh.full[s]);
      mb_expect_tx(bar, tx);
      const int kx = k_begin + kt * U3_BK;
      if (MODE == U3_MODE_Y2) {
        tma2d(base + lay.a0, &mA0, kx, m0, bar);
        tma2d(base + lay.b0, &mB0, kx, nb0, bar);
      } else if (MODE == U3_MODE_Y3) {
        tma2d(base + lay.a0, &mA0, kx, m0, bar);
        tma2d(base + lay.b0, &mB0, kx, nb0, bar);
        tma2d(base + lay.b1, &mB1, kx, nb0, bar);
      } else if (MODE == U3_MODE_C3) {
        tma2d(base + lay.a2, &mA0, m0, kx, bar);   // raw A: x = n (128 wide), y = m
        tma2d(base + lay.b0, &mB0, kx, nb0, bar);
        tma2d(base + lay.b1, &mB1, kx, nb0, bar);
      } else {
        tma2d(base + lay.a0, &mA0, kx, m0, bar);
        tma2d(base + lay.a1, &mA1, kx, m0, bar);
        tma2d(base + lay.b0, &mB0, kx, nb0, bar);
        tma2d(base + lay.b1, &mB1, kx, nb0, bar);
      }
      issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer --------------------------------------------------------------------
    const uint32_t idesc = u3_idesc(U3_BM, a.BN);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      const uint32_t par = (uint32_t)((kt / S) & 1);
      if (!mb_wait(su32(CONV ? &sh.conv[s] : &sh.full[s]), par)) {
        sh.err = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tiles + s * lay.stage;
      if (CONV) {
        // A's hi / lo parts of this k-step in TMEM buffer kt % U3_NA
        const uint32_t abuf = tmem + U3_ACOL + (uint32_t)(kt % U3_NA) * 64u;
#pragma unroll
        for (int kk = 0; kk < U3_BK / 8; ++kk) {
          const uint32_t off = kk * 32;
          const uint64_t bh = desc_sw128(base + lay.b0 + off), bl = desc_sw128(base + lay.b1 + off);
          const uint32_t ah = abuf + (uint32_t)kk * 8u, al = ah + 32u;
          mma_tf32_ts(tmem, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          mma_tf32_ts(tmem, al, bh, idesc, 1u);
          if (MODE != U3_MODE_Y2) mma_tf32_ts(tmem, ah, bl, idesc, 1u);
        }
        commit(su32(&sh.empty[s]));
        commit(su32(&sh.afree[kt % U3_NA]));
      } else {
#pragma unroll
        for (int kk = 0; kk < U3_BK / 8; ++kk) {
          const uint32_t off = kk * 32;
          const uint64_t ah = desc_sw128(base + lay.a0 + off), al = desc_sw128(base + lay.a1 + off);
          const uint64_t bh = desc_sw128(base + lay.b0 + off), bl = desc_sw128(base + lay.b1 + off);
          mma_tf32(tmem, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, al, bh, idesc, 1u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
        }
        commit(su32(&sh.empty[s]));
      }
    }
    commit(su32(&sh.accum));
  } else if (warp >= 2 && warp < 6) {
    // ---- epilogue ------------------------------------------------------------------------
    const bool ok = mb_wait(su32(&sh.accum), 0u);
    if (!ok) sh.err = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    float* __restrict__ out = a.out + (size_t)kz * a.split_stride;
    const bool sub = a.sub_pos != nullptr;  // out -= D in the rows still to be eliminated
    const bool live = row < a.M && (!sub || a.sub_pos[row] >= a.sub_min);
    for (int c0 = 0; c0 < a.BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (ok && live && sub) {
        // all 32 loads first: stores between them would serialise their latencies
        float cur[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = nb0 + c0 + j;
          cur[j] = col < a.N ? out[(size_t)col * a.ldo + row] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = nb0 + c0 + j;
          if (col < a.N) out[(size_t)col * a.ldo + row] = cur[j] - __uint_as_float(v[j]);
        }
      } else if (ok && live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = nb0 + c0 + j;
          if (col < a.N) {
            const float f = __uint_as_float(v[j]);
            if (a.out_colmajor)
              out[(size_t)col * a.ldo + row] = f;
            else
              out[(size_t)row * a.ldo + col] = f;
          }
        }
      }
    }
  } else if (CONV && warp >= 6) {
    // ---- converter: one thread per tile row; row r = TMEM lane r, so warp w serves the
    // rows of its lane quarter w % 4 ------------------------------------------------------
    const int q = warp & 3;
    const int r = q * 32 + lane;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      if (!mb_wait(su32(&sh.full[s]), (uint32_t)((kt / S) & 1))) {
        sh.err = 1;
        break;
      }
      // TMEM buffer kt % U3_NA is free once the MMAs of k-step kt - U3_NA completed
      if (kt >= U3_NA &&
          !mb_wait(su32(&sh.afree[kt % U3_NA]), (uint32_t)(((kt / U3_NA) - 1) & 1))) {
        sh.err = 1;
        break;
      }
      const uint32_t base = tiles + s * lay.stage;
      uint32_t h[32], l[32];
      if (MODE == U3_MODE_Y2 || MODE == U3_MODE_Y3) {
        // row r of the 128-byte-swizzled A tile: logical 16-byte chunk c sits at chunk
        // c ^ (r & 7), so the 8 threads of each quarter warp hit 8 different bank groups
        const float4* row =
            reinterpret_cast<const float4*>(u3_smem + (base + lay.a0 - su32(u3_smem))) + r * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = row[c ^ (r & 7)];
          float hx, lx;
          split_tf32(v.x, hx, lx);
          h[4 * c + 0] = __float_as_uint(hx);
          l[4 * c + 0] = __float_as_uint(lx);
          split_tf32(v.y, hx, lx);
          h[4 * c + 1] = __float_as_uint(hx);
          l[4 * c + 1] = __float_as_uint(lx);
          split_tf32(v.z, hx, lx);
          h[4 * c + 2] = __float_as_uint(hx);
          l[4 * c + 2] = __float_as_uint(lx);
          split_tf32(v.w, hx, lx);
          h[4 * c + 3] = __float_as_uint(hx);
          l[4 * c + 3] = __float_as_uint(lx);
        }
      } else {
        // raw tile: 32 rows (K) x 128 floats (M), row-major; tile row r is its column r
        const float* raw = reinterpret_cast<const float*>(u3_smem + (base + lay.a2 - su32(u3_smem)));
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float hx, lx;
          split_tf32(raw[j * U3_BM + r], hx, lx);
          h[j] = __float_as_uint(hx);
          l[j] = __float_as_uint(lx);
        }
      }
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + U3_ACOL + (uint32_t)(kt % U3_NA) * 64u;
      tmem_st32(taddr, h);
      tmem_st32(taddr + 32u, l);
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mb_arrive(su32(&sh.conv[s]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (sh.err) {
    // a wait gave up: let the work already issued finish (bounded) before TMEM is freed
    // and the CTA exits. The MMA issuer's final commit covers every MMA it issued; the
    // producer waits for the loads of the last S k-steps it started.
    if (warp == 1 && lane == 0) {
      commit(su32(&sh.drain));
      mb_wait(su32(&sh.drain), 0u);
    }
    if (warp == 0 && lane == 0)
      for (int kt = issued > S ? issued - S : 0; kt < issued; ++kt)
        mb_wait(su32(&sh.full[kt % S]), (uint32_t)((kt / S) & 1));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 ::"r"(tmem), "r"(TCOLS) : "memory");
  }
  if (threadIdx.x == 0 && sh.err && a.status) atomicExch(a.status, RLU_ETIMEOUT);
}

template <int MODE>
__global__ void __launch_bounds__(U3_THREADS, 1)
k_umma3(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
        const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
        Umma3Args a) {
  // grid x = N tile fastest, then 128-row tile: the CTAs that share an A tile run together
  // and A is fetched from DRAM once, the other N tiles hitting L2
  const int nt = (int)blockIdx.x % a.ntiles, mt = (int)blockIdx.x / a.ntiles;
  umma3_tile<MODE>(mA0, mA1, mB0, mB1, a, mt, blockIdx.y, nt);
}

// Persistent batched form (Y2 and C3, every BN <= 128). The producer thread takes the next
// tile of the list from a global counter (dynamic: CTAs that finish early take more, and
// neighbouring tiles of one problem start at about the same time, so the operand they
// share is read from L2) and passes its index to the other roles through a small queue in
// shared memory. Setup (barriers, TMEM) happens once; the producer, the converter and the
// MMA issuer run one ring of k-steps across the CTA's tiles, so a tile's first loads are in
// flight while the previous tile drains; the accumulator is double buffered in TMEM
// (columns 0 and 128), so the epilogue of one tile overlaps the MMAs of the next. Ring slots
// are slot bytes apart (the largest slot of the batch). With TA (one CTA per SM) the
// converter stores A's hi / lo parts into tensor memory (U3_NA buffers of 64 columns after
// the two accumulators) and the MMAs read A from there, as in the one-tile kernel; without
// it (two CTAs per SM, 256 TMEM columns each) they go through the ring slot in shared memory.
// Every wait is bounded: a wait that gives up sets RLU_ETIMEOUT in the tile's status (or its
// CTA's first tile's) and ends the role.
static constexpr int U3_QN = 4;  // tile queue depth
struct U3PSmem {
  uint64_t full[U3_MAXST];
  uint64_t conv[U3_MAXST];
  uint64_t empty[U3_MAXST];
  uint64_t accf[2];       // accumulator buffer b complete (MMA commit)
  uint64_t acce[2];       // accumulator buffer b read (4 epilogue warps)
  uint64_t qfull[U3_QN];  // queue entry written (producer)
  uint64_t qempty[U3_QN]; // queue entry read (MMA 1 + converter 4 warps + epilogue 4 warps)
  uint64_t drain;         // final commit of the MMA issuer when a wait gave up
  uint64_t afree[U3_NA];  // TA: TMEM A buffer b no longer read by the MMAs
  int queue[U3_QN];       // tile indices, -1 = no more tiles
  uint32_t tmem_base;
  int32_t err;
};

// Ring slot of the persistent kernel: the one-tile layout when A's parts live in TMEM.
__host__ __device__ inline U3Layout u3_persist_layout(int mode, int BN, bool ta) {
  return ta ? u3_tile_layout(mode, BN) : u3_layout(mode, BN);
}

template <int MODE, bool TA>
__global__ void __launch_bounds__(U3_THREADS, 1) k_umma3_persist(const U3Job* __restrict__ jobs,
                                                                 const int2* __restrict__ tiles,
                                                                 int ntiles, int S,
                                                                 uint32_t slot,
                                                                 unsigned* __restrict__ next) {
  using namespace u3;
  extern __shared__ __align__(1024) unsigned char u3_smem[];
  U3PSmem& sh = *reinterpret_cast<U3PSmem*>(u3_smem);
  const uint32_t ring = (su32(u3_smem) + sizeof(U3PSmem) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mb_init(su32(&sh.full[st]), 1);
      mb_init(su32(&sh.conv[st]), 128);
      mb_init(su32(&sh.empty[st]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mb_init(su32(&sh.accf[b]), 1);
      mb_init(su32(&sh.acce[b]), 4);
    }
    for (int q = 0; q < U3_QN; ++q) {
      mb_init(su32(&sh.qfull[q]), 1);
      mb_init(su32(&sh.qempty[q]), 9);
    }
    mb_init(su32(&sh.drain), 1);
    for (int b = 0; b < U3_NA; ++b) mb_init(su32(&sh.afree[b]), 1);
    sh.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  constexpr uint32_t TCOLS = TA ? 512u : 256u;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(su32(&sh.tmem_base)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sh.tmem_base;
  volatile int32_t* err = &sh.err;
  auto fail = [&](const Umma3Args& a) {
    *err = 1;
    if (a.status) atomicExch(a.status, RLU_ETIMEOUT);
  };
  const Umma3Args& a_first = jobs[tiles[min((int)blockIdx.x, ntiles - 1)].x].a;
  uint32_t issued = 0;  // ring k-steps whose loads the producer started
  // the it-th tile of this CTA from the queue (-1: none left, or a wait gave up); the
  // reader's arrival frees the entry
  auto take = [&](int it, int arrivals) -> int {
    const int q = it % U3_QN;
    if (!mb_wait(su32(&sh.qfull[q]), (uint32_t)((it / U3_QN) & 1))) {
      fail(a_first);
      return -1;
    }
    const int ti = *reinterpret_cast<volatile int*>(&sh.queue[q]);
    if (arrivals) mb_arrive(su32(&sh.qempty[q]));
    return ti;
  };

  if (warp == 0 && lane == 0) {
    // ---- TMA producer and tile scheduler -----------------------------------------------
    uint32_t g = 0;
    const uint64_t pol_a = evict_first_policy();
    for (int it = 0; !*err; ++it) {
      const int q = it % U3_QN;
      if (it >= U3_QN && !mb_wait(su32(&sh.qempty[q]), (uint32_t)(((it / U3_QN) - 1) & 1))) {
        fail(a_first);
        break;
      }
      const int ti = (int)atomicAdd(next, 1u);
      sh.queue[q] = ti < ntiles ? ti : -1;
      mb_arrive(su32(&sh.qfull[q]));
      if (ti >= ntiles) break;
      const int2 t = tiles[ti];
      const U3Job& j = jobs[t.x];
      const Umma3Args& a = j.a;
      const U3Layout lay = u3_persist_layout(MODE, a.BN, TA);
      const uint32_t tx = MODE == U3_MODE_Y2 ? U3_BM * 128 + (uint32_t)a.BN * 128
                                             : U3_BM * 128 + 2 * (uint32_t)a.BN * 128;
      const int m0 = t.y * U3_BM;
      const int nk = (a.K + U3_BK - 1) / U3_BK;
      for (int kt = 0; kt < nk; ++kt, ++g) {
        const uint32_t st = g % (uint32_t)S;
        if (g >= (uint32_t)S && !mb_wait(su32(&sh.empty[st]), ((g / S) - 1) & 1)) {
          fail(a);
          break;
        }
        const uint32_t base = ring + st * slot;
        const uint32_t bar = su32(&sh.full[st]);
        mb_expect_tx(bar, tx);
        const int kx = kt * U3_BK;
        // A is read once per tile; G (Y2) and L~'s parts (C3) are read by every row tile
        // of the problem, so A goes first when L2 evicts
        if (MODE == U3_MODE_Y2) {
          tma2d_hint(base + lay.a0, &j.map[0], kx, m0, bar, pol_a);
          tma2d(base + lay.b0, &j.map[2], kx, 0, bar);
        } else {
          tma2d_hint(base + lay.a2, &j.map[0], m0, kx, bar, pol_a);  // raw A: x = n, y = m
          tma2d(base + lay.b0, &j.map[2], kx, 0, bar);
          tma2d(base + lay.b1, &j.map[3], kx, 0, bar);
        }
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer --------------------------------------------------------------------
    uint32_t g = 0;
    for (int it = 0; !*err; ++it) {
      const int ti = take(it, 1);
      if (ti < 0) break;
      const int2 t = tiles[ti];
      const Umma3Args& a = jobs[t.x].a;
      const U3Layout lay = u3_persist_layout(MODE, a.BN, TA);
      const int buf = it & 1;
      if (it >= 2 && !mb_wait(su32(&sh.acce[buf]), (uint32_t)(((it / 2) - 1) & 1))) {
        fail(a);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t idesc = u3_idesc(U3_BM, a.BN);
      const uint32_t acc = tmem + (uint32_t)(buf * 128);
      const int nk = (a.K + U3_BK - 1) / U3_BK;
      bool ok = true;
      for (int kt = 0; kt < nk; ++kt, ++g) {
        const uint32_t st = g % (uint32_t)S;
        if (!mb_wait(su32(&sh.conv[st]), (g / S) & 1)) {
          fail(a);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t base = ring + st * slot;
        if (TA) {  // A's parts of ring step g in TMEM buffer g % U3_NA
          const uint32_t abuf = tmem + U3_ACOL + (g % (uint32_t)U3_NA) * 64u;
#pragma unroll
          for (int kk = 0; kk < U3_BK / 8; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t bh = desc_sw128(base + lay.b0 + off), bl = desc_sw128(base + lay.b1 + off);
            const uint32_t ah = abuf + (uint32_t)kk * 8u, al = ah + 32u;
            mma_tf32_ts(acc, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_tf32_ts(acc, al, bh, idesc, 1u);
            if (MODE != U3_MODE_Y2) mma_tf32_ts(acc, ah, bl, idesc, 1u);
          }
          commit(su32(&sh.empty[st]));
          commit(su32(&sh.afree[g % (uint32_t)U3_NA]));
        } else {
#pragma unroll
          for (int kk = 0; kk < U3_BK / 8; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t ah = desc_sw128(base + lay.a0 + off), al = desc_sw128(base + lay.a1 + off);
            const uint64_t bh = desc_sw128(base + lay.b0 + off), bl = desc_sw128(base + lay.b1 + off);
            mma_tf32(acc, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(acc, al, bh, idesc, 1u);
            if (MODE != U3_MODE_Y2) mma_tf32(acc, ah, bl, idesc, 1u);
          }
          commit(su32(&sh.empty[st]));
        }
      }
      if (!ok) break;
      commit(su32(&sh.accf[buf]));
    }
  } else if (warp >= 2 && warp < 6) {
    // ---- epilogue ------------------------------------------------------------------------
    const int quarter = warp & 3;
    for (int it = 0; !__shfl_sync(0xffffffffu, *err, 0); ++it) {  // warp-uniform test
      // every lane reads; lane 0's outcome is the warp's (the tcgen05.ld below needs all 32
      // lanes), and lane 0 frees the entry for the warp
      const int ti = __shfl_sync(0xffffffffu, take(it, 0), 0);
      if (lane == 0) mb_arrive(su32(&sh.qempty[it % U3_QN]));
      if (ti < 0) break;
      const int2 t = tiles[ti];
      const Umma3Args& a = jobs[t.x].a;
      const int buf = it & 1;
      const bool done = mb_wait(su32(&sh.accf[buf]), (uint32_t)((it / 2) & 1));
      if (!__shfl_sync(0xffffffffu, done ? 1 : 0, 0)) {
        fail(a);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int row = t.y * U3_BM + quarter * 32 + lane;
      for (int c0 = 0; c0 < a.BN; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr =
            tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 128 + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
            "%28, %29, %30, %31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (row < a.M) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int col = c0 + jj;
            if (col < a.N) {
              const float f = __uint_as_float(v[jj]);
              if (a.out_colmajor)
                a.out[(size_t)col * a.ldo + row] = f;
              else
                a.out[(size_t)row * a.ldo + col] = f;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mb_arrive(su32(&sh.acce[buf]));
    }
  } else if (warp >= 6) {
    // ---- converter: one thread per tile row (128 rows) ------------------------------------
    // TA: row r = TMEM lane r, so warp w serves the rows of its lane quarter w % 4
    const int r = TA ? (warp & 3) * 32 + lane : threadIdx.x - 192;  // 0..127
    uint32_t g = 0;
    for (int it = 0; !__shfl_sync(0xffffffffu, *err, 0); ++it) {  // warp-uniform test
      const int ti = __shfl_sync(0xffffffffu, take(it, 0), 0);  // lane 0's outcome
      if (lane == 0) mb_arrive(su32(&sh.qempty[it % U3_QN]));
      if (ti < 0) break;
      const int2 t = tiles[ti];
      const Umma3Args& a = jobs[t.x].a;
      const U3Layout lay = u3_persist_layout(MODE, a.BN, TA);
      const int nk = (a.K + U3_BK - 1) / U3_BK;
      bool ok = true;
      for (int kt = 0; kt < nk; ++kt, ++g) {
        const uint32_t st = g % (uint32_t)S;
        const bool got = mb_wait(su32(&sh.full[st]), (g / S) & 1);
        if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {  // lane 0's outcome, warp-uniform
          fail(a);
          ok = false;
          break;
        }
        const uint32_t base = ring + st * slot;
        if (TA) {
          // TMEM buffer g % U3_NA is free once the MMAs of ring step g - U3_NA completed
          const bool fr = g < (uint32_t)U3_NA ||
                          mb_wait(su32(&sh.afree[g % (uint32_t)U3_NA]), ((g / U3_NA) - 1) & 1);
          if (!__shfl_sync(0xffffffffu, fr ? 1 : 0, 0)) {
            fail(a);
            ok = false;
            break;
          }
          uint32_t h[32], l[32];
          if (MODE == U3_MODE_Y2) {  // swizzled row r: logical chunk c at chunk c ^ (r & 7)
            const float4* row =
                reinterpret_cast<const float4*>(u3_smem + (base + lay.a0 - su32(u3_smem))) + r * 8;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const float4 v = row[c ^ (r & 7)];
              const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                float hx, lx;
                split_tf32(vv[e], hx, lx);
                h[4 * c + e] = __float_as_uint(hx);
                l[4 * c + e] = __float_as_uint(lx);
              }
            }
          } else {  // raw tile: 32 rows (K) x 128 floats (M); tile row r is its column r
            const float* raw = reinterpret_cast<const float*>(u3_smem + (base + lay.a2 - su32(u3_smem)));
#pragma unroll
            for (int jx = 0; jx < 32; ++jx) {
              float hx, lx;
              split_tf32(raw[jx * U3_BM + r], hx, lx);
              h[jx] = __float_as_uint(hx);
              l[jx] = __float_as_uint(lx);
            }
          }
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + U3_ACOL +
                                 (g % (uint32_t)U3_NA) * 64u;
          tmem_st32(taddr, h);
          tmem_st32(taddr + 32u, l);
          asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          mb_arrive(su32(&sh.conv[st]));
          continue;
        }
        if (MODE == U3_MODE_Y2) {
          float* hi = reinterpret_cast<float*>(u3_smem + (base + lay.a0 - su32(u3_smem))) + r * 32;
          float* lo = reinterpret_cast<float*>(u3_smem + (base + lay.a1 - su32(u3_smem))) + r * 32;
#pragma unroll
          for (int c0 = 0; c0 < 8; ++c0) {
            const int c = (c0 + r) & 7;
            float4 v = *reinterpret_cast<float4*>(hi + 4 * c);
            float4 h, l;
            split_tf32(v.x, h.x, l.x);
            split_tf32(v.y, h.y, l.y);
            split_tf32(v.z, h.z, l.z);
            split_tf32(v.w, h.w, l.w);
            *reinterpret_cast<float4*>(hi + 4 * c) = h;
            *reinterpret_cast<float4*>(lo + 4 * c) = l;
          }
        } else {
          const float* raw = reinterpret_cast<const float*>(u3_smem + (base + lay.a2 - su32(u3_smem)));
          float* hi = reinterpret_cast<float*>(u3_smem + (base + lay.a0 - su32(u3_smem))) + r * 32;
          float* lo = reinterpret_cast<float*>(u3_smem + (base + lay.a1 - su32(u3_smem))) + r * 32;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            float4 h, l;
            split_tf32(raw[(4 * c + 0) * U3_BM + r], h.x, l.x);
            split_tf32(raw[(4 * c + 1) * U3_BM + r], h.y, l.y);
            split_tf32(raw[(4 * c + 2) * U3_BM + r], h.z, l.z);
            split_tf32(raw[(4 * c + 3) * U3_BM + r], h.w, l.w);
            const int pc = c ^ (r & 7);
            *reinterpret_cast<float4*>(hi + 4 * pc) = h;
            *reinterpret_cast<float4*>(lo + 4 * pc) = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mb_arrive(su32(&sh.conv[st]));
      }
      if (!ok) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (*err) {
    // a wait gave up: let the work already issued finish (bounded) before TMEM is freed
    // and the CTA exits (the MMA issuer's final commit covers every MMA it issued; the
    // producer waits for the loads of the last S ring steps it started)
    if (warp == 1 && lane == 0) {
      commit(su32(&sh.drain));
      mb_wait(su32(&sh.drain), 0u);
    }
    if (warp == 0 && lane == 0)
      for (uint32_t g = issued > (uint32_t)S ? issued - S : 0; g < issued; ++g)
        mb_wait(su32(&sh.full[g % S]), (g / S) & 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// FP32 row-major (rows x cols, ld) tensor map with a box of box_x columns x box_y rows.
static int32_t map2d(CUtensorMap* map, const float* base, int64_t rows, int64_t cols,
                     int64_t ld, int box_x, int box_y, bool swizzle) {
  auto enc = encode_fn();
  if (!enc) return RLU_ECUDA;
  if (((uintptr_t)base & 15u) != 0 || (ld * 4) % 16 != 0) return RLU_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RLU_OK : RLU_ECUDA;
}

template <int MODE>
static int32_t launch_u3(const Umma3Op& op, cudaStream_t s) {
  if (op.M <= 0 || op.N <= 0 || op.K <= 0) return RLU_EINVAL;
  // N tiles of up to 256 columns (one TMEM accumulator each), one per grid z index
  const int BN = op.N > 256 ? 256 : (int)round_up(op.N, 16);
  const int ntiles = (int)ceil_div(op.N, BN);
  const U3Layout lay = u3_tile_layout(MODE, BN);
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int ctrl = 2048;
  int stages = (int)((optin - ctrl) / (int)lay.stage);
  if (stages > U3_MAXST_TILE) stages = U3_MAXST_TILE;
  if (stages < 2) return RLU_EUNSUPPORTED;
  const size_t smem = (size_t)ctrl + (size_t)stages * lay.stage;
  CUtensorMap m0{}, m1{}, n0{}, n1{};
  if (MODE == U3_MODE_Y2) {
    RLU_TRY(map2d(&m0, op.A0, op.M, op.K, op.lda, U3_BK, U3_BM, true));
    RLU_TRY(map2d(&n0, op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    m1 = m0;
    n1 = n0;
  } else if (MODE == U3_MODE_Y3) {
    RLU_TRY(map2d(&m0, op.A0, op.M, op.K, op.lda, U3_BK, U3_BM, true));
    RLU_TRY(map2d(&n0, op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    RLU_TRY(map2d(&n1, op.B1, op.N, op.K, op.ldb, U3_BK, BN, true));
    m1 = m0;
  } else if (MODE == U3_MODE_C3) {
    // A stored row-major K x M (rows = K index, M contiguous): box 128 (M) x 32 (K)
    RLU_TRY(map2d(&m0, op.A0, op.K, op.M, op.lda, U3_BM, U3_BK, false));
    RLU_TRY(map2d(&n0, op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    RLU_TRY(map2d(&n1, op.B1, op.N, op.K, op.ldb, U3_BK, BN, true));
    m1 = m0;
  } else {
    RLU_TRY(map2d(&m0, op.A0, op.M, op.K, op.lda, U3_BK, U3_BM, true));
    RLU_TRY(map2d(&m1, op.A1, op.M, op.K, op.lda, U3_BK, U3_BM, true));
    RLU_TRY(map2d(&n0, op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    RLU_TRY(map2d(&n1, op.B1, op.N, op.K, op.ldb, U3_BK, BN, true));
  }
  int splits = op.splits < 1 ? 1 : op.splits;
  const int kchunk = (int)round_up(ceil_div(op.K, splits), U3_BK);
  splits = (int)ceil_div(op.K, kchunk);
  Umma3Args a{};
  a.M = (int)op.M;
  a.N = (int)op.N;
  a.K = (int)op.K;
  a.BN = BN;
  a.kchunk = kchunk;
  a.stages = stages;
  a.ntiles = ntiles;
  a.status = op.status;
  a.sub_pos = op.sub_pos;
  a.sub_min = op.sub_min;
  if (op.sub_pos && (splits != 1 || !op.out || !op.out_colmajor)) return RLU_EINVAL;
  if (splits == 1 && op.out) {
    a.out = op.out;
    a.ldo = op.ldo;
    a.out_colmajor = op.out_colmajor;
  } else {
    if (!op.partial) return RLU_ENOMEM;
    // partial slices in the output's layout: for a column-major output the epilogue's
    // thread-per-row stores are then coalesced (row-major slices scatter every warp store
    // over 32 rows), and the reduction is an element-wise sum
    const bool cm = op.out != nullptr && op.out_colmajor;
    a.out = op.partial;
    a.ldo = cm ? op.M : op.N;
    a.out_colmajor = cm;
    a.split_stride = (size_t)op.M * op.N;
  }
  auto kern = k_umma3<MODE>;
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // x: (row tile, N tile) with the N tile fastest
  dim3 grid((unsigned)(ceil_div(op.M, U3_BM) * ntiles), (unsigned)splits);
  kern<<<grid, U3_THREADS, smem, s>>>(m0, m1, n0, n1, a);
  RLU_TRY(last_launch_status());
  if (a.out == op.partial && op.out) {
    if (a.out_colmajor)
      return splitk_reduce_cm_f32(op.partial, splits, op.M, op.N, op.out, op.ldo, s);
    return splitk_reduce_f32(op.partial, splits, op.M, op.N, op.out, op.ldo, !op.out_colmajor, s);
  }
  return RLU_OK;
}

// Fills one problem's record of the batched form (whole K, one N tile: N <= 256).
template <int MODE>
static int32_t make_job(const Umma3Op& op, U3Job* job, int* stage_bytes, bool ta) {
  if (op.M <= 0 || op.N <= 0 || op.N > 256 || op.K <= 0 || !op.out) return RLU_EINVAL;
  if (ta && op.N > 128) return RLU_EINVAL;  // two accumulators of up to 128 columns
  const int BN = (int)round_up(op.N, 16);
  const U3Layout lay = u3_persist_layout(MODE, BN, ta);
  if (MODE == U3_MODE_Y2) {
    RLU_TRY(map2d(&job->map[0], op.A0, op.M, op.K, op.lda, U3_BK, U3_BM, true));
    RLU_TRY(map2d(&job->map[2], op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    job->map[1] = job->map[0];
    job->map[3] = job->map[2];
  } else if (MODE == U3_MODE_C3) {
    RLU_TRY(map2d(&job->map[0], op.A0, op.K, op.M, op.lda, U3_BM, U3_BK, false));
    RLU_TRY(map2d(&job->map[2], op.B0, op.N, op.K, op.ldb, U3_BK, BN, true));
    RLU_TRY(map2d(&job->map[3], op.B1, op.N, op.K, op.ldb, U3_BK, BN, true));
    job->map[1] = job->map[0];
  } else {
    return RLU_EINVAL;
  }
  Umma3Args& a = job->a;
  a = Umma3Args{};
  a.M = (int)op.M;
  a.N = (int)op.N;
  a.K = (int)op.K;
  a.BN = BN;
  a.kchunk = (int)round_up(op.K, U3_BK);
  a.ntiles = 1;
  a.out = op.out;
  a.ldo = op.ldo;
  a.out_colmajor = op.out_colmajor;
  a.status = op.status;
  *stage_bytes = (int)lay.stage;
  return RLU_OK;
}

int32_t umma3_make_job(int mode, const Umma3Op& op, U3Job* job, int* stage_bytes, bool ta) {
  if (mode == U3_MODE_Y2) return make_job<U3_MODE_Y2>(op, job, stage_bytes, ta);
  if (mode == U3_MODE_C3) return make_job<U3_MODE_C3>(op, job, stage_bytes, ta);
  return RLU_EINVAL;
}

int32_t umma3_stages_for(int stage_bytes, int ctas_per_sm) {
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0, per_sm = 0, reserved = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  int budget = optin;
  if (ctas_per_sm > 1) budget = std::min(budget, per_sm / ctas_per_sm - reserved);
  int stages = (budget - 2048) / stage_bytes;
  return stages > U3_MAXST ? U3_MAXST : stages;
}

int32_t umma3_batched(int mode, const U3Job* jobs_dev, const int2* tiles_dev, int ntiles,
                      int stages, int max_stage_bytes, unsigned* counter, cudaStream_t s,
                      bool ta) {
  if (ntiles <= 0) return RLU_OK;
  if (stages < 2) return RLU_EINVAL;
  size_t smem = 2048 + (size_t)stages * max_stage_bytes;
  if (ta) {  // 512 TMEM columns per CTA: ask for more than half the SM's shared memory
    int dev = 0, per_sm = 0, reserved = 0;
    RLU_CUDA_TRY(cudaGetDevice(&dev));
    RLU_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    RLU_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    smem = std::max(smem, (size_t)(per_sm / 2 - reserved + 1024));
  }
  // persistent: as many CTAs as stay resident (one or two per SM), each walking the list
  auto go = [&](auto kern) -> int32_t {
    RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, U3_THREADS, smem));
    if (per_sm < 1) return RLU_EUNSUPPORTED;
    const int grid = std::min(ntiles, per_sm * sm_count());
    RLU_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    kern<<<(unsigned)grid, U3_THREADS, smem, s>>>(jobs_dev, tiles_dev, ntiles, stages,
                                                  (uint32_t)max_stage_bytes, counter);
    return last_launch_status();
  };
  if (mode == U3_MODE_Y2) return ta ? go(k_umma3_persist<U3_MODE_Y2, true>)
                                    : go(k_umma3_persist<U3_MODE_Y2, false>);
  if (mode == U3_MODE_C3) return ta ? go(k_umma3_persist<U3_MODE_C3, true>)
                                    : go(k_umma3_persist<U3_MODE_C3, false>);
  return RLU_EINVAL;
}

// U^T's TF32 parts for the trailing update: bt_hi / bt_lo [c - c_begin][s] (row stride 96)
// from u12[s][c]; rows s >= w are zero.
__global__ void k_trail_bsplit(const float* __restrict__ u12, int64_t ldu, int c_begin, int nc,
                               int w, float* __restrict__ bhi, float* __restrict__ blo) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * 96) return;
  const int c = e / 96, t = e % 96;
  const float x = t < w ? u12[(int64_t)t * ldu + c_begin + c] : 0.f;
  float h, l;
  u3::split_tf32(x, h, l);
  bhi[e] = h;
  blo[e] = l;
}

int32_t umma3_trail(float* X, int64_t ldx, int R, int c_begin, int c_end, int p0, int w,
                    const int32_t* posg, const float* u12, int64_t ldu, float* bt,
                    int32_t* status, cudaStream_t s) {
  const int nc = c_end - c_begin;
  if (nc <= 0) return RLU_OK;
  if (w < 1 || w > 96 || R < 1 || !bt || (ldx & 3) != 0 || ((uintptr_t)X & 15) != 0)
    return RLU_EUNSUPPORTED;
  float* bhi = bt;
  float* blo = bt + (size_t)96 * nc;
  k_trail_bsplit<<<(unsigned)ceil_div((int64_t)nc * 96, 256), 256, 0, s>>>(u12, ldu, c_begin, nc,
                                                                         w, bhi, blo);
  RLU_TRY(last_launch_status());
  Umma3Op op{};
  op.A0 = X + (int64_t)p0 * ldx;  // the multipliers: K = w columns of R contiguous rows
  op.lda = ldx;
  op.B0 = bhi;
  op.B1 = blo;
  op.ldb = 96;
  op.M = R;
  op.N = nc;
  op.K = w;
  op.out = X + (int64_t)c_begin * ldx;
  op.ldo = ldx;
  op.out_colmajor = true;
  op.splits = 1;
  op.status = status;
  op.sub_pos = posg;
  op.sub_min = p0 + w;
  return launch_u3<U3_MODE_C3>(op, s);
}

int32_t umma3_gemm(int mode, const Umma3Op& op, cudaStream_t s) {
  if (mode == U3_MODE_Y2) return launch_u3<U3_MODE_Y2>(op, s);
  if (mode == U3_MODE_C3) return launch_u3<U3_MODE_C3>(op, s);
  if (mode == U3_MODE_G3) return launch_u3<U3_MODE_G3>(op, s);
  if (mode == U3_MODE_Y3) return launch_u3<U3_MODE_Y3>(op, s);
  return RLU_EINVAL;
}

int umma3_splits(int64_t M, int64_t K, int64_t N) {
  const int64_t tiles = ceil_div(M, U3_BM) * ceil_div(N, 256);
  int64_t s = (int64_t)sm_count() / (tiles > 0 ? tiles : 1);
  const int64_t kmax = K / 256 > 1 ? K / 256 : 1;
  return (int)(s < 1 ? 1 : (s > kmax ? kmax : s));
}

}  // namespace rlu
