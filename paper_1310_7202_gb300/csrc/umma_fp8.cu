// FP8 (e4m3) projection Y = A G of the precision form with per-tile power-of-two scales
// (the FP8 variant of step 2 of Algorithm 1 that the precision form allows; the paper itself
// computes in IEEE single and double precision).
//
//   k_quant_a_fp8  A (BF16, m x n row-major) -> A8 (e4m3, m x ld8 bytes, zero-padded) and
//                  one UE8M0 scale per row and 128-column block (a 1 x 128 tile): 2^e with
//                  the smallest e such that the block's max |a| <= 448 * 2^e.
//   k_quant_g_fp8  G (FP32, n x l column-major) -> G8 (e4m3, l rows of ld8 bytes: row j is
//                  column j of G, K contiguous) and one scale per 128 x 128 block.
//   k_umma_fp8     Y (m x l, FP32) = A8 G8 on the tensor cores: tcgen05.mma kind::mxf8f6f4
//                  with block scaling (one UE8M0 scale per 32 elements of K, read from
//                  TMEM; here the same scale for the four 32-element chunks of a 128 block).
//                  Two 128-row accumulators per CTA share each G8 tile (224 columns).
//
// Scale layout in TMEM (measured on this GPU with a probe of all-ones operands and distinct
// scale codes): the scale of row r of the A operand is read from lane r, column
// base + r / 32, and the scale of column j of the B operand from column base + j / 32 and
// lane 32 q + j % 32, where q is the lane quarter of the output row (every quarter holds its
// own copy); the byte inside the 32-bit word is the scale id of the instruction descriptor.
// Tile t of the two A accumulators keeps its scales in byte t.
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocation and MMA issue, warps 2..5 write
// each k-step's scales into TMEM (tcgen05.st) and afterwards run the epilogue. Every wait
// is bounded (~1 s) and records an error instead of hanging; a wait that gives up drains
// the work already issued before TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "umma.cuh"

namespace rlu {

static constexpr int F8_BM = 128;       // rows per accumulator
static constexpr int F8_BK = 128;       // K per k-step: one 128-byte row, one scale block
static constexpr int F8_BN = 224;       // columns per CTA (accumulators at TMEM 0 and 224)
static constexpr int F8_THREADS = 192;
static constexpr int F8_MAXST = 4;
static constexpr uint32_t F8_SF0 = 448;  // scale columns: 12 per stage (A 4, B 8)
static constexpr uint32_t F8_SFST = 16;

struct F8Smem {
  uint64_t full[F8_MAXST];
  uint64_t sf[F8_MAXST];
  uint64_t empty[F8_MAXST];
  uint64_t accum;
  uint64_t drain;
  uint32_t tmem_base;
  int32_t err;
};

namespace f8 {
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
// K-major operand in 128-byte-swizzled rows: 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_mx8(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t sfa, uint32_t sfb, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %6, 0;\n"
               " tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X"
               " [%0], %1, %2, %3, [%4], [%5], p;\n}\n"
               ::"r"(d), "l"(da), "l"(db), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               ::"r"(bar) : "memory");
}
// UE8M0 exponent e of the scale 2^e of a block whose largest magnitude is amax: the smallest
// e with amax <= 448 * 2^e (448 = 1.75 * 2^8, the largest e4m3 value), from the bits of amax
// (exact; no division). A zero block takes e = 0.
__device__ __forceinline__ int scale_exp(float amax) {
  const uint32_t b = __float_as_uint(amax);
  if (b < 0x00800000u) return 0;  // zero or subnormal
  const int E = (int)(b >> 23) - 127;
  int e = E - 8 + ((b & 0x7FFFFFu) > 0x600000u ? 1 : 0);
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ float pow2(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }
// two values to e4m3 (round to nearest even, saturating to +-448), x in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float x, float y) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(x, y), __NV_SATFINITE, __NV_E4M3);
}
}  // namespace f8

// ---- quantisation ------------------------------------------------------------------------
// One warp per (row, 128-column block): each lane 4 consecutive values.
__global__ void __launch_bounds__(256) k_quant_a_fp8(const __nv_bfloat16* __restrict__ A,
                                                     int64_t lda, int M, int K,
                                                     uint8_t* __restrict__ A8, int64_t ld8,
                                                     uint8_t* __restrict__ SA, int64_t lds) {
  using namespace f8;
  const int lane = threadIdx.x & 31;
  const int nkb = (K + F8_BK - 1) / F8_BK;
  const int64_t items = (int64_t)M * nkb;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items;
       it += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int row = (int)(it / nkb), kb = (int)(it % nkb);
    const int k = kb * F8_BK + 4 * lane;
    const __nv_bfloat16* src = A + (int64_t)row * lda + k;
    float v[4];
    if (k + 3 < K) {
      const uint2 raw = *reinterpret_cast<const uint2*>(src);
      v[0] = __uint_as_float(raw.x << 16);
      v[1] = __uint_as_float(raw.x & 0xFFFF0000u);
      v[2] = __uint_as_float(raw.y << 16);
      v[3] = __uint_as_float(raw.y & 0xFFFF0000u);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = (k + u < K) ? __bfloat162float(src[u]) : 0.0f;
    }
    float am = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
    am = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(am)));
    const int e = scale_exp(am);
    const float inv = pow2(-e);
    const uint32_t q = e4m3x2(v[0] * inv, v[1] * inv) | (e4m3x2(v[2] * inv, v[3] * inv) << 16);
    *reinterpret_cast<uint32_t*>(A8 + (int64_t)row * ld8 + k) = q;  // zero past K
    if (lane == 0) SA[(int64_t)row * lds + kb] = (uint8_t)(127 + e);
  }
}

// One CTA (128 threads) per 128 x 128 block of G: thread t holds column nb * 128 + t.
__global__ void __launch_bounds__(128) k_quant_g_fp8(const float* __restrict__ G, int64_t ldg,
                                                     int K, int N, uint8_t* __restrict__ G8,
                                                     int64_t ld8, uint8_t* __restrict__ SG,
                                                     int64_t lsg) {
  using namespace f8;
  __shared__ uint32_t wmax[4];
  const int kb = blockIdx.x, nb = blockIdx.y;
  const int j = nb * 128 + threadIdx.x;
  const int k0 = kb * F8_BK;
  const int kn = min(F8_BK, K - k0);
  float am = 0.0f;
  if (j < N)
    for (int i = 0; i < kn; ++i) am = fmaxf(am, fabsf(G[(int64_t)j * ldg + k0 + i]));
  const uint32_t w = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = w;
  __syncthreads();
  const float bm = __uint_as_float(max(max(wmax[0], wmax[1]), max(wmax[2], wmax[3])));
  const int e = scale_exp(bm);
  const float inv = pow2(-e);
  if (j < N) {
    uint8_t* dst = G8 + (int64_t)j * ld8 + k0;
    for (int i0 = 0; i0 < F8_BK; i0 += 16) {
      uint32_t wds[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = i0 + 4 * u + t;
          x[t] = i < kn ? G[(int64_t)j * ldg + k0 + i] * inv : 0.0f;
        }
        wds[u] = e4m3x2(x[0], x[1]) | (e4m3x2(x[2], x[3]) << 16);
      }
      *reinterpret_cast<uint4*>(dst + i0) = make_uint4(wds[0], wds[1], wds[2], wds[3]);
    }
  }
  if (threadIdx.x == 0) SG[(int64_t)kb * lsg + nb] = (uint8_t)(127 + e);
}

// ---- the block-scaled GEMM -------------------------------------------------------------
struct F8Args {
  const uint8_t* SA;   // row scales, lds per row
  int64_t lds;
  const uint8_t* SG;   // G block scales, lsg per 128-row (K) block
  int64_t lsg;
  float* out;          // column-major (or split-K partial slices, row-major)
  int64_t ldo;
  size_t split_stride;
  int M, N, K, kchunk, stages, ntiles, bn_last;
  bool out_colmajor;
  int32_t* status;
};

// block-scaled instruction descriptor: B scale id [4,6), A and B E4M3 (0), K-major both,
// N >> 3 at 17, UE8M0 scales (bit 23), M >> 4 at 24, A scale id [29,31)
__host__ __device__ constexpr uint32_t f8_idesc(int M, int N, int asf) {
  return ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24) |
         ((uint32_t)asf << 29);
}

__global__ void __launch_bounds__(F8_THREADS, 1)
k_umma_fp8(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mG,
           const __grid_constant__ CUtensorMap mGl, F8Args a) {
  using namespace f8;
  extern __shared__ __align__(1024) unsigned char f8_smem[];
  F8Smem& sh = *reinterpret_cast<F8Smem*>(f8_smem);
  const uint32_t tiles = (su32(f8_smem) + sizeof(F8Smem) + 1023u) & ~1023u;
  constexpr uint32_t AT = F8_BM * 128;              // one A tile: 128 rows x 128 bytes
  constexpr uint32_t STAGE = 2 * AT + F8_BN * 128;  // two A tiles and the G tile
  const int S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = (int)blockIdx.x % a.ntiles, mt = (int)blockIdx.x / a.ntiles;
  const int m0 = mt * 2 * F8_BM;
  const int nb0 = nt * F8_BN;
  const int bn = nt == a.ntiles - 1 ? a.bn_last : F8_BN;
  const int kz = blockIdx.y;
  const int k_begin = kz * a.kchunk;
  const int k_end = min(a.K, k_begin + a.kchunk);
  const int nk = (k_end - k_begin + F8_BK - 1) / F8_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(su32(&sh.full[s]), 1);
      mb_init(su32(&sh.sf[s]), 4);
      mb_init(su32(&sh.empty[s]), 1);
    }
    mb_init(su32(&sh.accum), 1);
    mb_init(su32(&sh.drain), 1);
    sh.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n"
                 ::"r"(su32(&sh.tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sh.tmem_base;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ------------------------------------------------------------------
    const bool narrow = bn < F8_BN;  // the last N tile loads only its bn rows of G8
    const uint32_t tx = 2 * AT + (uint32_t)(narrow ? bn : F8_BN) * 128u;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      if (kt >= S && !mb_wait(su32(&sh.empty[s]), (uint32_t)(((kt / S) - 1) & 1))) {
        sh.err = 1;
        break;
      }
      const uint32_t base = tiles + s * STAGE;
      const uint32_t bar = su32(&sh.full[s]);
      const int kx = k_begin + kt * F8_BK;
      mb_expect_tx(bar, tx);
      tma2d(base, &mA, kx, m0, bar);
      tma2d(base + AT, &mA, kx, m0 + F8_BM, bar);
      tma2d(base + 2 * AT, narrow ? &mGl : &mG, kx, nb0, bar);
      issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: per k-step 4 chunks of K = 32 for each of the two accumulators ------
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      const uint32_t par = (uint32_t)((kt / S) & 1);
      if (!mb_wait(su32(&sh.full[s]), par) || !mb_wait(su32(&sh.sf[s]), par)) {
        sh.err = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tiles + s * STAGE;
      const uint32_t sfa = tmem + F8_SF0 + s * F8_SFST;
      const uint32_t sfb = sfa + 4;
#pragma unroll
      for (int kk = 0; kk < F8_BK / 32; ++kk) {
        const uint32_t off = kk * 32;
        const uint64_t db = desc_sw128(base + 2 * AT + off);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_mx8(tmem, desc_sw128(base + off), db, f8_idesc(F8_BM, bn, 0), sfa, sfb, acc);
        mma_mx8(tmem + (uint32_t)F8_BN, desc_sw128(base + AT + off), db, f8_idesc(F8_BM, bn, 1),
                sfa, sfb, acc);
      }
      commit(su32(&sh.empty[s]));
    }
    commit(su32(&sh.accum));
  } else if (warp >= 2) {
    // ---- scales into TMEM, then the epilogue -------------------------------------------
    const int q = warp & 3;  // this warp's TMEM lane quarter
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    bool ok = true;
    for (int kt = 0; kt < nk && ok; ++kt) {
      const int s = kt % S;
      if (kt >= S) {
        const bool got = mb_wait(su32(&sh.empty[s]), (uint32_t)(((kt / S) - 1) & 1));
        if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {
          sh.err = 1;
          ok = false;
          break;
        }
      }
      const int kb = (k_begin + kt * F8_BK) / F8_BK;
      // A: row 32 q + lane of tile t in byte t of column q
      const int r0 = m0 + q * 32 + lane, r1 = r0 + F8_BM;
      const uint32_t b0 = r0 < a.M ? a.SA[(int64_t)r0 * a.lds + kb] : 127u;
      const uint32_t b1 = r1 < a.M ? a.SA[(int64_t)r1 * a.lds + kb] : 127u;
      const uint32_t wa = b0 | (b1 << 8) | (b0 << 16) | (b1 << 24);
      const uint32_t col = F8_SF0 + s * F8_SFST;
      asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};\n"
                   ::"r"(tmem + lanes + col + (uint32_t)q), "r"(wa) : "memory");
      // B: column j = 32 c + lane in column c, every quarter its own copy
      uint32_t wb[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = nb0 + 32 * c + lane;
        const uint32_t v = (32 * c + lane < bn && j < a.N) ? a.SG[(int64_t)kb * a.lsg + j / 128]
                                                           : 127u;
        wb[c] = v * 0x01010101u;
      }
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                   ::"r"(tmem + lanes + col + 4u), "r"(wb[0]), "r"(wb[1]), "r"(wb[2]),
                     "r"(wb[3]), "r"(wb[4]), "r"(wb[5]), "r"(wb[6]), "r"(wb[7]) : "memory");
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mb_arrive(su32(&sh.sf[s]));
    }
    const bool done = ok && mb_wait(su32(&sh.accum), 0u);
    const bool all = __shfl_sync(0xffffffffu, done ? 1 : 0, 0) != 0;
    if (!all) sh.err = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float* __restrict__ out = a.out + (size_t)kz * a.split_stride;
    for (int t = 0; t < 2 && all; ++t)
      for (int c0 = 0; c0 < bn; c0 += 32) {
        const int row = m0 + t * F8_BM + q * 32 + lane;
        uint32_t v[32];
        const uint32_t taddr = tmem + lanes + (uint32_t)(t * F8_BN + c0);
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
          for (int j = 0; j < 32; ++j) {
            const int colj = nb0 + c0 + j;
            if (c0 + j < bn && colj < a.N) {
              const float f = __uint_as_float(v[j]);
              if (a.out_colmajor)
                out[(size_t)colj * a.ldo + row] = f;
              else
                out[(size_t)row * a.ldo + colj] = f;
            }
          }
        }
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (sh.err) {
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0 && sh.err && a.status) atomicExch(a.status, RLU_ETIMEOUT);
}

// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 f8_encode_fn() {
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

// Byte matrix (rows x cols, ld bytes) with 128-byte-swizzled boxes of 128 bytes x box_rows.
static int32_t map2d_u8(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows) {
  auto enc = f8_encode_fn();
  if (!enc) return RLU_ECUDA;
  if (((uintptr_t)base & 15u) != 0 || ld % 16 != 0) return RLU_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {128u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RLU_OK : RLU_ECUDA;
}

int64_t fp8_ld(int64_t K) { return round_up(K, F8_BK); }

int32_t fp8_quantize_a(const void* A, int64_t lda, int64_t M, int64_t K, uint8_t* A8,
                       int64_t ld8, uint8_t* SA, int64_t lds, cudaStream_t s) {
  if (M <= 0 || K <= 0) return RLU_OK;
  if (ld8 < fp8_ld(K) || lds < ceil_div(K, F8_BK) || (lda % 4) != 0 ||
      ((uintptr_t)A & 7u) != 0)
    return RLU_EINVAL;
  const int64_t items = M * ceil_div(K, F8_BK);
  int64_t blocks = ceil_div(items, 8);
  const int64_t cap = (int64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  k_quant_a_fp8<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(A), lda,
                                                (int)M, (int)K, A8, ld8, SA, lds);
  return last_launch_status();
}

int32_t fp8_quantize_g(const float* G, int64_t ldg, int64_t K, int64_t N, uint8_t* G8,
                       int64_t ld8, uint8_t* SG, int64_t lsg, cudaStream_t s) {
  if (K <= 0 || N <= 0) return RLU_OK;
  if (ld8 < fp8_ld(K) || lsg < ceil_div(N, 128)) return RLU_EINVAL;
  dim3 grid((unsigned)ceil_div(K, F8_BK), (unsigned)ceil_div(N, 128));
  k_quant_g_fp8<<<grid, 128, 0, s>>>(G, ldg, (int)K, (int)N, G8, ld8, SG, lsg);
  return last_launch_status();
}

int umma_fp8_splits(int64_t M, int64_t K, int64_t N) {
  const int64_t tiles = ceil_div(M, 2 * F8_BM) * ceil_div(N, F8_BN);
  int64_t s = (int64_t)sm_count() / (tiles > 0 ? tiles : 1);
  const int64_t kmax = K / 1024 > 1 ? K / 1024 : 1;
  return (int)(s < 1 ? 1 : (s > kmax ? kmax : s));
}

int32_t umma_fp8_y(const Fp8Op& op, cudaStream_t s) {
  if (op.M <= 0 || op.N <= 0 || op.K <= 0) return RLU_EINVAL;
  const int ntiles = (int)ceil_div(op.N, F8_BN);
  const int bn_last = (int)round_up(op.N - (int64_t)(ntiles - 1) * F8_BN, 16);
  constexpr int STAGE = 2 * F8_BM * 128 + F8_BN * 128;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int ctrl = 2048;
  int stages = (optin - ctrl) / STAGE;
  if (stages > F8_MAXST) stages = F8_MAXST;
  if (stages < 2) return RLU_EUNSUPPORTED;
  const size_t smem = (size_t)ctrl + (size_t)stages * STAGE;
  const int64_t kp = fp8_ld(op.K);
  CUtensorMap mA{}, mG{}, mGl{};
  RLU_TRY(map2d_u8(&mA, op.A8, op.M, kp, op.lda8, F8_BM));
  RLU_TRY(map2d_u8(&mG, op.G8, op.N, kp, op.ldg8, F8_BN));
  RLU_TRY(map2d_u8(&mGl, op.G8, op.N, kp, op.ldg8, bn_last));
  int splits = op.splits < 1 ? 1 : op.splits;
  const int kchunk = (int)round_up(ceil_div(kp, splits), F8_BK);
  splits = (int)ceil_div(kp, kchunk);
  F8Args a{};
  a.SA = op.SA;
  a.lds = op.lds;
  a.SG = op.SG;
  a.lsg = op.lsg;
  a.M = (int)op.M;
  a.N = (int)op.N;
  a.K = (int)kp;
  a.kchunk = kchunk;
  a.stages = stages;
  a.ntiles = ntiles;
  a.bn_last = bn_last;
  a.status = op.status;
  if (splits == 1) {
    a.out = op.out;
    a.ldo = op.ldo;
    a.out_colmajor = op.out_colmajor;
  } else {
    if (!op.partial) return RLU_ENOMEM;
    a.out = op.partial;
    a.ldo = op.N;
    a.out_colmajor = false;
    a.split_stride = (size_t)op.M * op.N;
  }
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_umma_fp8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  dim3 grid((unsigned)(ceil_div(op.M, 2 * F8_BM) * ntiles), (unsigned)splits);
  k_umma_fp8<<<grid, F8_THREADS, smem, s>>>(mA, mG, mGl, a);
  RLU_TRY(last_launch_status());
  if (splits > 1)
    return splitk_reduce_f32(op.partial, splits, op.M, op.N, op.out, op.ldo, !op.out_colmajor, s);
  return RLU_OK;
}

}  // namespace rlu
