// BF16 tensor-core GEMMs on tcgen05/TMEM (sm_103a) for the precision form of Algorithm 1
// (A stored in BF16): D (M x N, FP32 accumulation in TMEM) = A (M x K) * B (N x K)^T with
// kind::f16 MMAs on BF16 operands.
//
//   UB_MODE_Y   Y = A G (step 2): A row-major (K = n contiguous), G column-major (K
//               contiguous); both arrive by TMA in 128-byte-swizzled K-major tiles. One
//               product: the range finder only needs Y's column space, so BF16 A and G with
//               FP32 accumulation suffice.
//   UB_MODE_C3  C = L~^T A (step 5), k x n: the A operand is L~ in three BF16 parts
//               hi + mid + lo (8 significant bits each, FP32 accurate), K-major (L~ is
//               column-major, so a row of L~^T is contiguous), 64-byte-swizzled boxes of
//               32 (m) x 128 (k); the B operand is A itself: A is stored m x n row-major, so
//               the operand is N-major, 128-byte-swizzled boxes of 64 (n) x 32 (m) that the
//               MMA reads MN-major (A is exact in BF16: nothing to split or transpose). The
//               three products L_hi^T A + L_mid^T A + L_lo^T A accumulate in FP32. With the
//               three parts as the 128-row operand and 256 columns of A as the other, one
//               k-step moves 40 KB into shared memory for six 128 x 256 x 16 MMAs.
//
//   UB_MODE_Y3  Y = A Z (the power iterations of Section 5): A as in UB_MODE_Y, Z in three
//               BF16 parts (FP32 accurate; Z is not a random matrix whose rounding is
//               harmless), three products A Z_hi + A Z_mid + A Z_lo; N tiles of 128.
//
// N tiles: BN columns each, the last one only as wide as the columns left (rounded up to
// 16), so that no MMA work is spent on padding.
//
// Warp roles as in the TF32 kernels: warp 0 TMA producer over a ring of slots, warp 1 TMEM
// allocation and MMA issue, warps 2..5 epilogue. Every wait is bounded (~1 s) and records an
// error instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "umma.cuh"

namespace rlu {

static constexpr int UB_BM = 128;
static constexpr int UB_BK = 64;   // Y: BF16 elements of K per k-step (one 128-byte row)
static constexpr int UB_BKC = 32;  // C: 32 elements (one 64-byte row of the L~ parts)
static constexpr int UB_THREADS = 192;
static constexpr int UB_MAXST = 6;

struct UbSmem {
  uint64_t full[UB_MAXST];
  uint64_t empty[UB_MAXST];
  uint64_t accum;
  uint64_t drain;  // final commit of the MMA issuer when a wait gave up
  uint32_t tmem_base;
  int32_t err;
};

namespace ub {
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
// K-major operand in 64-byte-swizzled rows: 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(512u >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// MN-major operand in 128-byte-swizzled boxes of 64 (MN) x rows (K): a row of a box holds 64
// consecutive MN elements of one K index; groups of 8 K rows lie 1024 bytes apart (stride
// offset) and the next 64 MN elements start one box further (leading offset, box bytes).
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr, uint32_t box_bytes) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(box_bytes >> 4) << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               ::"r"(bar) : "memory");
}
}  // namespace ub

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), A K-major, B MN-major if b_mn (bit 16), N >> 3 at bit 17, M >> 4
// at bit 24.
__host__ __device__ constexpr uint32_t ub_idesc(int M, int N, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One ring slot. Y: a0, a1 = two A tiles (128 x 64 each, K-major), b0 = G tile (BN x 64).
// Y3: a0 = A tile, b0..b2 = the Z parts (BN x 64 each).
// C3: a0..a2 = the L~ parts (128 x 32 each, K-major), b0 = four 64 (n) x 32 (m) boxes of A.
struct UbLayout {
  uint32_t a0, a1, a2, b0, stage, tx;
};
__host__ __device__ inline UbLayout ub_layout(int mode, int BN) {
  UbLayout L{};
  if (mode == UB_MODE_Y) {  // two 128-row tiles of A (a0, a1) share the G tile
    const uint32_t at = UB_BM * 128, bt = (uint32_t)BN * 128;
    L.a0 = 0; L.a1 = at; L.a2 = 0; L.b0 = 2 * at; L.stage = 2 * at + bt;
  } else if (mode == UB_MODE_Y3) {
    const uint32_t at = UB_BM * 128, bt = (uint32_t)BN * 128;
    L.a0 = 0; L.b0 = at; L.a1 = at + bt; L.a2 = at + 2 * bt; L.stage = at + 3 * bt;
  } else {
    const uint32_t pt = UB_BM * 64;  // one part: 128 rows of 64 bytes
    L.a0 = 0; L.a1 = pt; L.a2 = 2 * pt; L.b0 = 3 * pt;
    L.stage = 3 * pt + (uint32_t)BN * UB_BKC * 2;
  }
  L.tx = L.stage;
  L.stage = (L.stage + 1023u) & ~1023u;
  return L;
}

template <int MODE>
__global__ void __launch_bounds__(UB_THREADS, 1)
k_ummab(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB0,
        const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
        Umma3Args a) {
  using namespace ub;
  extern __shared__ __align__(1024) unsigned char ub_smem[];
  UbSmem& sh = *reinterpret_cast<UbSmem*>(ub_smem);
  const uint32_t tiles = (su32(ub_smem) + sizeof(UbSmem) + 1023u) & ~1023u;
  const UbLayout lay = ub_layout(MODE, a.BN);
  const int S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // The CTAs that read the same tiles of BF16 A run together, so that A is fetched from
  // DRAM once and the other CTAs hit L2. Y: grid x = (row tile, N tile), N tile fastest.
  // C3: A is the N operand, grid x = (N tile, row tile), row tile fastest.
  constexpr bool YM = MODE == UB_MODE_Y || MODE == UB_MODE_Y3;  // A is the M operand
  constexpr int BK = YM ? UB_BK : UB_BKC;
  // Y: two 128-row accumulators per CTA (TMEM columns 0 and 256), one G tile for both, so
  // that a k-step moves 64 KB for eight MMAs instead of 48 KB for four
  constexpr int MT = MODE == UB_MODE_Y ? 2 : 1;
  constexpr uint32_t TCOLS = MT == 2 ? 512u : 256u;
  const int mtiles = (a.M + UB_BM * MT - 1) / (UB_BM * MT);
  const int mt = YM ? (int)blockIdx.x / a.ntiles : (int)blockIdx.x % mtiles;
  const int nt = YM ? (int)blockIdx.x % a.ntiles : (int)blockIdx.x / mtiles;
  const int m0 = mt * UB_BM * MT;
  const int kz = blockIdx.y;
  const int nb0 = nt * a.BN;
  const int bn = nt == a.ntiles - 1 ? a.bn_last : a.BN;  // this tile's MMA width
  const int k_begin = kz * a.kchunk;
  const int k_end = min(a.K, k_begin + a.kchunk);
  const int nk = (k_end - k_begin + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(su32(&sh.full[s]), 1);
      mb_init(su32(&sh.empty[s]), 1);
    }
    mb_init(su32(&sh.accum), 1);
    mb_init(su32(&sh.drain), 1);
    sh.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(su32(&sh.tmem_base)), "n"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sh.tmem_base;
  int issued = 0;  // k-steps whose loads the producer started

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ------------------------------------------------------------------
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      if (kt >= S && !mb_wait(su32(&sh.empty[s]), (uint32_t)(((kt / S) - 1) & 1))) {
        sh.err = 1;
        break;
      }
      const uint32_t base = tiles + s * lay.stage;
      const uint32_t bar = su32(&sh.full[s]);
      const int kx = k_begin + kt * BK;
      if (MODE == UB_MODE_Y) {
        // the last N tile loads only its bn rows of G (map B1 has a box of bn_last rows)
        const bool narrow = bn < a.BN;
        mb_expect_tx(bar, narrow ? lay.tx - (uint32_t)(a.BN - bn) * 128u : lay.tx);
        tma2d(base + lay.a0, &mA, kx, m0, bar);
        tma2d(base + lay.a1, &mA, kx, m0 + UB_BM, bar);
        tma2d(base + lay.b0, narrow ? &mB1 : &mB0, kx, nb0, bar);
      } else if (MODE == UB_MODE_Y3) {
        mb_expect_tx(bar, lay.tx);
        tma2d(base + lay.a0, &mA, kx, m0, bar);
        tma2d(base + lay.b0, &mB0, kx, nb0, bar);  // Z parts: x = K, y = N
        tma2d(base + lay.a1, &mB1, kx, nb0, bar);
        tma2d(base + lay.a2, &mB2, kx, nb0, bar);
      } else {
        mb_expect_tx(bar, lay.tx);
        tma2d(base + lay.a0, &mB0, kx, m0, bar);  // L~ parts: x = m (32 wide), y = k (128)
        tma2d(base + lay.a1, &mB1, kx, m0, bar);
        tma2d(base + lay.a2, &mB2, kx, m0, bar);
        for (int j = 0; j < a.BN / 64; ++j)        // A: x = n (64 wide), y = m (32)
          tma2d(base + lay.b0 + (uint32_t)j * 4096u, &mA, nb0 + 64 * j, kx, bar);
      }
      issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: 4 MMAs of K = 16 per 64-wide slot ---------------------------------
    const uint32_t idesc = ub_idesc(UB_BM, bn, MODE == UB_MODE_C3);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % S;
      const uint32_t par = (uint32_t)((kt / S) & 1);
      if (!mb_wait(su32(&sh.full[s]), par)) {
        sh.err = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tiles + s * lay.stage;
      if (MODE == UB_MODE_Y) {  // 4 x 2 MMAs of K = 16 along the 128-byte rows
#pragma unroll
        for (int kk = 0; kk < UB_BK / 16; ++kk) {
          const uint32_t off = kk * 32;
          const uint64_t db = desc_sw128(base + lay.b0 + off);
          const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
          mma_bf16(tmem, desc_sw128(base + lay.a0 + off), db, idesc, acc);
          mma_bf16(tmem + 256u, desc_sw128(base + lay.a1 + off), db, idesc, acc);
        }
      } else if (MODE == UB_MODE_Y3) {  // 4 x 3 MMAs of K = 16, the three parts of Z
#pragma unroll
        for (int kk = 0; kk < UB_BK / 16; ++kk) {
          const uint32_t off = kk * 32;
          const uint64_t da = desc_sw128(base + lay.a0 + off);
          mma_bf16(tmem, da, desc_sw128(base + lay.b0 + off), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          mma_bf16(tmem, da, desc_sw128(base + lay.a1 + off), idesc, 1u);
          mma_bf16(tmem, da, desc_sw128(base + lay.a2 + off), idesc, 1u);
        }
      } else {  // 2 x 3 MMAs of K = 16: 32 bytes along the parts' rows, 16 rows of the A boxes
#pragma unroll
        for (int kk = 0; kk < UB_BKC / 16; ++kk) {
          const uint64_t db = desc_mn_sw128(base + lay.b0 + kk * 2048u, 4096u);
          const uint32_t off = kk * 32;
          mma_bf16(tmem, desc_sw64(base + lay.a0 + off), db, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          mma_bf16(tmem, desc_sw64(base + lay.a1 + off), db, idesc, 1u);
          mma_bf16(tmem, desc_sw64(base + lay.a2 + off), db, idesc, 1u);
        }
      }
      commit(su32(&sh.empty[s]));
    }
    commit(su32(&sh.accum));
  } else if (warp >= 2 && warp < 6) {
    // ---- epilogue ------------------------------------------------------------------------
    const bool ok = mb_wait(su32(&sh.accum), 0u);
    if (!ok) sh.err = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int quarter = warp & 3;
    float* __restrict__ out = a.out + (size_t)kz * a.split_stride;
    const bool vec_out = ((uintptr_t)out % 16 == 0) && a.ldo % 4 == 0;
    for (int t = 0; t < MT; ++t)
    for (int c0 = 0; c0 < bn; c0 += 32) {
      const int row = m0 + t * UB_BM + quarter * 32 + lane;
      uint32_t v[32];
      const uint32_t taddr =
          tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * 256 + c0);
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
      if (ok && row < a.M) {
        const int col0 = nb0 + c0;
        if (!a.out_colmajor && vec_out && col0 + 32 <= a.N && c0 + 32 <= bn) {
          float4* o4 = reinterpret_cast<float4*>(out + (size_t)row * a.ldo + col0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            o4[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = col0 + j;
            if (c0 + j < bn && col < a.N) {
              const float f = __uint_as_float(v[j]);
              if (a.out_colmajor)
                out[(size_t)col * a.ldo + row] = f;
              else
                out[(size_t)row * a.ldo + col] = f;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (sh.err) {
    // a wait gave up: let the work already issued finish (bounded) before TMEM is freed
    // and the CTA exits (the MMA issuer's final commit covers every MMA it issued; the
    // producer waits for the loads of the last S k-steps it started)
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
                 ::"r"(tmem), "n"(TCOLS) : "memory");
  }
  if (threadIdx.x == 0 && sh.err && a.status) atomicExch(a.status, RLU_ETIMEOUT);
}

// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 ub_encode_fn() {
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

// BF16 row-major (rows x cols, ld elements) tensor map with a box of box_x x box_y.
static int32_t map2d_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                          int64_t ld, int box_x, int box_y, CUtensorMapSwizzle swizzle) {
  auto enc = ub_encode_fn();
  if (!enc) return RLU_ECUDA;
  if (((uintptr_t)base & 15u) != 0 || (ld * 2) % 16 != 0) return RLU_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RLU_OK : RLU_ECUDA;
}

template <int MODE>
static int32_t launch_ub(const UmmaBf16Op& op, cudaStream_t s) {
  if (op.M <= 0 || op.N <= 0 || op.K <= 0) return RLU_EINVAL;
  // N tiles of up to 256 columns (C3: whole 64-column boxes of A)
  constexpr int BK = MODE == UB_MODE_C3 ? UB_BKC : UB_BK;
  const int bnmax = MODE == UB_MODE_Y3 ? 128 : 256;
  const int BN = op.N > bnmax ? bnmax : (int)round_up(op.N, MODE == UB_MODE_C3 ? 64 : 16);
  const int ntiles = (int)ceil_div(op.N, BN);
  const int bn_last = (int)round_up(op.N - (int64_t)(ntiles - 1) * BN, 16);
  const UbLayout lay = ub_layout(MODE, BN);
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int ctrl = 2048;
  int stages = (int)((optin - ctrl) / (int)lay.stage);
  if (stages > UB_MAXST) stages = UB_MAXST;
  if (stages < 2) return RLU_EUNSUPPORTED;
  const size_t smem = (size_t)ctrl + (size_t)stages * lay.stage;
  CUtensorMap mA{}, b0{}, b1{}, b2{};
  const auto SW128 = CU_TENSOR_MAP_SWIZZLE_128B, SW64 = CU_TENSOR_MAP_SWIZZLE_64B;
  if (MODE == UB_MODE_Y) {
    RLU_TRY(map2d_bf16(&mA, op.A, op.M, op.K, op.lda, UB_BK, UB_BM, SW128));
    RLU_TRY(map2d_bf16(&b0, op.B0, op.N, op.K, op.ldb, UB_BK, BN, SW128));
    RLU_TRY(map2d_bf16(&b1, op.B0, op.N, op.K, op.ldb, UB_BK, bn_last, SW128));
    b2 = b0;
  } else if (MODE == UB_MODE_Y3) {
    RLU_TRY(map2d_bf16(&mA, op.A, op.M, op.K, op.lda, UB_BK, UB_BM, SW128));
    RLU_TRY(map2d_bf16(&b0, op.B0, op.N, op.K, op.ldb, UB_BK, BN, SW128));
    RLU_TRY(map2d_bf16(&b1, op.B1, op.N, op.K, op.ldb, UB_BK, BN, SW128));
    RLU_TRY(map2d_bf16(&b2, op.B2, op.N, op.K, op.ldb, UB_BK, BN, SW128));
  } else {
    // A stored row-major K x N (rows = K index, N contiguous): boxes 64 (N) x 32 (K);
    // the L~ parts M x K (K contiguous): boxes 32 (K) x 128 (M)
    RLU_TRY(map2d_bf16(&mA, op.A, op.K, op.N, op.lda, 64, UB_BKC, SW128));
    RLU_TRY(map2d_bf16(&b0, op.B0, op.M, op.K, op.ldb, UB_BKC, UB_BM, SW64));
    RLU_TRY(map2d_bf16(&b1, op.B1, op.M, op.K, op.ldb, UB_BKC, UB_BM, SW64));
    RLU_TRY(map2d_bf16(&b2, op.B2, op.M, op.K, op.ldb, UB_BKC, UB_BM, SW64));
  }
  int splits = op.splits < 1 ? 1 : op.splits;
  const int kchunk = (int)round_up(ceil_div(op.K, splits), BK);
  splits = (int)ceil_div(op.K, kchunk);
  Umma3Args a{};
  a.M = (int)op.M;
  a.N = (int)op.N;
  a.K = (int)op.K;
  a.BN = BN;
  a.kchunk = kchunk;
  a.stages = stages;
  a.ntiles = ntiles;
  a.bn_last = bn_last;
  a.status = op.status;
  if (splits == 1 && op.out) {
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
  auto kern = k_ummab<MODE>;
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int rows_per_cta = MODE == UB_MODE_Y ? 2 * UB_BM : UB_BM;
  dim3 grid((unsigned)(ceil_div(op.M, rows_per_cta) * ntiles), (unsigned)splits);
  kern<<<grid, UB_THREADS, smem, s>>>(mA, b0, b1, b2, a);
  RLU_TRY(last_launch_status());
  if (a.out == op.partial && op.out)
    return splitk_reduce_f32(op.partial, splits, op.M, op.N, op.out, op.ldo, !op.out_colmajor, s);
  return RLU_OK;
}

int32_t umma_bf16_gemm(int mode, const UmmaBf16Op& op, cudaStream_t s) {
  if (mode == UB_MODE_Y) return launch_ub<UB_MODE_Y>(op, s);
  if (mode == UB_MODE_C3) return launch_ub<UB_MODE_C3>(op, s);
  if (mode == UB_MODE_Y3) return launch_ub<UB_MODE_Y3>(op, s);
  return RLU_EINVAL;
}

int umma_bf16_splits(int64_t M, int64_t K, int64_t N, int bn) {
  const int64_t tiles = ceil_div(M, UB_BM) * ceil_div(N, bn);
  int64_t s = (int64_t)sm_count() / (tiles > 0 ? tiles : 1);
  const int64_t kmax = K / 512 > 1 ? K / 512 : 1;
  return (int)(s < 1 ? 1 : (s > kmax ? kmax : s));
}

}  // namespace rlu
