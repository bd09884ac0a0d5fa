// Tensor-core (tcgen05 / TMEM, sm_103a) GEMM fed by TMA: D (M x N) = A (M x K) * B (N x K)^T
// with both operands K-major FP32 in global memory and TF32 multiplies, FP32 accumulation.
// Used for step 2 of Algorithm 1 (Y = A G: A row-major is K-major, G column-major is K-major
// for N) in the mixed-precision path.
//
// One CTA computes a BM = 128 row block times all N <= 256 columns (one accumulator in
// TMEM) over a K range (split-K across blockIdx.y). Warp roles:
//   warp 0      TMA producer: a ring of STAGES shared-memory slots, 128-byte swizzled
//               32-float K slices of A (128 rows) and B (BN rows), full/empty mbarriers
//   warp 1      TMEM allocation and the MMA issuer (one thread): 4 tcgen05.mma (K = 8)
//               per slot, tcgen05.commit releases the slot, a final commit signals the
//               epilogue
//   warps 2..5  epilogue: tcgen05.ld 32 lanes x 32 columns per instruction, stores to D
//               (column-major) or to a row-major split-K partial slice
// Every mbarrier wait gives up after about a second (globaltimer) and records an error.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "umma.cuh"

namespace rlu {

static constexpr int UM_BM = 128;
static constexpr int UM_BK = 32;        // floats per 128-byte swizzle row
static constexpr int UM_STAGES = 4;
static constexpr int UM_THREADS = 192;

struct UmmaSmem {
  uint64_t full[UM_STAGES];
  uint64_t empty[UM_STAGES];
  uint64_t accum;
  uint32_t tmem_base;
  int32_t err;
};

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
__device__ __forceinline__ bool mb_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase completed, false after ~1 s.
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity) {
  if (mb_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mb_try(bar, parity))
    if (now_ns() - t0 > 1000000000ull) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B
// apart (stride byte offset), descriptor version 1 (bits 46-48), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)(16u >> 4) << 16;                   // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                            // version
  d |= (uint64_t)2 << 61;                            // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4)            // D format: F32
         | (2u << 7)          // A format: TF32
         | (2u << 10)         // B format: TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(UM_THREADS, 1)
k_umma_tf32(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            UmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char um_smem[];
  // 1024-byte aligned tiles after the control block
  const uint32_t raw = su32(um_smem);
  const uint32_t tiles = (raw + sizeof(UmmaSmem) + 1023u) & ~1023u;
  UmmaSmem& sh = *reinterpret_cast<UmmaSmem*>(um_smem);
  const uint32_t a_bytes = UM_BM * 128u;
  const uint32_t b_bytes = (uint32_t)a.BN * 128u;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * UM_BM;
  const int kz = blockIdx.y;
  const int k_begin = kz * a.kchunk;
  const int k_end = min(a.K, k_begin + a.kchunk);
  const int nk = (k_end - k_begin + UM_BK - 1) / UM_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < UM_STAGES; ++s) {
      mb_init(su32(&sh.full[s]), 1);
      mb_init(su32(&sh.empty[s]), 1);
    }
    mb_init(su32(&sh.accum), 1);
    sh.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {  // TMEM: 256 columns x 128 lanes of FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n"
                 ::"r"(su32(&sh.tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sh.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ------------------------------------------------------------------
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % UM_STAGES;
      if (kt >= UM_STAGES) {
        if (!mb_wait(su32(&sh.empty[s]), (uint32_t)(((kt / UM_STAGES) - 1) & 1))) {
          sh.err = 1;
          break;
        }
      }
      const uint32_t sa = tiles + s * stage_bytes;
      const uint32_t bar = su32(&sh.full[s]);
      mb_expect_tx(bar, stage_bytes);
      const int kx = k_begin + kt * UM_BK;
      tma_load_2d(sa, &mapA, kx, m0, bar);
      tma_load_2d(sa + a_bytes, &mapB, kx, 0, bar);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer --------------------------------------------------------------------
    const uint32_t idesc = tf32_idesc(UM_BM, a.BN);
    bool ok = true;
    for (int kt = 0; kt < nk && ok; ++kt) {
      const int s = kt % UM_STAGES;
      if (!mb_wait(su32(&sh.full[s]), (uint32_t)((kt / UM_STAGES) & 1))) {
        sh.err = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = tiles + s * stage_bytes;
      const uint32_t sb = sa + a_bytes;
#pragma unroll
      for (int kk = 0; kk < UM_BK / 8; ++kk) {
        const uint64_t da = sw128_desc(sa + kk * 32);
        const uint64_t db = sw128_desc(sb + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   ::"r"(su32(&sh.empty[s])) : "memory");
    }
    // all MMAs issued (or none): signal the epilogue
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(su32(&sh.accum)) : "memory");
  } else if (warp >= 2) {
    // ---- epilogue ------------------------------------------------------------------------
    const bool ok = mb_wait(su32(&sh.accum), 0u);
    if (!ok) sh.err = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int row = m0 + quarter * 32 + lane;
    float* __restrict__ out = a.out + (size_t)kz * a.split_stride;
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
      if (ok && row < a.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c0 + j;
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0 && sh.err && a.status) atomicExch(a.status, RLU_ETIMEOUT);
}

// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

// 2-D FP32 row-major tensor (rows x cols, ld elements) read in boxes of 32 columns x box_rows.
static int32_t make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows) {
  auto enc = get_encode();
  if (!enc) return RLU_ECUDA;
  if (((uintptr_t)base & 15u) != 0 || (ld * 4) % 16 != 0) return RLU_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)UM_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RLU_OK : RLU_ECUDA;
}

size_t umma_smem_bytes(int BN) {
  return 2048 + (size_t)UM_STAGES * (UM_BM * 128 + (size_t)BN * 128);
}

int32_t umma_tf32_gemm(const UmmaOp& op, cudaStream_t s) {
  if (op.M <= 0 || op.N <= 0 || op.N > 256) return RLU_EINVAL;
  const int BN = (int)round_up(op.N, 16);
  CUtensorMap mA, mB;
  RLU_TRY(make_map(&mA, op.A, op.M, op.K, op.lda, UM_BM));
  RLU_TRY(make_map(&mB, op.B, op.N, op.K, op.ldb, BN));
  int splits = op.splits < 1 ? 1 : op.splits;
  int kchunk = (int)round_up(ceil_div(op.K, splits), UM_BK);
  splits = (int)ceil_div(op.K, kchunk);
  UmmaArgs a{};
  a.M = (int)op.M;
  a.N = (int)op.N;
  a.K = (int)op.K;
  a.BN = BN;
  a.kchunk = kchunk;
  a.status = op.status;
  if (splits == 1) {
    a.out = op.out;
    a.ldo = op.ldo;
    a.out_colmajor = op.out_colmajor;
    a.split_stride = 0;
  } else {
    if (!op.partial) return RLU_ENOMEM;
    a.out = op.partial;
    a.ldo = op.N;
    a.out_colmajor = false;
    a.split_stride = (size_t)op.M * op.N;
  }
  const size_t smem = umma_smem_bytes(BN);
  static bool attr = false;
  if (!attr) {
    RLU_CUDA_TRY(cudaFuncSetAttribute(k_umma_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)umma_smem_bytes(256)));
    attr = true;
  }
  dim3 grid((unsigned)ceil_div(op.M, UM_BM), (unsigned)splits);
  k_umma_tf32<<<grid, UM_THREADS, smem, s>>>(mA, mB, a);
  RLU_TRY(last_launch_status());
  if (splits > 1) return splitk_reduce_f32(op.partial, splits, op.M, op.N, op.out, op.ldo,
                                           !op.out_colmajor, s);
  return RLU_OK;
}

}  // namespace rlu
