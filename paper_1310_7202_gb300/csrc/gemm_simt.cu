// SIMT (CUDA-core) GEMMs for the plain FP32 and FP64 paths:
//   step 2  Y = A G,   step 5  C = L~^T A,  M = L~^T L~,  T = R^-T C,  B = R^-1 T,
//   step 7  L = L_y L_b.
// C(M x N) = A(M x K) * B(K x N). Each operand is either K-contiguous ("K-major") or
// contiguous along its other dimension; C is row- or column-major. Split-K writes dense
// row-major partial slices that a second kernel sums in a fixed order (deterministic).
//
// Tiling: BM x BN x BK tiles in double-buffered shared memory; each thread owns a
// (2*V) x (2*V) register micro-tile split into two V-wide column groups and two V-tall row
// groups (V = 16 bytes / sizeof(T)) so that shared-memory fragment reads are 16-byte vector
// loads without bank conflicts.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "umma.cuh"

namespace rlu {

template <typename T> struct GemmCfg;
template <> struct GemmCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 16, V = 4, TX = 16, TY = 16;
};
template <> struct GemmCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, V = 2, TX = 16, TY = 16;
};
// the smaller FP32 tile of the batched products (chosen per step by the autotuner)
struct GemmCfgF64x64 {
  static constexpr int BM = 64, BN = 64, BK = 16, V = 2, TX = 16, TY = 16;
};

// V consecutive elements of T as one vector load
template <typename T, int V> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<double, 2> { using type = double2; };

// One BM x BN output tile (bx, by) of K range slice bz; the output element type OutT may be
// wider than T (the batched Gram matrix is stored in FP64 for the LDL^T).
template <typename T, typename OutT, bool AK, bool BKM, bool CR, typename Cfg = GemmCfg<T>>
__device__ __forceinline__ void gemm_tile(const GemmArgs& p, int bx, int by, int bz) {
  constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, V = Cfg::V;
  constexpr int NT = Cfg::TX * Cfg::TY;
  constexpr int PAD = V;
  constexpr int A_LD = BM * BK / NT, B_LD = BN * BK / NT;
  using VT = typename Vec<T, V>::type;

  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];

  const T* __restrict__ A = static_cast<const T*>(p.A);
  const T* __restrict__ Bm = static_cast<const T*>(p.B);
  const int tid = threadIdx.x;
  const int tx = tid % Cfg::TX, ty = tid / Cfg::TX;
  const int64_t m0 = (int64_t)by * BM, n0 = (int64_t)bx * BN;
  const int64_t kbeg = (int64_t)bz * p.kchunk;
  const int64_t kend = (kbeg + p.kchunk < p.K) ? kbeg + p.kchunk : p.K;

  T acc[2 * V][2 * V];
#pragma unroll
  for (int i = 0; i < 2 * V; ++i)
#pragma unroll
    for (int j = 0; j < 2 * V; ++j) acc[i][j] = T(0);

  T ra[A_LD], rb[B_LD];
  auto load_tile = [&](int64_t k0) {
#pragma unroll
    for (int i = 0; i < A_LD; ++i) {
      const int idx = tid + i * NT;
      const int r = AK ? idx / BK : idx % BM;
      const int kk = AK ? idx % BK : idx / BM;
      const int64_t gm = m0 + r, gk = k0 + kk;
      ra[i] = (gm < p.M && gk < kend) ? A[AK ? gm * p.lda + gk : gk * p.lda + gm] : T(0);
    }
#pragma unroll
    for (int i = 0; i < B_LD; ++i) {
      const int idx = tid + i * NT;
      const int c = BKM ? idx / BK : idx % BN;
      const int kk = BKM ? idx % BK : idx / BN;
      const int64_t gn = n0 + c, gk = k0 + kk;
      rb[i] = (gn < p.N && gk < kend) ? Bm[BKM ? gn * p.ldb + gk : gk * p.ldb + gn] : T(0);
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int i = 0; i < A_LD; ++i) {
      const int idx = tid + i * NT;
      const int r = AK ? idx / BK : idx % BM;
      const int kk = AK ? idx % BK : idx / BM;
      As[buf][kk][r] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < B_LD; ++i) {
      const int idx = tid + i * NT;
      const int c = BKM ? idx / BK : idx % BN;
      const int kk = BKM ? idx % BK : idx / BN;
      Bs[buf][kk][c] = rb[i];
    }
  };

  if (kbeg < kend) {
    load_tile(kbeg);
    store_tile(0);
  }
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool has_next = k0 + BK < kend;
    if (has_next) load_tile(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[2 * V], b[2 * V];
      const VT a0 = *reinterpret_cast<const VT*>(&As[buf][kk][ty * V]);
      const VT a1 = *reinterpret_cast<const VT*>(&As[buf][kk][BM / 2 + ty * V]);
      const VT b0 = *reinterpret_cast<const VT*>(&Bs[buf][kk][tx * V]);
      const VT b1 = *reinterpret_cast<const VT*>(&Bs[buf][kk][BN / 2 + tx * V]);
      memcpy(&a[0], &a0, sizeof(VT));
      memcpy(&a[V], &a1, sizeof(VT));
      memcpy(&b[0], &b0, sizeof(VT));
      memcpy(&b[V], &b1, sizeof(VT));
#pragma unroll
      for (int i = 0; i < 2 * V; ++i)
#pragma unroll
        for (int j = 0; j < 2 * V; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (has_next) store_tile(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  OutT* __restrict__ Cm = static_cast<OutT*>(p.C) + (int64_t)bz * p.split_stride;
#pragma unroll
  for (int i = 0; i < 2 * V; ++i) {
    const int64_t gm = m0 + (i < V ? ty * V + i : BM / 2 + ty * V + (i - V));
    if (gm >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 2 * V; ++j) {
      const int64_t gn = n0 + (j < V ? tx * V + j : BN / 2 + tx * V + (j - V));
      if (gn >= p.N) continue;
      const OutT v = (OutT)(p.alpha_neg ? -acc[i][j] : acc[i][j]);
      if (CR)
        Cm[gm * p.ldc + gn] = v;
      else
        Cm[gn * p.ldc + gm] = v;
    }
  }
}

template <typename T, bool AK, bool BKM, bool CR>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmArgs p) {
  gemm_tile<T, T, AK, BKM, CR>(p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched form: problem blockIdx.z of the table, whole K range (no split); CTAs past the
// problem's own tile counts return at once.
template <typename T, typename OutT, bool AK, bool BKM, bool CR, typename Cfg>
__global__ void __launch_bounds__(256) k_gemm_simt_batched(const GemmArgs* __restrict__ table) {
  const GemmArgs p = table[blockIdx.z];
  if ((int64_t)blockIdx.y * Cfg::BM >= p.M || (int64_t)blockIdx.x * Cfg::BN >= p.N) return;
  gemm_tile<T, OutT, AK, BKM, CR, Cfg>(p, blockIdx.x, blockIdx.y, 0);
}

// out(i, j) = sum_z part[z][i][j], z ascending; accumulation and output in OutT.
template <typename T, typename OutT>
__global__ void k_splitk_reduce(const T* __restrict__ part, int splits, int64_t M, int64_t N,
                                int64_t slice, OutT* __restrict__ out, int64_t ldo,
                                bool out_rowmajor) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    OutT s = OutT(0);
    for (int z = 0; z < splits; ++z) s += (OutT)part[z * slice + e];
    const int64_t i = e / N, j = e % N;
    if (out_rowmajor)
      out[i * ldo + j] = s;
    else
      out[j * ldo + i] = s;
  }
}

// The same sum for a column-major output (out(i, j) at out[j * ldo + i]): 32 x 32 tiles
// staged in shared memory, so that the partial slices are read along their rows and the
// output is written along its columns (both coalesced); z ascending as above.
template <typename T, typename OutT>
__global__ void __launch_bounds__(256) k_splitk_reduce_t(const T* __restrict__ part, int splits,
                                                         int64_t M, int64_t N, int64_t slice,
                                                         OutT* __restrict__ out, int64_t ldo) {
  __shared__ OutT tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + tx;
    OutT s = OutT(0);
    if (i < M && j < N)
      for (int z = 0; z < splits; ++z) s += (OutT)part[z * slice + i * N + j];
    tile[r][tx] = s;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int64_t j = j0 + c, i = i0 + tx;
    if (i < M && j < N) out[j * ldo + i] = tile[tx][c];
  }
}

template <typename T>
static void launch_variant(const GemmArgs& a, bool AK, bool BKM, bool CR, dim3 grid,
                           cudaStream_t s) {
#define RLU_GEMM_CASE(x, y, z)                                              \
  if (AK == x && BKM == y && CR == z) {                                    \
    k_gemm_simt<T, x, y, z><<<grid, 256, 0, s>>>(a);                       \
    return;                                                                \
  }
  RLU_GEMM_CASE(true, true, true)
  RLU_GEMM_CASE(true, true, false)
  RLU_GEMM_CASE(true, false, true)
  RLU_GEMM_CASE(true, false, false)
  RLU_GEMM_CASE(false, true, true)
  RLU_GEMM_CASE(false, true, false)
  RLU_GEMM_CASE(false, false, true)
  RLU_GEMM_CASE(false, false, false)
#undef RLU_GEMM_CASE
}

template <typename T, typename OutT, typename Cfg>
static int32_t gemm_batched_cfg(const GemmArgs* table_dev, int count, int64_t max_m,
                                int64_t max_n, bool a_kmajor, bool b_kmajor, bool c_rowmajor,
                                cudaStream_t s) {
  const dim3 grid((unsigned)ceil_div(max_n, Cfg::BN), (unsigned)ceil_div(max_m, Cfg::BM),
                  (unsigned)count);
#define RLU_GEMM_BCASE(x, y, z)                                                        \
  if (a_kmajor == x && b_kmajor == y && c_rowmajor == z) {                             \
    k_gemm_simt_batched<T, OutT, x, y, z, Cfg><<<grid, 256, 0, s>>>(table_dev);        \
    return last_launch_status();                                                       \
  }
  RLU_GEMM_BCASE(true, true, true)
  RLU_GEMM_BCASE(true, true, false)
  RLU_GEMM_BCASE(true, false, true)
  RLU_GEMM_BCASE(true, false, false)
  RLU_GEMM_BCASE(false, true, true)
  RLU_GEMM_BCASE(false, true, false)
  RLU_GEMM_BCASE(false, false, true)
  RLU_GEMM_BCASE(false, false, false)
#undef RLU_GEMM_BCASE
  return RLU_EINVAL;
}

template <typename T, typename OutT>
int32_t gemm_simt_batched(const GemmArgs* table_dev, int count, int64_t max_m, int64_t max_n,
                          bool a_kmajor, bool b_kmajor, bool c_rowmajor, cudaStream_t s,
                          int tile) {
  if (count <= 0) return RLU_OK;
  if (count > 65535) return RLU_EINVAL;
  if (tile == 1)
    return gemm_batched_cfg<T, OutT, GemmCfgF64x64>(table_dev, count, max_m, max_n, a_kmajor,
                                                    b_kmajor, c_rowmajor, s);
  return gemm_batched_cfg<T, OutT, GemmCfg<T>>(table_dev, count, max_m, max_n, a_kmajor,
                                               b_kmajor, c_rowmajor, s);
}
template int32_t gemm_simt_batched<float, float>(const GemmArgs*, int, int64_t, int64_t, bool,
                                                 bool, bool, cudaStream_t, int);
template int32_t gemm_simt_batched<float, double>(const GemmArgs*, int, int64_t, int64_t, bool,
                                                  bool, bool, cudaStream_t, int);

template <typename T>
size_t gemm_partial_bytes(int64_t M, int64_t N, int splits) {
  return splits > 1 ? (size_t)splits * (size_t)M * (size_t)N * sizeof(T) : 0;
}

template <typename T, typename OutT>
int32_t gemm_simt(const GemmOp& op, cudaStream_t s) {
  using Cfg = GemmCfg<T>;
  if (op.M == 0 || op.N == 0) return RLU_OK;
  const int64_t tiles_m = ceil_div(op.M, Cfg::BM), tiles_n = ceil_div(op.N, Cfg::BN);
  int splits = op.splits < 1 ? 1 : op.splits;
  int64_t kchunk = round_up(ceil_div(op.K > 0 ? op.K : 1, splits), Cfg::BK);
  splits = (int)ceil_div(op.K > 0 ? op.K : 1, kchunk);
  GemmArgs a;
  a.A = op.A; a.lda = op.lda;
  a.B = op.B; a.ldb = op.ldb;
  a.M = op.M; a.N = op.N; a.K = op.K;
  a.kchunk = kchunk;
  a.alpha_neg = op.negate;
  const dim3 grid((unsigned)tiles_n, (unsigned)tiles_m, (unsigned)splits);
  const bool direct = (splits == 1) && std::is_same<T, OutT>::value;
  if (direct) {
    a.C = op.C; a.ldc = op.ldc; a.split_stride = 0;
    launch_variant<T>(a, op.a_kmajor, op.b_kmajor, op.c_rowmajor, grid, s);
    return last_launch_status();
  }
  if (op.partial == nullptr) return RLU_ENOMEM;
  a.C = op.partial; a.ldc = op.N; a.split_stride = op.M * op.N;
  launch_variant<T>(a, op.a_kmajor, op.b_kmajor, true, grid, s);
  RLU_TRY(last_launch_status());  // the split-K product
  if (!op.c_rowmajor && ceil_div(op.M, 32) <= 65535) {
    const dim3 tgrid((unsigned)ceil_div(op.N, 32), (unsigned)ceil_div(op.M, 32));
    k_splitk_reduce_t<T, OutT><<<tgrid, 256, 0, s>>>(static_cast<const T*>(op.partial), splits,
                                                     op.M, op.N, op.M * op.N,
                                                     static_cast<OutT*>(op.C), op.ldc);
    return last_launch_status();
  }
  const int threads = 256;
  int64_t blocks = ceil_div(op.M * op.N, threads);
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_splitk_reduce<T, OutT><<<(unsigned)blocks, threads, 0, s>>>(
      static_cast<const T*>(op.partial), splits, op.M, op.N, op.M * op.N,
      static_cast<OutT*>(op.C), op.ldc, op.c_rowmajor);
  return last_launch_status();
}

template int32_t gemm_simt<float, float>(const GemmOp&, cudaStream_t);
template int32_t gemm_simt<float, double>(const GemmOp&, cudaStream_t);
template int32_t gemm_simt<double, double>(const GemmOp&, cudaStream_t);
template size_t gemm_partial_bytes<float>(int64_t, int64_t, int);
template size_t gemm_partial_bytes<double>(int64_t, int64_t, int);

int32_t splitk_reduce_f32(const float* part, int splits, int64_t M, int64_t N, float* out,
                          int64_t ldo, bool out_rowmajor, cudaStream_t s) {
  if (!out_rowmajor) {
    if (ceil_div(M, 32) > 65535) return RLU_EUNSUPPORTED;
    const dim3 grid((unsigned)ceil_div(N, 32), (unsigned)ceil_div(M, 32));
    k_splitk_reduce_t<float, float><<<grid, 256, 0, s>>>(part, splits, M, N, M * N, out, ldo);
    return last_launch_status();
  }
  const int threads = 256;
  int64_t blocks = ceil_div(M * N, threads);
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_splitk_reduce<float, float><<<(unsigned)blocks, threads, 0, s>>>(part, splits, M, N, M * N,
                                                                    out, ldo, out_rowmajor);
  return last_launch_status();
}

__global__ void __launch_bounds__(256) k_splitk_reduce_cm(const float* __restrict__ part,
                                                          int splits, int64_t M, int64_t N,
                                                          float* __restrict__ out,
                                                          int64_t ldo) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[z * total + e];
    const int64_t j = e / M, i = e - j * M;
    out[j * ldo + i] = s;
  }
}

int32_t splitk_reduce_cm_f32(const float* part, int splits, int64_t M, int64_t N, float* out,
                             int64_t ldo, cudaStream_t s) {
  int64_t blocks = ceil_div(M * N, 256);
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_splitk_reduce_cm<<<(unsigned)blocks, 256, 0, s>>>(part, splits, M, N, out, ldo);
  return last_launch_status();
}

int32_t splitk_reduce_f64(const float* part, int splits, int64_t M, int64_t N, double* out,
                          int64_t ldo, cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = ceil_div(M * N, threads);
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_splitk_reduce<float, double><<<(unsigned)blocks, threads, 0, s>>>(part, splits, M, N, M * N,
                                                                     out, ldo, true);
  return last_launch_status();
}

int gemm_tile_m(int32_t dtype) { return dtype == RLU_F64 ? GemmCfg<double>::BM : GemmCfg<float>::BM; }
int gemm_tile_n(int32_t dtype) { return dtype == RLU_F64 ? GemmCfg<double>::BN : GemmCfg<float>::BN; }

}  // namespace rlu
