// Algorithm 3 of "Randomized LU Decomposition" (Section 5, rank-deficient least squares) on
// the GPU, from the factors P, Q, L, U of Algorithm 1 (A ~ P^T L U Q^T):
//   c = P b                        k_gather_rows       (c[i] = b[P[i]], gather form of P)
//   y = L^+ c = (L^T L)^{-1} L^T c  Gram in FP64 (SIMT), LDL^T and the blocked substitution
//                                  of step 5 (ldl_factor, trsm_ldl), L^T c (SIMT)
//   z_1 = U_1^{-1} y               k_upper_solve: U_1 = U[:, :k] (upper triangular k x k),
//                                  32-row blocks from the bottom: the solved part's
//                                  contribution by a warp-per-row matrix-vector product, the
//                                  diagonal block by one warp in registers
//   x = Q (z_1, 0)                 the same kernel: x[Q[j]] = z_1[j] for j < k, 0 elsewhere
// One right-hand side per CTA of k_upper_solve; several right-hand sides share the Gram,
// LDL^T and the products.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "small.cuh"

namespace rlu {

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ b, int64_t ldb, const int32_t* __restrict__ P,
                              int64_t m, T* __restrict__ c, int64_t ldc) {
  const int r = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    c[(int64_t)r * ldc + i] = b[(int64_t)r * ldb + P[i]];
}

static constexpr int US_T = 1024;  // threads of k_upper_solve: 32 warps
static constexpr int US_B = 32;    // rows per block

// Column r of Y (row-major k x nrhs, ldy) -> x[:, r] (column-major n x nrhs, ldx).
template <typename T>
__global__ void __launch_bounds__(US_T) k_upper_solve(const T* __restrict__ U, int64_t ldu, int k,
                                                     int64_t n, const int32_t* __restrict__ Q,
                                                     const T* __restrict__ Y, int64_t ldy,
                                                     T* __restrict__ x, int64_t ldx,
                                                     int32_t* __restrict__ zero_pivot) {
  extern __shared__ __align__(16) unsigned char us_smem[];
  T* z = reinterpret_cast<T*>(us_smem);  // [k] the solution, filled from the bottom
  __shared__ T part[US_B];
  const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (k + US_B - 1) / US_B;
  for (int J = nb - 1; J >= 0; --J) {
    const int j0 = J * US_B, bw = min(US_B, k - j0), j1 = j0 + bw;
    // part[i] = y[j0 + i] - sum_{c >= j1} U[j0 + i][c] z[c]: warp i, lanes over columns
    if (warp < bw) {
      const int i = j0 + warp;
      T acc = T(0);
      for (int c = j1 + lane; c < k; c += 32) acc = fma(U[(int64_t)i * ldu + c], z[c], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) part[warp] = Y[(int64_t)i * ldy + r] - acc;
    }
    __syncthreads();
    // the diagonal block: lane i holds row j0 + i; back substitution column by column
    if (warp == 0) {
      T v = lane < bw ? part[lane] : T(0);
      T urow[US_B];
#pragma unroll
      for (int c = 0; c < US_B; ++c)
        urow[c] = (lane < bw && c < bw) ? U[(int64_t)(j0 + lane) * ldu + j0 + c] : T(0);
#pragma unroll
      for (int c = US_B - 1; c >= 0; --c) {
        if (c >= bw) continue;  // uniform across the warp
        const T d = __shfl_sync(0xffffffffu, urow[c], c);  // U[j0 + c][j0 + c]
        T zc = __shfl_sync(0xffffffffu, v, c);
        if (d != T(0)) {
          zc = zc / d;
        } else {  // U_1 singular (rank below k): that component of z_1 is set to 0
          zc = T(0);
          if (lane == 0 && zero_pivot) atomicCAS(zero_pivot, -1, j0 + c);
        }
        if (lane == c) z[j0 + c] = zc;
        if (lane < c) v = fma(-urow[c], zc, v);
      }
    }
    __syncthreads();
  }
  // x = Q (z_1, 0): zeros, then the k entries at their columns Q[j]
  T* xr = x + (int64_t)r * ldx;
  for (int64_t i = tid; i < n; i += US_T) xr[i] = T(0);
  __syncthreads();
  for (int j = tid; j < k; j += US_T) xr[Q[j]] = z[j];
}

struct LsPlan {
  int64_t ldc = 0, nr = 0;
  int kp = 0, split = 1;
  size_t off_c = 0, off_M = 0, off_dinv = 0, off_LT = 0, off_LR = 0, off_W = 0, off_WT = 0,
         off_Cr = 0, off_Y = 0, off_part = 0, total = 0;
};

static size_t ls_carve(size_t& cur, size_t bytes) {
  const size_t at = cur;
  cur += (size_t)round_up((int64_t)bytes, 256);
  return at;
}

static bool ls_plan(int64_t m, int64_t n, int k, int nrhs, int32_t dtype, LsPlan& p) {
  if (m < 1 || n < 1 || k < 1 || k > m || k > n || nrhs < 1) return false;
  if (dtype != RLU_F32 && dtype != RLU_F64) return false;
  const size_t e = dtype == RLU_F64 ? 8 : 4;
  p.ldc = round_up(m, 8);
  p.nr = round_up(nrhs, 4);
  p.kp = (int)round_up(k, 32);
  const int bm = gemm_tile_m(dtype), bn = gemm_tile_n(dtype);
  const int64_t tiles = ceil_div(k, bm) * ceil_div(k, bn);
  int64_t sp = ceil_div(2 * (int64_t)sm_count(), tiles);
  const int64_t kmax = m / 64 > 1 ? m / 64 : 1;
  sp = sp > kmax ? kmax : sp;
  if (dtype == RLU_F32 && sp < 2) sp = 2;  // FP32 partials, FP64 reduction
  p.split = (int)sp;
  size_t cur = 0;
  p.off_c = ls_carve(cur, (size_t)p.ldc * nrhs * e);
  p.off_M = ls_carve(cur, (size_t)k * k * 8);
  p.off_dinv = ls_carve(cur, (size_t)k * 8);
  p.off_LT = ls_carve(cur, (size_t)p.kp * p.kp * e);
  p.off_LR = ls_carve(cur, (size_t)p.kp * p.kp * e);
  p.off_W = ls_carve(cur, (size_t)p.kp * 32 * e);
  p.off_WT = ls_carve(cur, (size_t)p.kp * 32 * e);
  p.off_Cr = ls_carve(cur, (size_t)k * p.nr * e);
  p.off_Y = ls_carve(cur, (size_t)k * p.nr * e);
  p.off_part = ls_carve(cur, (size_t)(p.split + 1) * k * (k > nrhs ? k : nrhs) * e);
  p.total = cur;
  return true;
}

template <typename T>
static int32_t lstsq_t(const LsPlan& p, int64_t m, int64_t n, int k, const int32_t* P,
                       const int32_t* Q, const T* L, int64_t ldl, const T* U, int64_t ldu,
                       const T* b, int64_t ldb, int nrhs, T* x, int64_t ldx, rlu_info* info,
                       char* ws, cudaStream_t s) {
  T* c = reinterpret_cast<T*>(ws + p.off_c);
  double* M = reinterpret_cast<double*>(ws + p.off_M);
  T* Cr = reinterpret_cast<T*>(ws + p.off_Cr);
  T* Yk = reinterpret_cast<T*>(ws + p.off_Y);
  void* part = ws + p.off_part;
  LdlOut<T> o{};
  o.LT = reinterpret_cast<T*>(ws + p.off_LT);
  o.LR = reinterpret_cast<T*>(ws + p.off_LR);
  o.W = reinterpret_cast<T*>(ws + p.off_W);
  o.WT = reinterpret_cast<T*>(ws + p.off_WT);
  o.dinv = reinterpret_cast<double*>(ws + p.off_dinv);
  o.k = k;
  o.kp = p.kp;
  if (info) RLU_TRY(info_init(info, s));
  // c = P b
  int64_t bx = ceil_div(m, 256);
  if (bx > 1024) bx = 1024;
  k_gather_rows<T><<<dim3((unsigned)bx, (unsigned)nrhs), 256, 0, s>>>(b, ldb, P, m, c, p.ldc);
  RLU_TRY(last_launch_status());
  // M = L^T L (FP64), its LDL^T
  {
    GemmOp op{L, ldl, true, L, ldl, true, M, k, true, k, k, m, p.split, part, false};
    RLU_TRY((gemm_simt<T, double>(op, s)));
  }
  RLU_TRY(ldl_factor<T>(M, k, o, info ? &info->status : nullptr, s));
  // Cr = L^T c (k x nrhs, row-major), y = M^{-1} Cr
  {
    GemmOp op{L, ldl, true, c, p.ldc, true, Cr, p.nr, true, k, nrhs, m, p.split, part, false};
    RLU_TRY((gemm_simt<T, T>(op, s)));
  }
  RLU_TRY(trsm_ldl<T>(o, Cr, p.nr, nrhs, Yk, p.nr, s));
  // z_1 = U_1^{-1} y, x = Q (z_1, 0)
  k_upper_solve<T><<<(unsigned)nrhs, US_T, sizeof(T) * (size_t)k, s>>>(
      U, ldu, k, n, Q, Yk, p.nr, x, ldx, info ? &info->first_zero_pivot_b : nullptr);
  return last_launch_status();
}

}  // namespace rlu

using namespace rlu;

extern "C" size_t rlu_lstsq_workspace_size(int64_t m, int64_t n, int32_t k, int32_t nrhs,
                                           int32_t dtype) {
  LsPlan p;
  return ls_plan(m, n, k, nrhs, dtype, p) ? p.total : 0;
}

extern "C" int32_t rlu_lstsq(int32_t dtype, int64_t m, int64_t n, int32_t k, const int32_t* P,
                             const int32_t* Q, const void* L, int64_t ldl, const void* U,
                             int64_t ldu, const void* b, int64_t ldb, int32_t nrhs, void* x,
                             int64_t ldx, rlu_info* info, void* workspace, size_t ws_bytes,
                             void* stream) {
  if (!P || !Q || !L || !U || !b || !x) return RLU_EINVAL;
  if (ldl < m || ldu < n || ldb < m || ldx < n) return RLU_EINVAL;
  LsPlan p;
  if (!ls_plan(m, n, k, nrhs, dtype, p)) return dtype == RLU_BF16 ? RLU_EUNSUPPORTED : RLU_EINVAL;
  if (k > 4096) return RLU_EUNSUPPORTED;  // z_1 in shared memory
  if (workspace == nullptr || ws_bytes < p.total) return RLU_ENOMEM;
  if (((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == RLU_F64)
    return lstsq_t<double>(p, m, n, k, P, Q, (const double*)L, ldl, (const double*)U, ldu,
                           (const double*)b, ldb, nrhs, (double*)x, ldx, info, (char*)workspace, s);
  return lstsq_t<float>(p, m, n, k, P, Q, (const float*)L, ldl, (const float*)U, ldu,
                        (const float*)b, ldb, nrhs, (float*)x, ldx, info, (char*)workspace, s);
}
