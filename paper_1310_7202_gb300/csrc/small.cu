// Small kernels around the two LUs and the pseudo-inverse of Algorithm 1.
//
//  * build_ly (steps 4-5): from the swap-free factored Y and its position map, L_y in pivot
//    row order (Lp, for step 7) and L~ = P^T L_y in original row order (Lt, so that
//    L_y^T P A = L~^T A without permuting A).
//  * chol_inv (step 5, remark after Algorithm 1): M = L_y^T L_y = L L^T (FP64 Cholesky on a
//    thread-block cluster), then R^{-1} = L^{-T} (R = L^T) by forward substitution, one warp
//    per column; written in FP64 and in the path's type.
//  * gather_lb / gather_u (steps 6 and 8): L_b and U_b read out of the swap-free factored
//    B^T with the column permutation Q.
#include <cooperative_groups.h>

#include "common.cuh"
#include "small.cuh"

namespace rlu {

template <typename T>
__global__ void k_build_ly(const T* __restrict__ Y, int64_t ldy, int64_t m, int k,
                           const int32_t* __restrict__ perm, T* __restrict__ Lt,
                           T* __restrict__ Lp, int64_t ldl) {
  const int c = blockIdx.y;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = perm[p];
    const T v = (c < p) ? Y[(int64_t)c * ldy + r] : (c == p ? T(1) : T(0));
    if (Lp) Lp[(int64_t)c * ldl + p] = v;
    if (Lt) Lt[(int64_t)c * ldl + r] = v;
  }
}

template <typename T>
int32_t build_ly(const T* Y, int64_t ldy, int64_t m, int k, const int32_t* perm, T* Lt, T* Lp,
                 int64_t ldl, cudaStream_t s) {
  const int threads = 256;
  int64_t bx = ceil_div(m, threads);
  if (bx > 4096) bx = 4096;
  k_build_ly<T><<<dim3((unsigned)bx, (unsigned)k), threads, 0, s>>>(Y, ldy, m, k, perm, Lt, Lp, ldl);
  return last_launch_status();
}
template int32_t build_ly<float>(const float*, int64_t, int64_t, int, const int32_t*, float*,
                                 float*, int64_t, cudaStream_t);
template int32_t build_ly<double>(const double*, int64_t, int64_t, int, const int32_t*, double*,
                                  double*, int64_t, cudaStream_t);

// Cholesky M = L L^T (FP64) on one thread-block cluster. M (k x k, row-major, global) is
// read once; block columns of width CB are dealt round-robin to the cluster's CTAs and kept
// in their shared memory. Block step J: the owner factors its panel (rows >= CB*J), one
// cluster barrier, every CTA copies that panel from the owner's shared memory and applies
// the rank-CB update to the block columns it owns. L (lower) is written back over M.
static constexpr int CH_CB = 8;
static constexpr int CH_NT = 256;

// 1/sqrt(d) in FP64 without the long-latency FP64 sqrt and divide: an FP32 seed refined by
// two Newton steps y <- y + y/2 (1 - d y^2) (error ~2^-23 -> ~2^-46 -> rounding level).
// Magnitudes outside the FP32 range take the IEEE path.
__device__ __forceinline__ double rsqrt_fp64(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double r = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, r, y);
  }
  return y;
}

__global__ void __launch_bounds__(CH_NT, 1) k_chol_cluster(double* __restrict__ M, int k,
                                                         double* __restrict__ rdiag,
                                                         int32_t* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int nc = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int nblk = (k + CH_CB - 1) / CH_CB;
  const int mine = (nblk - me + nc - 1) / nc;  // number of block columns this CTA owns
  extern __shared__ __align__(16) double ch_smem[];
  double* panels = ch_smem;                              // [mine][k][CB]
  double* buf = ch_smem + (size_t)mine * k * CH_CB;      // [k][CB] copy of the current panel
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  for (int q = 0; q < mine; ++q) {
    const int J = me + q * nc;
    double* P = panels + (size_t)q * k * CH_CB;
    for (int e = tid; e < k * CH_CB; e += CH_NT) {
      const int i = e / CH_CB, c = e % CH_CB, col = J * CH_CB + c;
      P[e] = (col < k && i >= J * CH_CB) ? M[(int64_t)i * k + col] : 0.0;
    }
  }
  cl.sync();
  for (int J = 0; J < nblk; ++J) {
    const int j0 = J * CH_CB, bw = min(CH_CB, k - j0);
    if (J % nc == me) {
      double* P = panels + (size_t)(J / nc) * k * CH_CB;
      for (int t = 0; t < bw; ++t) {
        const double d = P[(j0 + t) * CH_CB + t];
        if (!(d > 0.0) && tid == 0) s_bad = 1;
        const double inv = d > 0.0 ? rsqrt_fp64(d) : 1.0;  // 1 / L[j0+t][j0+t]
        const double r = d > 0.0 ? d * inv : 1.0;          // L[j0+t][j0+t]
        __syncthreads();
        for (int i = j0 + t + 1 + tid; i < k; i += CH_NT) P[i * CH_CB + t] *= inv;
        if (tid == 0) {
          P[(j0 + t) * CH_CB + t] = r;
          rdiag[j0 + t] = inv;
        }
        __syncthreads();
        const int rows = k - (j0 + t + 1), cols = bw - t - 1;
        for (int e = tid; e < rows * cols; e += CH_NT) {
          const int i = j0 + t + 1 + e / cols, c = t + 1 + e % cols;
          P[i * CH_CB + c] -= P[i * CH_CB + t] * P[(j0 + c) * CH_CB + t];
        }
        __syncthreads();
      }
    }
    cl.sync();
    {
      const double* src = cl.map_shared_rank(panels + (size_t)(J / nc) * k * CH_CB, J % nc);
      for (int e = j0 * CH_CB + tid; e < k * CH_CB; e += CH_NT) buf[e] = src[e];
    }
    __syncthreads();
    for (int q = 0; q < mine; ++q) {
      const int K = me + q * nc;
      if (K <= J) continue;
      double* P = panels + (size_t)q * k * CH_CB;
      const int k0 = K * CH_CB, kw = min(CH_CB, k - k0);
      const int rows = k - k0;
      for (int e = tid; e < rows * kw; e += CH_NT) {
        const int i = k0 + e / kw, c = e % kw;
        double acc = P[i * CH_CB + c];
#pragma unroll
        for (int t = 0; t < CH_CB; ++t)
          if (t < bw) acc = fma(-buf[i * CH_CB + t], buf[(k0 + c) * CH_CB + t], acc);
        P[i * CH_CB + c] = acc;
      }
    }
    __syncthreads();  // the next owner reads its freshly updated panel
  }
  cl.sync();
  for (int q = 0; q < mine; ++q) {
    const int J = me + q * nc;
    const double* P = panels + (size_t)q * k * CH_CB;
    for (int e = tid; e < k * CH_CB; e += CH_NT) {
      const int i = e / CH_CB, c = e % CH_CB, col = J * CH_CB + c;
      if (col < k) M[(int64_t)i * k + col] = (i >= col) ? P[e] : 0.0;
    }
  }
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
  cl.sync();
}

// R^{-1} = L^{-T}: one warp per column j of L^{-1} (forward substitution over i >= j, the
// dot products split across the lanes and summed by shuffles, the diagonal applied as the
// reciprocal computed by the Cholesky); row j of R^{-1} is column j of L^{-1}. Written in
// FP64 (Rinv) and in the path's type (RinvT), both row-major k x k. When the packed lower
// triangle fits, every CTA first copies it into shared memory.
static constexpr int TI_WARPS = 8;

template <typename T, bool PACKED>
__global__ void __launch_bounds__(TI_WARPS * 32) k_tri_inverse(const double* __restrict__ Lm,
                                                              const double* __restrict__ rdiag,
                                                              int k, double* __restrict__ Rinv,
                                                              T* __restrict__ RinvT) {
  extern __shared__ double ti_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * TI_WARPS + warp;
  double* Lp = ti_smem;                                            // packed rows (PACKED)
  double* xs = ti_smem + (PACKED ? (size_t)k * (k + 1) / 2 : 0) + (size_t)warp * k;
  if (PACKED) {
    for (int i = 0; i < k; ++i) {
      const size_t base = (size_t)i * (i + 1) / 2;
      for (int t = threadIdx.x; t <= i; t += TI_WARPS * 32) Lp[base + t] = Lm[(int64_t)i * k + t];
    }
    __syncthreads();
  }
  if (j >= k) return;
  for (int i = lane; i < j; i += 32) {
    Rinv[(int64_t)j * k + i] = 0.0;
    RinvT[(int64_t)j * k + i] = T(0);
  }
  for (int i = j; i < k; ++i) {
    const double* row = PACKED ? Lp + (size_t)i * (i + 1) / 2 : Lm + (int64_t)i * k;
    double s = 0.0;
    for (int t = j + lane; t < i; t += 32) s = fma(row[t], xs[t], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double xi = ((i == j) ? 1.0 - s : -s) * rdiag[i];
    if (lane == 0) {
      xs[i] = xi;
      Rinv[(int64_t)j * k + i] = xi;
      RinvT[(int64_t)j * k + i] = (T)xi;
    }
    __syncwarp();
  }
}

template <typename T>
int32_t chol_inv(double* M, int k, double* Rinv, T* RinvT, int32_t* status, cudaStream_t s) {
  double* rdiag = Rinv + (size_t)k * k;  // k extra doubles after R^{-1}
  const int nblk = (k + CH_CB - 1) / CH_CB;
  int nc = nblk < 16 ? nblk : 16;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  auto bytes_for = [&](int c) {
    const int mine = (nblk + c - 1) / c;
    return (size_t)(mine + 1) * k * CH_CB * sizeof(double);
  };
  while (nc < 16 && bytes_for(nc) + 1024 > (size_t)optin) ++nc;
  const size_t bytes = bytes_for(nc);
  if (bytes + 1024 > (size_t)optin) return RLU_EUNSUPPORTED;
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(CH_NT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_chol_cluster, M, k, rdiag, status));
  RLU_TRY(last_launch_status());
  const size_t xbytes = (size_t)TI_WARPS * k * sizeof(double);
  const size_t pbytes = (size_t)k * (k + 1) / 2 * sizeof(double) + xbytes;
  const unsigned grid = (unsigned)ceil_div(k, TI_WARPS);
  if (pbytes + 1024 <= (size_t)optin) {
    RLU_CUDA_TRY(cudaFuncSetAttribute(k_tri_inverse<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pbytes));
    k_tri_inverse<T, true><<<grid, TI_WARPS * 32, pbytes, s>>>(M, rdiag, k, Rinv, RinvT);
  } else {
    if (xbytes > 48 * 1024)
      RLU_CUDA_TRY(cudaFuncSetAttribute(k_tri_inverse<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xbytes));
    k_tri_inverse<T, false><<<grid, TI_WARPS * 32, xbytes, s>>>(M, rdiag, k, Rinv, RinvT);
  }
  return last_launch_status();
}
template int32_t chol_inv<float>(double*, int, double*, float*, int32_t*, cudaStream_t);
template int32_t chol_inv<double>(double*, int, double*, double*, int32_t*, cudaStream_t);

// L_b (k x k, column-major, ld k): L_b[i][j] = X^T-stored B[i][Q[j]] for i > j, 1 on the
// diagonal, 0 above. B is row-major k x n (ld ldb).
template <typename T>
__global__ void k_gather_lb(const T* __restrict__ B, int64_t ldb, const int32_t* __restrict__ Q,
                            int k, T* __restrict__ Lb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / k), i = (int)(e % k);
    Lb[e] = i > j ? B[(int64_t)i * ldb + Q[j]] : (i == j ? T(1) : T(0));
  }
}

// U (k x n, row-major, ld ldu): U[i][j] = B[i][Q[j]] for j >= i, 0 below the diagonal.
template <typename T>
__global__ void k_gather_u(const T* __restrict__ B, int64_t ldb, const int32_t* __restrict__ Q,
                           int k, int64_t n, T* __restrict__ U, int64_t ldu) {
  const int i = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    U[(int64_t)i * ldu + j] = j >= i ? B[(int64_t)i * ldb + Q[j]] : T(0);
}

template <typename T>
int32_t gather_lb_u(const T* B, int64_t ldb, const int32_t* Q, int k, int64_t n, T* Lb, T* U,
                    int64_t ldu, cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = ceil_div((int64_t)k * k, threads);
  if (blocks > 1024) blocks = 1024;
  k_gather_lb<T><<<(unsigned)blocks, threads, 0, s>>>(B, ldb, Q, k, Lb);
  RLU_TRY(last_launch_status());
  int64_t bx = ceil_div(n, threads);
  if (bx > 1024) bx = 1024;
  k_gather_u<T><<<dim3((unsigned)bx, (unsigned)k), threads, 0, s>>>(B, ldb, Q, k, n, U, ldu);
  return last_launch_status();
}
template int32_t gather_lb_u<float>(const float*, int64_t, const int32_t*, int, int64_t, float*,
                                    float*, int64_t, cudaStream_t);
template int32_t gather_lb_u<double>(const double*, int64_t, const int32_t*, int, int64_t,
                                     double*, double*, int64_t, cudaStream_t);

// Contiguous copy with stride change: dst (rows x cols, column-major ld ldd) <- src (ld lds).
template <typename T>
__global__ void k_copy_cm(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                          int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e % rows;
    dst[c * ldd + r] = src[c * lds + r];
  }
}

template <typename T>
int32_t copy_cm(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                cudaStream_t s) {
  if (rows * cols == 0) return RLU_OK;
  const int threads = 256;
  int64_t blocks = ceil_div(rows * cols, threads);
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_copy_cm<T><<<(unsigned)blocks, threads, 0, s>>>(src, lds, dst, ldd, rows, cols);
  return last_launch_status();
}
template int32_t copy_cm<float>(const float*, int64_t, float*, int64_t, int64_t, int64_t,
                                cudaStream_t);
template int32_t copy_cm<double>(const double*, int64_t, double*, int64_t, int64_t, int64_t,
                                 cudaStream_t);

__global__ void k_info_init(rlu_info* info) {
  info->status = RLU_OK;
  info->first_zero_pivot_y = -1;
  info->first_zero_pivot_b = -1;
  info->nonfinite = 0;
}

int32_t info_init(rlu_info* info, cudaStream_t s) {
  k_info_init<<<1, 1, 0, s>>>(info);
  return last_launch_status();
}

}  // namespace rlu
