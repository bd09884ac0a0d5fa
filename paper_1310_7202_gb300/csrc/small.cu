// Small kernels around the two LUs and the pseudo-inverse of Algorithm 1.
//
//  * build_ly (steps 4-5): from the swap-free factored Y and its position map, L_y in pivot
//    row order (Lp, for step 7) and L~ = P^T L_y in original row order (Lt, so that
//    L_y^T P A = L~^T A without permuting A); optionally L~ split exactly into a TF32 part
//    and an FP32 remainder for the tensor-core products of step 5.
//  * chol_inv (step 5, remark after Algorithm 1): M = L_y^T L_y = L L^T (FP64 Cholesky on a
//    thread-block cluster), then R^{-1} = L^{-T} (R = L^T) by forward substitution, one warp
//    per column; written in FP64 and in the path's type.
//  * gather_lb / gather_u (steps 6 and 8): L_b and U_b read out of the swap-free factored
//    B^T with the column permutation Q.
#include <cooperative_groups.h>

#include "common.cuh"
#include "small.cuh"

namespace rlu {

__device__ __forceinline__ void tf32_split(float x, float* hi, float* lo, int64_t at) {
  const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  hi[at] = h;
  lo[at] = x - h;
}
__device__ __forceinline__ void tf32_split(double, double*, double*, int64_t) {}

template <typename T>
__global__ void k_build_ly(const T* __restrict__ Y, int64_t ldy, int64_t m, int k,
                           const int32_t* __restrict__ perm, T* __restrict__ Lt,
                           T* __restrict__ Lp, int64_t ldl, T* __restrict__ Lhi,
                           T* __restrict__ Llo) {
  const int c = blockIdx.y;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = perm[p];
    const T v = (c < p) ? Y[(int64_t)c * ldy + r] : (c == p ? T(1) : T(0));
    if (Lp) Lp[(int64_t)c * ldl + p] = v;
    if (Lt) Lt[(int64_t)c * ldl + r] = v;
    if (Lhi) tf32_split(v, Lhi, Llo, (int64_t)c * ldl + r);
  }
}

template <typename T>
int32_t build_ly(const T* Y, int64_t ldy, int64_t m, int k, const int32_t* perm, T* Lt, T* Lp,
                 int64_t ldl, cudaStream_t s, T* Lhi, T* Llo) {
  const int threads = 256;
  int64_t bx = ceil_div(m, threads);
  if (bx > 4096) bx = 4096;
  k_build_ly<T><<<dim3((unsigned)bx, (unsigned)k), threads, 0, s>>>(Y, ldy, m, k, perm, Lt, Lp,
                                                                   ldl, Lhi, Llo);
  return last_launch_status();
}
template int32_t build_ly<float>(const float*, int64_t, int64_t, int, const int32_t*, float*,
                                 float*, int64_t, cudaStream_t, float*, float*);
template int32_t build_ly<double>(const double*, int64_t, int64_t, int, const int32_t*, double*,
                                  double*, int64_t, cudaStream_t, double*, double*);

// LDL^T factorization M = L D L^T (FP64, L unit lower) on one thread-block cluster; the
// Cholesky factor is R = D^{1/2} L^T. M (k x k, row-major, global) is read once; block
// columns of width CH_CB are dealt round-robin to the cluster's CTAs and kept in their
// shared memory. Block step J: every CTA copies the factored panel J from its owner's
// shared memory; the owner of panel J+1 first applies that update to panel J+1 and factors
// it (look-ahead), then arrives at the cluster barrier; all CTAs apply the rank-CH_CB
// update to the rest of their panels before waiting on it. The only sequential FP64 chain
// is one reciprocal per column (FP32 seed and one Newton step, no divide or square root).
// L overwrites M in column-major order (M[c*k + i] = L[i][c]); D^{-1/2} goes to rdiag (k
// square roots, independent of each other).
static constexpr int CH_CB = 4;
static constexpr int CH_NT = 256;

// 1/d in FP64: FP32 reciprocal seed and one Newton step (relative error ~2^-44), the IEEE
// divide for magnitudes outside the FP32 range.
__device__ __forceinline__ double rcp_fp64(double d) {
  const double a = fabs(d);
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / d;
  const double y = (double)__frcp_rn((float)d);
  const double e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Factor the panel P (rows j0..k-1, columns 0..bw-1 of block J), right-looking LDL^T:
// column t: d = P[j0+t][t]; L[i][t] = P[i][t] / d (i > j0+t); P[i][c] -= L[i][t] * P[j0+c][t]
// for t < c < bw (the unscaled column value of row j0+c). D and 1/d go to Dd / Di.
__device__ void ldl_panel(double* P, int j0, int bw, int k, double* Dd, double* Di,
                          int* bad) {
  const int tid = threadIdx.x;
  __shared__ double ucol[CH_CB];  // unscaled column t of the diagonal block's rows
  for (int t = 0; t < bw; ++t) {
    const double d = P[(j0 + t) * CH_CB + t];
    const double rd = (d != 0.0) ? rcp_fp64(d) : 0.0;
    if (tid == 0) {
      if (!(d > 0.0)) *bad = 1;
      Dd[j0 + t] = d;
      Di[j0 + t] = rd;
    }
    if (tid > t && tid < bw) ucol[tid] = P[(j0 + tid) * CH_CB + t];
    __syncthreads();
    // rows below: update columns t+1.. with the unscaled column, then scale column t
    const int rows = k - (j0 + t + 1);
    for (int r = tid; r < rows; r += CH_NT) {
      const int i = j0 + t + 1 + r;
      const double l = P[i * CH_CB + t] * rd;
      for (int c = t + 1; c < bw; ++c)
        if (i >= j0 + c) P[i * CH_CB + c] = fma(-l, ucol[c], P[i * CH_CB + c]);
      P[i * CH_CB + t] = l;
    }
    __syncthreads();
  }
}

// Apply the factored panel J (buf: L values, bufs: L values times D, rows j0..k-1) to
// panel K (P): P[i][c] -= sum_t L[i][t] D[t] L[k0+c][t].
__device__ void ldl_update(double* P, const double* buf, const double* bufs, int bw, int k0,
                           int kw, int k) {
  const int tid = threadIdx.x;
  const int rows = k - k0;
  for (int e = tid; e < rows * kw; e += CH_NT) {
    const int i = k0 + e / kw, c = e % kw;
    if (i < k0 + c) continue;  // strictly upper part of the diagonal block: unused
    double acc = P[i * CH_CB + c];
#pragma unroll
    for (int t = 0; t < CH_CB; ++t)
      if (t < bw) acc = fma(-buf[i * CH_CB + t], bufs[(k0 + c) * CH_CB + t], acc);
    P[i * CH_CB + c] = acc;
  }
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
  const int most = (nblk + nc - 1) / nc;       // the same shared-memory layout in every CTA
  extern __shared__ __align__(16) double ch_smem[];
  double* panels = ch_smem;                              // [most][k][CB]
  double* buf = ch_smem + (size_t)most * k * CH_CB;      // [k][CB] copy of the current panel
  double* bufs = buf + (size_t)k * CH_CB;                // [k][CB] the copy times D
  double* Dd = bufs + (size_t)k * CH_CB;                 // [k] D
  double* Di = Dd + k;                                   // [k] 1/D (owner's panels only)
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
  __syncthreads();
  if (me == 0) ldl_panel(panels, 0, min(CH_CB, k), k, Dd, Di, &s_bad);
  cluster_arrive();
  cluster_wait();
  for (int J = 0; J < nblk; ++J) {
    const int j0 = J * CH_CB, bw = min(CH_CB, k - j0);
    const int owner = J % nc;
    {  // copy panel J and its D values from the owner
      const double* src = cl.map_shared_rank(panels + (size_t)(J / nc) * k * CH_CB, owner);
      for (int e = j0 * CH_CB + tid; e < k * CH_CB; e += CH_NT) buf[e] = src[e];
      const double* srcD = cl.map_shared_rank(Dd, owner);
      if (tid < bw) Dd[j0 + tid] = srcD[j0 + tid];
    }
    __syncthreads();
    for (int e = j0 * CH_CB + tid; e < k * CH_CB; e += CH_NT)
      bufs[e] = (e % CH_CB < bw) ? buf[e] * Dd[j0 + e % CH_CB] : 0.0;
    __syncthreads();
    const int Jn = J + 1;
    if (Jn < nblk && Jn % nc == me) {  // look-ahead: next panel first, then factor it
      double* Pn = panels + (size_t)(Jn / nc) * k * CH_CB;
      const int k0 = Jn * CH_CB, kw = min(CH_CB, k - k0);
      ldl_update(Pn, buf, bufs, bw, k0, kw, k);
      __syncthreads();
      ldl_panel(Pn, k0, kw, k, Dd, Di, &s_bad);
    }
    cluster_arrive();  // panel J+1 is final in its owner's shared memory
    for (int q = 0; q < mine; ++q) {
      const int K = me + q * nc;
      if (K <= Jn) continue;
      ldl_update(panels + (size_t)q * k * CH_CB, buf, bufs, bw, K * CH_CB,
                 min(CH_CB, k - K * CH_CB), k);
    }
    __syncthreads();
    cluster_wait();
  }
  // write L (unit lower, row-major, zero above) and D^{-1/2}
  for (int q = 0; q < mine; ++q) {
    const int J = me + q * nc;
    const double* P = panels + (size_t)q * k * CH_CB;
    for (int e = tid; e < k * CH_CB; e += CH_NT) {
      const int i = e / CH_CB, c = e % CH_CB, col = J * CH_CB + c;
      if (col < k) M[(int64_t)col * k + i] = (i > col) ? P[e] : (i == col ? 1.0 : 0.0);
    }
    for (int c = tid; c < CH_CB; c += CH_NT) {
      const int col = J * CH_CB + c;
      if (col < k) rdiag[col] = Dd[col] > 0.0 ? sqrt(Di[col]) : 0.0;
    }
  }
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
  cl.sync();
}

// R^{-1} = L^{-T} D^{-1/2}: one single-warp CTA per column j of L^{-1} (L unit lower,
// column-major), so the FP64 work spreads over all SMs. Right-looking substitution: once
// x_t is final it is broadcast and every lane folds L[i][t] x_t into the partial sums of the
// rows i it owns, so the sequential chain per step is one shuffle and one FMA. Row j of
// R^{-1} is column j of L^{-1} scaled elementwise by D^{-1/2}; written in FP64 (Rinv) and in
// the path's type (RinvT), both row-major k x k.

template <typename T>
__global__ void __launch_bounds__(32) k_tri_inverse(const double* __restrict__ Lc,
                                                   const double* __restrict__ rdiag, int k,
                                                   double* __restrict__ Rinv,
                                                   T* __restrict__ RinvT) {
  const int lane = threadIdx.x;
  const int j = blockIdx.x;
  for (int i = lane; i < j; i += 32) {
    Rinv[(int64_t)j * k + i] = 0.0;
    RinvT[(int64_t)j * k + i] = T(0);
  }
  // right-looking substitution for column j of L^{-1}: s_i accumulates sum_t L[i][t] x_t;
  // lane (i mod 32) owns s_i; x_t = -s_t (x_j = 1) is broadcast once it is final. Column t of
  // L (contiguous in Lc) is loaded one step ahead.
  constexpr int MAXQ = 16;  // k <= 512
  constexpr int PF = 4;     // columns loaded ahead
  const int nq = (k + 31) / 32;
  double sacc[MAXQ], col[PF][MAXQ];
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) sacc[q] = 0.0;
#pragma unroll
  for (int f = 0; f < PF; ++f)
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int i = lane + 32 * q;
      col[f][q] = (q < nq && j + f < k && i < k) ? Lc[(int64_t)(j + f) * k + i] : 0.0;
    }
  for (int t = j; t < k; ++t) {
    const int qt = t >> 5;
    double xt = 0.0;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q)
      if (q == qt) xt = sacc[q];
    xt = (t == j) ? 1.0 : -xt;
    xt = __shfl_sync(0xffffffffu, xt, t & 31);
    if (lane == 0) {
      const double r = xt * rdiag[t];
      Rinv[(int64_t)j * k + t] = r;
      RinvT[(int64_t)j * k + t] = (T)r;
    }
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int i = lane + 32 * q;
      if (q < nq && i > t && i < k) sacc[q] = fma(col[0][q], xt, sacc[q]);
    }
    // shift the prefetch window and load column t + PF
#pragma unroll
    for (int f = 0; f + 1 < PF; ++f)
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) col[f][q] = col[f + 1][q];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int i = lane + 32 * q;
      col[PF - 1][q] = (q < nq && t + PF < k && i < k) ? Lc[(int64_t)(t + PF) * k + i] : 0.0;
    }
  }
}

template <typename T>
int32_t chol_inv(double* M, int k, double* Rinv, T* RinvT, int32_t* status, cudaStream_t s) {
  double* rdiag = Rinv + (size_t)k * k;  // k extra doubles after R^{-1}: D^{-1/2}
  const int nblk = (k + CH_CB - 1) / CH_CB;
  int nc = nblk < 16 ? nblk : 16;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  auto bytes_for = [&](int c) {
    const int mine = (nblk + c - 1) / c;
    return (size_t)(mine + 2) * k * CH_CB * sizeof(double) + 2 * (size_t)k * sizeof(double);
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
  if (k > 512) return RLU_EUNSUPPORTED;
  k_tri_inverse<T><<<(unsigned)k, 32, 0, s>>>(M, rdiag, k, Rinv, RinvT);
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
