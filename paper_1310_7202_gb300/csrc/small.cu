// Small kernels around the two LUs and the pseudo-inverse of Algorithm 1.
//
//  * build_ly (steps 4-5): from the swap-free factored Y and its position map, L_y in pivot
//    row order (Lp, for step 7) and L~ = P^T L_y in original row order (Lt, so that
//    L_y^T P A = L~^T A without permuting A).
//  * chol_inv (step 5, remark after Algorithm 1): M = L_y^T L_y = R^T R (FP64 Cholesky,
//    upper R), then R^{-1} by back substitution; written in FP64 and in the path's type.
//  * gather_lb / gather_u (steps 6 and 8): L_b and U_b read out of the swap-free factored
//    B^T with the column permutation Q.
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

// One CTA. M (k x k, row-major, FP64) is overwritten by R in its upper triangle.
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_inv(double* __restrict__ M, int k,
                                                   double* __restrict__ Rinv,
                                                   T* __restrict__ RinvT,
                                                   int32_t* __restrict__ status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const double d = M[(int64_t)j * k + j];
    if (!(d > 0.0)) {
      if (tid == 0) s_bad = 1;
    }
    const double r = d > 0.0 ? sqrt(d) : 1.0;
    __syncthreads();
    for (int c = j + 1 + tid; c < k; c += nt) M[(int64_t)j * k + c] /= r;
    __syncthreads();
    if (tid == 0) M[(int64_t)j * k + j] = r;
    const int w = k - j - 1;
    for (int64_t e = tid; e < (int64_t)w * w; e += nt) {
      const int a = (int)(e / w), b = (int)(e % w);
      if (b < a) continue;  // upper triangle of the trailing block only
      const int i = j + 1 + a, c = j + 1 + b;
      M[(int64_t)i * k + c] -= M[(int64_t)j * k + i] * M[(int64_t)j * k + c];
    }
    __syncthreads();
  }
  // R^{-1}: column c solves R x = e_c by back substitution (one thread per column)
  for (int c = tid; c < k; c += nt) {
    for (int i = k - 1; i >= 0; --i) {
      double v = 0.0;
      if (i <= c) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int t = i + 1; t <= c; ++t) s -= M[(int64_t)i * k + t] * Rinv[(int64_t)t * k + c];
        v = s / M[(int64_t)i * k + i];
      }
      Rinv[(int64_t)i * k + c] = v;
    }
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)k * k; e += nt) RinvT[e] = (T)Rinv[e];
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
}

template <typename T>
int32_t chol_inv(double* M, int k, double* Rinv, T* RinvT, int32_t* status, cudaStream_t s) {
  k_chol_inv<T><<<1, 1024, 0, s>>>(M, k, Rinv, RinvT, status);
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
