// Small kernels around the two LUs and the pseudo-inverse of Algorithm 1.
//
//  * build_ly (steps 4-5): from the swap-free factored Y and its position map, L_y in pivot
//    row order (Lp, for step 7) and L~ = P^T L_y in original row order (Lt, so that
//    L_y^T P A = L~^T A without permuting A); optionally L~ split exactly into a TF32 part
//    and an FP32 remainder, and into three BF16 parts, for the tensor-core products of
//    step 5.
//  * ldl_factor (step 5, remark after Algorithm 1): M = L_y^T L_y = L D L^T (the Cholesky
//    factor is D^{1/2} L^T), plus the inverses of L's 32 x 32 diagonal blocks: in FP32 on
//    one CTA for the single-precision paths (k <= 256), else in FP64 on a thread-block
//    cluster; trsm_ldl then forms B = M^{-1} C = L^{-T} D^{-1} L^{-1} C by blocked
//    substitution in the path's type.
//  * gather_lb / gather_u (steps 6 and 8): L_b and U_b read out of the swap-free factored
//    B^T with the column permutation Q.
#include <cooperative_groups.h>

#include <algorithm>

#include <utility>

#include "common.cuh"
#include "small.cuh"
#include "batched.cuh"

namespace rlu {

__device__ __forceinline__ void tf32_split(float x, float* hi, float* lo, int64_t at) {
  const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  hi[at] = h;
  lo[at] = x - h;
}
__device__ __forceinline__ void tf32_split(double, double*, double*, int64_t) {}

// x = hi + mid + lo with each part a BF16 (8 significant bits): hi = bf16(x), the
// remainders x - hi and (x - hi) - mid are exact in FP32, so hi + mid + lo carries 24 bits.
__device__ __forceinline__ void bf16_split3(float x, __nv_bfloat16* h, __nv_bfloat16* mi,
                                            __nv_bfloat16* lo, int64_t at) {
  const __nv_bfloat16 a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  h[at] = a;
  mi[at] = b;
  lo[at] = __float2bfloat16_rn(r2);
}

template <typename T>
__global__ void k_build_ly(const T* __restrict__ Y, int64_t ldy, int64_t m, int k,
                           const int32_t* __restrict__ perm, T* __restrict__ Lt,
                           T* __restrict__ Lp, int64_t ldl, T* __restrict__ Lhi,
                           T* __restrict__ Llo, Bf16Parts bp) {
  const int c = blockIdx.y;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = perm[p];
    const T v = (c < p) ? Y[(int64_t)c * ldy + r] : (c == p ? T(1) : T(0));
    if (Lp) Lp[(int64_t)c * ldl + p] = v;
    if (Lt) Lt[(int64_t)c * ldl + r] = v;
    if (Lhi) tf32_split(v, Lhi, Llo, (int64_t)c * ldl + r);
    if (bp.hi) bf16_split3((float)v, bp.hi, bp.mid, bp.lo, (int64_t)c * ldl + r);
  }
}

// Splits of a column-major rows x cols FP32 matrix X (ld) for the FP32-accurate products:
// exact TF32 pairs (hi, lo; when hi != NULL) and/or three BF16 parts (when bp.hi != NULL),
// written with the same ld.
__global__ void k_split_parts(const float* __restrict__ X, int64_t ld, int64_t rows, int cols,
                              float* __restrict__ hi, float* __restrict__ lo, Bf16Parts bp,
                              int64_t ldo) {
  const int c = blockIdx.y;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[(int64_t)c * ld + r];
    const int64_t at = (int64_t)c * ldo + r;
    if (hi) tf32_split(v, hi, lo, at);
    if (bp.hi) bf16_split3(v, bp.hi, bp.mid, bp.lo, at);
  }
}

int32_t split_parts(const float* X, int64_t ld, int64_t rows, int cols, float* hi, float* lo,
                    Bf16Parts bp, cudaStream_t s, int64_t ldo) {
  if (rows <= 0 || cols <= 0) return RLU_OK;
  int64_t bx = ceil_div(rows, 256);
  if (bx > 1024) bx = 1024;
  k_split_parts<<<dim3((unsigned)bx, (unsigned)cols), 256, 0, s>>>(X, ld, rows, cols, hi, lo, bp,
                                                                  ldo > 0 ? ldo : ld);
  return last_launch_status();
}

template <typename T>
int32_t build_ly(const T* Y, int64_t ldy, int64_t m, int k, const int32_t* perm, T* Lt, T* Lp,
                 int64_t ldl, cudaStream_t s, T* Lhi, T* Llo, Bf16Parts bp) {
  const int threads = 256;
  int64_t bx = ceil_div(m, threads);
  if (bx > 4096) bx = 4096;
  k_build_ly<T><<<dim3((unsigned)bx, (unsigned)k), threads, 0, s>>>(Y, ldy, m, k, perm, Lt, Lp,
                                                                   ldl, Lhi, Llo, bp);
  return last_launch_status();
}
template int32_t build_ly<float>(const float*, int64_t, int64_t, int, const int32_t*, float*,
                                 float*, int64_t, cudaStream_t, float*, float*, Bf16Parts);
template int32_t build_ly<double>(const double*, int64_t, int64_t, int, const int32_t*, double*,
                                  double*, int64_t, cudaStream_t, double*, double*, Bf16Parts);

// LDL^T factorization M = L D L^T (FP64, L unit lower) on one thread-block cluster; the
// Cholesky factor is R = D^{1/2} L^T. M (k x k, row-major, global) is read once; block
// columns of width CH_CB are dealt round-robin to the cluster's CTAs and kept in their
// shared memory. Block step J: every CTA copies the factored panel J from its owner's
// shared memory; the owner of panel J+1 first applies that update to panel J+1 and factors
// it (look-ahead), then arrives at the cluster barrier; all CTAs apply the rank-CH_CB
// update to the rest of their panels before waiting on it. The only sequential FP64 chain
// is one reciprocal per column (FP32 seed and one Newton step, no divide or square root).
// L overwrites M in column-major order (M[c*k + i] = L[i][c]); 1/D goes to dinv.
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
                                                         double* __restrict__ rdiag,  // 1/D
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
  // write L (unit lower, column-major, zero above) and 1/D
  for (int q = 0; q < mine; ++q) {
    const int J = me + q * nc;
    const double* P = panels + (size_t)q * k * CH_CB;
    for (int e = tid; e < k * CH_CB; e += CH_NT) {
      const int i = e / CH_CB, c = e % CH_CB, col = J * CH_CB + c;
      if (col < k) M[(int64_t)col * k + i] = (i > col) ? P[e] : (i == col ? 1.0 : 0.0);
    }
    for (int c = tid; c < CH_CB; c += CH_NT) {
      const int col = J * CH_CB + c;
      if (col < k) rdiag[col] = Di[col];
    }
  }
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
  cl.sync();
}

// Inverses of the TB x TB diagonal blocks of the unit lower L (FP64, column-major k x k),
// one warp per block, column by column (right-looking, no divides); results and L itself
// converted to the path's type for the triangular solves.
static constexpr int TB = 32;

template <typename T>
__global__ void __launch_bounds__(32) k_diag_inv(const double* __restrict__ Lc, int k,
                                                 LdlOut<T> o) {
  const int lane = threadIdx.x, b = blockIdx.x;
  const int b0 = b * TB, bw = min(TB, k - b0);
  // this block's columns of L in the path's type, zero-padded to kp x kp, both layouts
  for (int c = b0; c < b0 + TB; ++c)
    for (int i = lane; i < o.kp; i += 32) {
      const T v = (c < k && i < k) ? (T)Lc[(int64_t)c * k + i] : (i == c ? T(1) : T(0));
      o.LT[(int64_t)c * o.kp + i] = v;
      o.LR[(int64_t)i * o.kp + c] = v;
    }
  // column j of the block inverse: x_j = 1, x_i = -sum_{t<i} L[i][t] x_t (lane i owns x_i)
  for (int j = 0; j < TB; ++j) {
    double x = (lane == j) ? 1.0 : 0.0;
    for (int t = j; t < bw; ++t) {
      const double xt = __shfl_sync(0xffffffffu, x, t);
      if (lane > t && lane < bw) x = fma(-Lc[(int64_t)(b0 + t) * k + b0 + lane], xt, x);
    }
    // W block b row-major (element (lane, j)) and its transpose
    const T w = (lane < bw && j < bw) ? (T)x : (lane == j ? T(1) : T(0));
    o.W[(size_t)b * TB * TB + lane * TB + j] = w;
    o.WT[(size_t)b * TB * TB + j * TB + lane] = w;
  }
}

// FP32 LDL^T for k <= 256 on one CTA (the normal-equation matrix of Algorithm 1's step 5
// in single precision: its rounding enters the factorization error ||PAQ - LU|| only
// through L_y (B - B*), orthogonal to the residual of the exact least-squares B*). Blocked
// right-looking with 32 x 32 blocks of the lower triangle in shared memory:
//   diagonal block J: one warp, in registers (lane i holds row i): d_t, L_JJ and
//     W_J = L_JJ^{-1};
//   block column J: U_IJ = M_IJ W_J^T (= L_IJ D_J), L_IJ = U_IJ D_J^{-1};
//   trailing blocks: M_IK -= L_IJ U_KJ^T (I >= K > J), 4 x 4 register tiles per thread.
// Rows/columns past k are padded with the identity, which factors trivially.
static constexpr int LB = 32;       // block size
static constexpr int LBP = LB + 1;  // padded row of a block in shared memory
static constexpr int L32_NT = 512;
static constexpr int L32_MAXB = 8;  // k <= 256

__device__ __forceinline__ int tri_blk(int I, int J) { return I * (I + 1) / 2 + J; }

// Reciprocal of a pivot: the hardware approximation refined by one Newton-Raphson step
// (y' = y + y (1 - d y)), within an ulp or so of 1/d.
__device__ __forceinline__ float rcp_nr(float d) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(d));
  return isfinite(y) ? fmaf(y, fmaf(-d, y, 1.0f), y) : y;
}

// Column t of the register-resident LDL^T of a 32 x 32 block (lane i holds row i):
// d = M[t][t]; rows below get L[i][t] = M[i][t] / d and the rank-1 update of columns > t.
// Column t (= row t, by symmetry) is broadcast through the 32-float shared row bc: one
// store per lane, then 16-byte broadcast loads, cheaper than one shuffle per column.
template <int t>
__device__ __forceinline__ void ldl_col(float (&a)[LB], float* bc, int lane, float* d_out,
                                        bool& bad) {
  __syncwarp();
  bc[lane] = a[t];  // M[lane][t], the unscaled column
  __syncwarp();
  const float d = bc[t];
  const float rd = rcp_nr(d);
  bad |= !(d > 0.f) || !(d < INFINITY);
  const float l = a[t] * rd;
#pragma unroll
  for (int c0 = (t + 1) / 4 * 4; c0 < LB; c0 += 4) {
    const float4 u = *reinterpret_cast<const float4*>(bc + c0);
    const float uc[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c0 + q > t && lane > t) a[c0 + q] = fmaf(-l, uc[q], a[c0 + q]);
  }
  if (lane == t) d_out[t] = d;
  if (lane > t) a[t] = l;
}
template <int... ts>
__device__ __forceinline__ void ldl_cols(float (&a)[LB], float* bc, int lane, float* d_out,
                                         bool& bad, std::integer_sequence<int, ts...>) {
  (ldl_col<ts>(a, bc, lane, d_out, bad), ...);
}

// One warp: LDL^T of the 32 x 32 block BJJ in place (L unit lower, zero above), D into dJ
// and W = L^{-1} (row-major, padded rows) into W. Returns true in the lanes whose pivot was
// not positive and finite.
__device__ __forceinline__ bool ldl_diag_block(float* BJJ, float* dJ, float* W, int lane) {
  __shared__ __align__(16) float bc[LB];
  float a[LB];
#pragma unroll
  for (int c = 0; c < LB; ++c) a[c] = BJJ[lane * LBP + c];
  bool bad = false;
  ldl_cols(a, bc, lane, dJ, bad, std::make_integer_sequence<int, LB>{});
#pragma unroll
  for (int c = 0; c < LB; ++c) BJJ[lane * LBP + c] = (c < lane) ? a[c] : (c == lane ? 1.f : 0.f);
  __syncwarp();
  // W = L^{-1} by forward substitution, lane c computing column c:
  // W[i][c] = [i == c] - sum_{j < i} L[i][j] W[j][c] (zero above the diagonal by itself);
  // L[i][j] is the same for every lane, a broadcast load. Two partial sums per entry.
  float w[LB];
#pragma unroll
  for (int i = 0; i < LB; ++i) {
    float s0 = (i == lane) ? 1.f : 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const float lij = BJJ[i * LBP + j];
      if (j & 1) s1 = fmaf(-lij, w[j], s1);
      else s0 = fmaf(-lij, w[j], s0);
    }
    w[i] = s0 + s1;
  }
#pragma unroll
  for (int i = 0; i < LB; ++i) W[i * LBP + lane] = w[i];
  __syncwarp();
  return bad;
}

// C (32 x 32 block) -= A B^T (kSub) or C = A B^T for 32 x 32 blocks A, B (padded rows), one
// 4 x 4 register tile (tile 0..63) per call.
template <bool kSub = true>
__device__ __forceinline__ void gemm_nt_tile(float* C, const float* A, const float* B, int tile) {
  const int r0 = (tile / 8) * 4, c0 = (tile % 8) * 4;
  float acc[4][4] = {};
#pragma unroll 8
  for (int t = 0; t < LB; ++t) {
    float lv[4], uv[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      lv[x] = A[(r0 + x) * LBP + t];
      uv[x] = B[(c0 + x) * LBP + t];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(lv[x], uv[y], acc[x][y]);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      if (kSub) C[(r0 + x) * LBP + c0 + y] -= acc[x][y];
      else C[(r0 + x) * LBP + c0 + y] = acc[x][y];
    }
}

template <int NT>
__device__ __forceinline__ void ldl32_body(const double* __restrict__ M, int k,
                                           const LdlOut<float>& o, int32_t* __restrict__ status) {
  extern __shared__ __align__(16) float l32_smem[];
  const int nb = (k + LB - 1) / LB;
  const int nblk = nb * (nb + 1) / 2;
  float* Bk = l32_smem;                         // [nblk][LB][LBP] lower-triangle blocks
  float* Ub = Bk + (size_t)nblk * LB * LBP;     // [nb][LB][LBP] U_IJ of the current J
  float* Wb = Ub + (size_t)nb * LB * LBP;       // [nb][LB][LBP] W_J = L_JJ^{-1}
  float* dd = Wb + (size_t)nb * LB * LBP;       // [nb * LB] D
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_bad = 0;
  // block (I, J) row r: warp-wide rows, 8 of them in flight per warp
  for (int q0 = warp; q0 < nblk * LB; q0 += (NT / 32) * 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * (NT / 32);  // block row: block q / LB, row q % LB
      const int b = q / LB, r = q % LB;
      int I = 0;
      while (tri_blk(I + 1, 0) <= b) ++I;
      const int i = I * LB + r, j = (b - tri_blk(I, 0)) * LB + lane;
      v[u] = (q < nblk * LB && i < k && j < k) ? (float)M[(int64_t)i * k + j] : (i == j ? 1.f : 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * (NT / 32);
      if (q < nblk * LB) Bk[(size_t)(q / LB) * LB * LBP + (q % LB) * LBP + lane] = v[u];
    }
  }
  __syncthreads();
  for (int J = 0; J < nb; ++J) {
    if (warp == 0) {
      const bool bad = ldl_diag_block(Bk + (size_t)tri_blk(J, J) * LB * LBP, dd + J * LB,
                                      Wb + (size_t)J * LB * LBP, lane);
      if (bad && J * LB + lane < k) s_bad = 1;
    }
    __syncthreads();
    // U_IJ = M_IJ W_J^T in 4 x 4 register tiles (16 independent sums per thread), then
    // L_IJ = U_IJ D_J^{-1} in place once every tile of the block column has read M_IJ
    const int rest = nb - 1 - J;
    const float* W = Wb + (size_t)J * LB * LBP;
    for (int q = tid; q < rest * 64; q += NT) {
      const int I = J + 1 + q / 64;
      gemm_nt_tile<false>(Ub + (size_t)(I - J - 1) * LB * LBP,
                          Bk + (size_t)tri_blk(I, J) * LB * LBP, W, q % 64);
    }
    __syncthreads();
    for (int e = tid; e < rest * LB * LB; e += NT) {
      const int I = J + 1 + e / (LB * LB), r = (e / LB) % LB, c = e % LB;
      Bk[(size_t)tri_blk(I, J) * LB * LBP + r * LBP + c] =
          Ub[(size_t)(I - J - 1) * LB * LBP + r * LBP + c] / dd[J * LB + c];
    }
    __syncthreads();
    // trailing update of the lower-triangle blocks I >= K > J; 64 4x4 tiles per block
    const int ntask = rest * (rest + 1) / 2 * 64;
    for (int q = tid; q < ntask; q += NT) {
      const int pb = q / 64, tile = q % 64;
      int ii = 0;
      while ((ii + 1) * (ii + 2) / 2 <= pb) ++ii;
      const int kk = pb - ii * (ii + 1) / 2;
      const int I = J + 1 + ii, K = J + 1 + kk;
      gemm_nt_tile(Bk + (size_t)tri_blk(I, K) * LB * LBP, Bk + (size_t)tri_blk(I, J) * LB * LBP,
                   Ub + (size_t)(K - J - 1) * LB * LBP, tile);
    }
    __syncthreads();
  }
  // L (unit lower, zero above, identity past k) in both layouts, the diagonal-block
  // inverses and their transposes, 1/D
  const int kp = o.kp;
  for (int x = warp; x < kp; x += NT / 32) {  // LT row x = column x of L; LR row x
    for (int y = lane; y < kp; y += 32) {
      const int X = x / LB, Y = y / LB;
      float lt = 0.f, lr = 0.f;
      if (y > x) lt = Bk[(size_t)tri_blk(Y, X) * LB * LBP + (y % LB) * LBP + x % LB];
      else if (y == x) lt = 1.f;
      if (x > y) lr = Bk[(size_t)tri_blk(X, Y) * LB * LBP + (x % LB) * LBP + y % LB];
      else if (x == y) lr = 1.f;
      o.LT[(size_t)x * kp + y] = lt;
      o.LR[(size_t)x * kp + y] = lr;
    }
  }
  for (int q = warp; q < nb * LB; q += NT / 32) {  // row q % LB of block q / LB
    const float* Wq = Wb + (size_t)(q / LB) * LB * LBP;
    const int r = q % LB;
    o.W[(size_t)q * LB + lane] = Wq[r * LBP + lane];
    o.WT[(size_t)q * LB + lane] = Wq[lane * LBP + r];
  }
  for (int i = tid; i < k; i += NT) o.dinv[i] = 1.0 / (double)dd[i];
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
}

__global__ void __launch_bounds__(L32_NT, 1) k_ldl32(const double* __restrict__ M, int k,
                                                    LdlOut<float> o, int32_t* __restrict__ status) {
  ldl32_body<L32_NT>(M, k, o, status);
}

// Batched form: problem blockIdx.x of the table. Batches whose k stay within 128 (at most
// four 32 x 32 block columns) take 128 threads, so that several problems share an SM.
template <int NT>
__global__ void __launch_bounds__(NT) k_ldl32_batched(const Ldl32Job* __restrict__ jobs) {
  const Ldl32Job& j = jobs[blockIdx.x];
  ldl32_body<NT>(j.M, j.k, j.o, j.status);
}

static size_t ldl32_smem_bytes(int k) {
  const int nb = (k + LB - 1) / LB;
  return sizeof(float) * ((size_t)(nb * (nb + 1) / 2 + 2 * nb) * LB * LBP + (size_t)nb * LB);
}

static int32_t ldl_cluster_f64(double* M, int k, double* dinv, int32_t* status, cudaStream_t s) {
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
  RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_chol_cluster, M, k, dinv, status));
  return last_launch_status();
}

// FP32 LDL^T for k <= 512 on a thread-block cluster of nc <= 8 CTAs: the blocked
// algorithm of k_ldl32 with the block rows of the lower triangle dealt round-robin (row I
// to CTA I mod nc, blocks (I, 0..I) in its shared memory). Block step J:
//   the owner of row J factors the diagonal block (one warp): D_J, L_JJ, W_J = L_JJ^{-1};
//   cluster barrier; every CTA copies W_J and D_J and forms U_IJ = M_IJ W_J^T and
//     L_IJ = U_IJ D_J^{-1} for its rows I > J;
//   cluster barrier; every CTA copies the U_KJ it needs (K > J) from their owners and
//     updates its blocks M_IK -= L_IJ U_KJ^T (I >= K > J).
// Two cluster barriers per block step; the trailing work is spread over the cluster.
static constexpr int LC_NT = 512;
static constexpr int LC_MAXB = 16;  // k <= 512
static constexpr int LC_BS = LB * LBP;

__host__ __device__ __forceinline__ int lc_mine(int nb, int me, int nc) {
  return (nb - me + nc - 1) / nc;
}
// blocks held before owned row q (rows me, me + nc, ...: row I holds I + 1 blocks)
__host__ __device__ __forceinline__ int lc_row_off(int q, int me, int nc) {
  return q * (me + 1) + nc * q * (q - 1) / 2;
}

__global__ void __launch_bounds__(LC_NT, 1) k_ldl32c(const double* __restrict__ M, int k,
                                                    LdlOut<float> o,
                                                    int32_t* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int nc = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (k + LB - 1) / LB;
  const int mine = lc_mine(nb, me, nc);
  // the same layout in every CTA (remote addresses are mapped from local ones): room for
  // the largest row set and the most rows of any CTA
  int most = 0;
  for (int c = 0; c < nc; ++c) most = max(most, lc_row_off(lc_mine(nb, c, nc), c, nc));
  const int mmax = lc_mine(nb, 0, nc);
  extern __shared__ __align__(16) float lc_smem[];
  float* Rw = lc_smem;                     // owned rows' blocks
  float* Ub = Rw + (size_t)most * LC_BS;   // [mmax] U_IJ of the owned rows I > J
  float* Uf = Ub + (size_t)mmax * LC_BS;   // [nb] U_KJ of this step, fetched
  float* Wo = Uf + (size_t)nb * LC_BS;     // W_J when this CTA owns row J
  float* Wf = Wo + LC_BS;                  // W_J of this step, fetched
  float* dd = Wf + LC_BS;                  // [nb * LB] D
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  auto blk = [&](int q, int K) { return Rw + (size_t)(lc_row_off(q, me, nc) + K) * LC_BS; };

  for (int q = 0; q < mine; ++q) {
    const int I = me + q * nc;
    float* R = blk(q, 0);
    const int ne = (I + 1) * LB * LB;
    for (int e0 = tid; e0 < ne; e0 += LC_NT * 4) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * LC_NT;
        const int K = e / (LB * LB), r = (e / LB) % LB, c = e % LB;
        const int i = I * LB + r, j = K * LB + c;
        v[u] = (e < ne && i < k && j < k) ? (float)M[(int64_t)i * k + j] : (i == j ? 1.f : 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * LC_NT;
        const int K = e / (LB * LB), r = (e / LB) % LB, c = e % LB;
        if (e < ne) R[(size_t)K * LC_BS + r * LBP + c] = v[u];
      }
    }
  }
  __syncthreads();
  const int imax = me + (mine - 1) * nc;  // last owned row (mine >= 1: nc <= nb)

  for (int J = 0; J < nb; ++J) {
    const int ow = J % nc;
    if (me == ow && warp == 0) {
      const int q = (J - me) / nc;
      const bool bad = ldl_diag_block(blk(q, J), dd + J * LB, Wo, lane);
      if (bad && J * LB + lane < k) s_bad = 1;
      for (int e = lane; e < LB * LB; e += 32) {  // W_J and its transpose for the solves
        const int r = e / LB, c = e % LB;
        o.W[(size_t)J * LB * LB + e] = Wo[r * LBP + c];
        o.WT[(size_t)J * LB * LB + e] = Wo[c * LBP + r];
      }
    }
    cluster_arrive();
    cluster_wait();
    {
      const float* src = cl.map_shared_rank(Wo, ow);
      for (int e = tid; e < LC_BS; e += LC_NT) Wf[e] = src[e];
      if (me != ow && tid < LB) dd[J * LB + tid] = cl.map_shared_rank(dd, ow)[J * LB + tid];
    }
    __syncthreads();
    // U_IJ = M_IJ W_J^T for the owned rows I > J
    const int q0 = (J < me) ? 0 : (J - me) / nc + 1;  // first owned row below J
    for (int t = tid; t < (mine - q0) * 64; t += LC_NT) {
      const int q = q0 + t / 64;
      gemm_nt_tile<false>(Ub + (size_t)q * LC_BS, blk(q, J), Wf, t % 64);
    }
    __syncthreads();
    for (int q = q0; q < mine; ++q) {  // L_IJ = U_IJ D_J^{-1} in place
      float* Lr = blk(q, J);
      const float* U = Ub + (size_t)q * LC_BS;
      for (int e = tid; e < LB * LB; e += LC_NT) {
        const int r = e / LB, c = e % LB;
        Lr[r * LBP + c] = U[r * LBP + c] / dd[J * LB + c];
      }
    }
    cluster_arrive();
    cluster_wait();
    if (imax > J) {  // fetch U_KJ, J < K <= imax, from the owners of rows K
      const int nf = (imax - J) * LC_BS;
      for (int e = tid; e < nf; e += LC_NT) {
        const int K = J + 1 + e / LC_BS, x = e % LC_BS;
        const int own = K % nc;
        Uf[(size_t)K * LC_BS + x] = cl.map_shared_rank(Ub, own)[(size_t)((K - own) / nc) * LC_BS + x];
      }
    }
    __syncthreads();
    for (int q = q0; q < mine; ++q) {  // M_IK -= L_IJ U_KJ^T, J < K <= I
      const int I = me + q * nc;
      const float* Lr = blk(q, J);
      const int ntask = (I - J) * 64;
      for (int t = tid; t < ntask; t += LC_NT) {
        const int K = J + 1 + t / 64;
        gemm_nt_tile(blk(q, K), Lr, Uf + (size_t)K * LC_BS, t % 64);
      }
    }
    __syncthreads();
  }
  // the owned rows of L (unit lower, zero above, identity past k) in both layouts, 1/D
  const int kp = o.kp;
  for (int q = 0; q < mine; ++q) {
    const int I = me + q * nc;
    for (int e = tid; e < LB * kp; e += LC_NT) {
      const int r = e / kp, c = e % kp, i = I * LB + r;
      if (i >= kp) continue;
      float v = 0.f;
      if (i > c) v = blk(q, c / LB)[(r)*LBP + c % LB];
      else if (i == c) v = 1.f;
      o.LR[(size_t)i * kp + c] = v;
      o.LT[(size_t)c * kp + i] = v;
    }
    for (int r = tid; r < LB; r += LC_NT) {
      const int i = I * LB + r;
      if (i < k) o.dinv[i] = 1.0 / (double)dd[i];
    }
  }
  if (tid == 0 && s_bad && status) *status = RLU_EINVAL;
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

static size_t ldl32c_smem_bytes(int k, int nc) {
  const int nb = (k + LB - 1) / LB;
  int most = 0, mmax = 0;
  for (int me = 0; me < nc; ++me) {
    const int mine = lc_mine(nb, me, nc);
    most = std::max(most, lc_row_off(mine, me, nc));
    mmax = std::max(mmax, mine);
  }
  return sizeof(float) * ((size_t)(most + mmax + nb + 2) * LC_BS + (size_t)nb * LB);
}

static int32_t ldl32_cluster(const double* M, int k, const LdlOut<float>& o, int32_t* status,
                             cudaStream_t s) {
  const int nb = (k + LB - 1) / LB;
  const int nc = nb < 8 ? nb : 8;
  const size_t bytes = ldl32c_smem_bytes(k, nc);
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (bytes + 1024 > (size_t)optin) return RLU_EUNSUPPORTED;
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_ldl32c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(LC_NT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_ldl32c, M, k, o, status));
  return last_launch_status();
}

template <typename T>
int32_t ldl_factor(double* M, int k, const LdlOut<T>& o, int32_t* status, cudaStream_t s) {
  if (sizeof(T) == sizeof(float) && k <= L32_MAXB * LB) {
    const size_t bytes = ldl32_smem_bytes(k);
    RLU_CUDA_TRY(cudaFuncSetAttribute(k_ldl32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k_ldl32<<<1, L32_NT, bytes, s>>>(M, k, reinterpret_cast<const LdlOut<float>&>(o), status);
    return last_launch_status();
  }
  if (sizeof(T) == sizeof(float) && k <= LC_MAXB * LB)
    return ldl32_cluster(M, k, reinterpret_cast<const LdlOut<float>&>(o), status, s);
  RLU_TRY(ldl_cluster_f64(M, k, o.dinv, status, s));
  k_diag_inv<T><<<(unsigned)ceil_div(k, TB), 32, 0, s>>>(M, k, o);
  return last_launch_status();
}
bool ldl_factor_supported(int k, bool f32) {
  if (k < 1) return false;
  if (f32 && k <= LC_MAXB * LB) return true;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int nblk = (k + CH_CB - 1) / CH_CB;
  const int mine = (nblk + 15) / 16;
  return (size_t)(mine + 2) * k * CH_CB * sizeof(double) + 2 * (size_t)k * sizeof(double) + 1024 <=
         (size_t)optin;
}

template int32_t ldl_factor<float>(double*, int, const LdlOut<float>&, int32_t*, cudaStream_t);
template int32_t ldl_factor<double>(double*, int, const LdlOut<double>&, int32_t*, cudaStream_t);

// B = L^{-T} D^{-1} L^{-1} C (step 5, the normal equations M B = C with M = L D L^T), TC
// columns of C per CTA. The kp x TC block X stays in shared memory (rows past k are zero)
// through blocked forward substitution -- row block I is updated by the solved blocks above
// it (X_I -= L_IJ X_J, a 32 x 32 x TC product per block), then multiplied by W_I, the
// inverse of L's diagonal block --, the D^{-1} scaling, and blocked backward substitution
// (X_I -= L_JI^T X_J for J > I, then W_I^T). The 32 x 32 blocks of L, L^T, W^T and W are
// consumed in a fixed order and streamed through a ring of shared-memory stages with
// cp.async, several blocks ahead of the arithmetic. C and B: k x n row-major (ld ldc / ldb).
static constexpr int TSTAGES = 4;
static constexpr int LSP = TB + 4;  // staged block row: 16-byte aligned rows, [t][r] order

template <typename T>
struct Vec4 {
  T v[4];
};
__device__ __forceinline__ Vec4<float> lds4(const float* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return {{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ Vec4<double> lds4(const double* p) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0];
  const double2 q1 = reinterpret_cast<const double2*>(p)[1];
  return {{q0.x, q0.y, q1.x, q1.y}};
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Source of the s-th block of the sequence, stored so that the staged block reads [t][r]:
// forward row block I: L(I, J) for J < I (from LT: t = column of L, r = row), then W_I^T;
// backward row block I (descending): L(J, I)^T for J > I (from LR), then W_I.
template <typename T>
__device__ __forceinline__ const T* trsm_block_src(const LdlOut<T>& o, int nb, int s,
                                                   int64_t* stride) {
  const int F = nb * (nb + 1) / 2;
  const bool fwd = s < F;
  const int q = fwd ? s : s - F;
  int I = 0;  // q-th item: I-th group (I + 1 items, the last one the diagonal inverse)
  while ((I + 1) * (I + 2) / 2 <= q) ++I;
  const int J = q - I * (I + 1) / 2;
  *stride = (J < I) ? o.kp : TB;  // rows of L / L^T blocks have stride kp, inverses TB
  if (fwd) {
    if (J < I) return o.LT + (int64_t)(J * TB) * o.kp + I * TB;
    return o.WT + (size_t)I * TB * TB;
  }
  const int Ib = nb - 1 - I;  // backward row block
  if (J < I) return o.LR + (int64_t)((nb - 1 - J) * TB) * o.kp + Ib * TB;
  return o.W + (size_t)Ib * TB * TB;
}

template <typename T, int TC>
__device__ __forceinline__ void trsm_body(const LdlOut<T>& o, const T* __restrict__ C, int64_t ldc,
                                          int64_t n, T* __restrict__ B, int64_t ldb, int bx) {
  // two thread groups split the 32 rows of each staged block (the reduction index) in
  // halves; their partial sums meet in the diagonal step, where every thread owns 2 x 4
  constexpr int NG = TB / 4 * TC / 4;  // threads of one group
  constexpr int NT = 2 * NG;
  constexpr int CH = 16 / sizeof(T);   // elements per 16-byte copy
  constexpr int CPB = TB * TB / CH;    // copies per block
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  const int k = o.k, kp = o.kp, nb = kp / TB;
  T* Xs = reinterpret_cast<T*>(trsm_smem);  // [kp][TC]
  T* Ls = Xs + (size_t)kp * TC;             // [TSTAGES][TB][LSP]
  T* Ws = Ls + (size_t)TSTAGES * TB * LSP;  // [2][TB][TC] the groups' partial sums
  const int tid = threadIdx.x;
  const int g = tid / NG, gt = tid % NG;
  const int64_t c0 = (int64_t)bx * TC;
  const int nseq = nb * (nb + 1);
  auto issue = [&](int sidx) {
    if (sidx < nseq) {
      int64_t stride = 0;
      const T* src = trsm_block_src(o, nb, sidx, &stride);
      T* dst = Ls + (size_t)(sidx % TSTAGES) * TB * LSP;
      for (int e = tid; e < CPB; e += NT) {
        const int t = e / (TB / CH), r = (e % (TB / CH)) * CH;
        cp_async16(dst + t * LSP + r, src + (int64_t)t * stride + r);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int sidx = 0; sidx < TSTAGES - 1; ++sidx) issue(sidx);
  // batches of independent loads, so that their latencies overlap
  constexpr int LDU = 8;
  for (int e0 = tid; e0 < kp * TC; e0 += NT * LDU) {
    T v[LDU];
#pragma unroll
    for (int u = 0; u < LDU; ++u) {
      const int e = e0 + u * NT, i = e / TC, c = e % TC;
      v[u] = (i < k && c0 + c < n) ? C[(int64_t)i * ldc + c0 + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LDU; ++u)
      if (e0 + u * NT < kp * TC) Xs[e0 + u * NT] = v[u];
  }
  const int r0 = (gt / (TC / 4)) * 4, cc = (gt % (TC / 4)) * 4;  // update tile (4 x 4)
  const int q0 = (tid / (TC / 4)) * 2, qc = (tid % (TC / 4)) * 4;  // diagonal tile (2 x 4)
  const int th = g * (TB / 2);                                    // this group's rows t
  int sidx = 0;
  // wait for block sidx, prefetch block sidx + TSTAGES - 1; returns the staged block
  auto next_block = [&]() -> const T* {
    cp_async_wait<TSTAGES - 2>();
    __syncthreads();
    issue(sidx + TSTAGES - 1);
    return Ls + (size_t)(sidx++ % TSTAGES) * TB * LSP;
  };
  T acc[4][4];
  auto start_row_block = [&](int I) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        acc[a][b] = (g == 0) ? Xs[(size_t)(I * TB + r0 + a) * TC + cc + b] : T(0);
  };
  auto update = [&](int j0) {  // acc -= staged [t][r] (this group's half of t) x X[j0 + t]
    const T* Lb = next_block();
#pragma unroll 4
    for (int t = th; t < th + TB / 2; ++t) {
      const Vec4<T> l = lds4(Lb + t * LSP + r0);
      const Vec4<T> x = lds4(Xs + (size_t)(j0 + t) * TC + cc);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(-l.v[a], x.v[b], acc[a][b]);
    }
  };
  auto diag = [&](int I) {  // X_I = W-block (staged [t][r]) applied to the summed partials
    T* Wg = Ws + (size_t)g * TB * TC;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Wg[(r0 + a) * TC + cc + b] = acc[a][b];
    const T* Db = next_block();  // its __syncthreads also publishes the partials
    T v[2][4] = {};
#pragma unroll 4
    for (int t = 0; t < TB; ++t) {
      const T w0 = Db[t * LSP + q0], w1 = Db[t * LSP + q0 + 1];
      const Vec4<T> x0 = lds4(Ws + t * TC + qc);
      const Vec4<T> x1 = lds4(Ws + (size_t)TB * TC + t * TC + qc);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const T x = x0.v[b] + x1.v[b];
        v[0][b] = fma(w0, x, v[0][b]);
        v[1][b] = fma(w1, x, v[1][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Xs[(size_t)(I * TB + q0 + a) * TC + qc + b] = v[a][b];
  };
  __syncthreads();
  for (int I = 0; I < nb; ++I) {
    start_row_block(I);
    for (int J = 0; J < I; ++J) update(J * TB);
    diag(I);
  }
  __syncthreads();
  for (int e = tid; e < k * TC; e += NT) Xs[e] = (T)((double)Xs[e] * o.dinv[e / TC]);
  __syncthreads();
  for (int I = nb - 1; I >= 0; --I) {
    start_row_block(I);
    for (int J = nb - 1; J > I; --J) update(J * TB);
    diag(I);
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int e = tid; e < k * TC; e += NT) {
    const int i = e / TC, c = e % TC;
    if (c0 + c < n) B[(int64_t)i * ldb + c0 + c] = Xs[e];
  }
}

template <typename T, int TC>
__global__ void __launch_bounds__(TB / 2 * TC / 4) k_trsm_ldl(LdlOut<T> o, const T* __restrict__ C,
                                                             int64_t ldc, int64_t n,
                                                             T* __restrict__ B, int64_t ldb) {
  trsm_body<T, TC>(o, C, ldc, n, B, ldb, blockIdx.x);
}

// Batched form over a tile list: entry blockIdx.x = (problem, 64-column block).
__global__ void __launch_bounds__(TB / 2 * 64 / 4) k_trsm_batched(const TrsmJob* __restrict__ jobs,
                                                                 const int2* __restrict__ tiles) {
  const int2 t = tiles[blockIdx.x];
  const TrsmJob& j = jobs[t.x];
  trsm_body<float, 64>(j.o, j.C, j.ldc, j.n, j.B, j.ldb, t.y);
}

// The same solve, right-looking: per block column J of L one pass X_J = W_J X_J, then one
// pass X_I -= L_IJ X_J over every row block below J at once (forward), D^{-1}, then from the
// last block Y_J = W_J^T Y_J and Y_I -= L_JI^T Y_J over every row block above J (backward).
// 2 nb passes per direction instead of nb (nb + 1) / 2 block steps, each with all its rows'
// work in flight. A pass needs 32 contiguous rows of L^T (forward: L^T row 32 J + t, columns
// past the block) or of L (backward: L row 32 J + t, columns before the block) and the
// diagonal block's inverse (W_J, or W_J^T backward): they stream into the other slot of a
// two-slot cp.async ring while the current pass computes. 256 threads; in the update passes
// each thread owns a TR x 4 tile (a warp: 32 / (TC / 4) row groups x TC / 4 column groups),
// so every k-step is TR / 4 + 1 16-byte shared loads for 4 TR multiply-adds. D^{-1} is
// applied in the storage precision (its reciprocals rounded once).
static constexpr int RL_NT = 256;

template <typename T>
__host__ __device__ constexpr int rl_lpad(int kp) { return kp + 16 / (int)sizeof(T); }

template <typename T, int TC, int TR>
__global__ void __launch_bounds__(RL_NT) k_trsm_rl(LdlOut<T> o, const T* __restrict__ C,
                                                   int64_t ldc, int64_t n, T* __restrict__ B,
                                                   int64_t ldb) {
  constexpr int CH = 16 / sizeof(T);  // elements per 16-byte copy
  constexpr int CG = TC / 4;          // column groups of a warp in the update passes
  constexpr int RG = 32 / CG;         // row groups (8 rows each) of a warp
  constexpr int CPT = TC / 32;        // columns per thread in the diagonal passes
  static_assert(TC == 32 || TC == 64, "TC");
  extern __shared__ __align__(16) unsigned char rl_smem[];
  const int k = o.k, kp = o.kp, nb = kp / TB, LP = rl_lpad<T>(kp);
  T* Xs = reinterpret_cast<T*>(rl_smem);        // [kp][TC]
  T* Ls = Xs + (size_t)kp * TC;                 // [2][TB][LP] rows of L^T / L
  T* Wsm = Ls + (size_t)2 * TB * LP;            // [2][TB][LSP] W_J / W_J^T
  T* Dsm = Wsm + (size_t)2 * TB * LSP;          // [kp] 1 / D
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int npass = 2 * nb;  // pass q: forward block q (q < nb), backward block 2 nb - 1 - q
  // stage pass q's operands into slot q & 1
  auto stage = [&](int q) {
    if (q < npass) {
      const bool fwd = q < nb;
      const int J = fwd ? q : npass - 1 - q;
      const int i0 = fwd ? (J + 1) * TB : 0, i1 = fwd ? kp : J * TB;  // rows updated
      const T* Lsrc = fwd ? o.LT : o.LR;
      T* Ld = Ls + (size_t)(q & 1) * TB * LP;
      const int per = (i1 - i0) / CH;  // 16-byte pieces per row
      for (int e = tid; e < TB * per; e += RL_NT) {
        const int t = e / per, i = i0 + (e % per) * CH;
        cp_async16(Ld + t * LP + (i - i0), Lsrc + (int64_t)(J * TB + t) * kp + i);
      }
      const T* Wsrc = (fwd ? o.W : o.WT) + (size_t)J * TB * TB;
      T* Wd = Wsm + (size_t)(q & 1) * TB * LSP;
      for (int e = tid; e < TB * TB / CH; e += RL_NT) {
        const int r = e / (TB / CH), c = (e % (TB / CH)) * CH;
        cp_async16(Wd + r * LSP + c, Wsrc + r * TB + c);
      }
    }
    cp_async_commit();
  };
  stage(0);
  for (int i = tid; i < kp; i += RL_NT) Dsm[i] = i < k ? (T)o.dinv[i] : T(0);
  constexpr int LDU = 8;  // batches of independent loads
  for (int e0 = tid; e0 < kp * TC; e0 += RL_NT * LDU) {
    T v[LDU];
#pragma unroll
    for (int u = 0; u < LDU; ++u) {
      const int e = e0 + u * RL_NT, i = e / TC, c = e % TC;
      v[u] = (i < k && c0 + c < n) ? C[(int64_t)i * ldc + c0 + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LDU; ++u)
      if (e0 + u * RL_NT < kp * TC) Xs[e0 + u * RL_NT] = v[u];
  }
  const int dr = warp * 4;          // diagonal pass: rows dr .. dr + 3 of the block
  const int dc = lane * CPT;        //   and columns dc .. dc + CPT - 1
  const int ug = lane / CG;         // update pass: row group of this thread in the warp strip
  const int uc = (lane % CG) * 4;   //   and its 4 columns
  for (int q = 0; q < npass; ++q) {
    const bool fwd = q < nb;
    const int J = fwd ? q : npass - 1 - q;
    if (q == nb) {  // between the directions: X = D^{-1} X
      __syncthreads();
      for (int e = tid; e < k * TC; e += RL_NT) Xs[e] *= Dsm[e / TC];
    }
    cp_async_wait<0>();
    __syncthreads();  // pass q's operands and the previous pass's rows of X are in place
    stage(q + 1);     // the other slot was last read by pass q - 1
    const T* Lq = Ls + (size_t)(q & 1) * TB * LP;
    const T* Wq = Wsm + (size_t)(q & 1) * TB * LSP;
    // diagonal pass: X_J = W X_J (W = W_J forward, W_J^T backward), 4 x CPT per thread
    T* XJ = Xs + (size_t)J * TB * TC;
    T d[4][CPT] = {};
#pragma unroll 8
    for (int t = 0; t < TB; ++t) {
      T xv[CPT];
#pragma unroll
      for (int b = 0; b < CPT; ++b) xv[b] = XJ[t * TC + dc + b];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T w = Wq[(dr + a) * LSP + t];
#pragma unroll
        for (int b = 0; b < CPT; ++b) d[a][b] = fma(w, xv[b], d[a][b]);
      }
    }
    __syncthreads();  // every thread has read X_J
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < CPT; ++b) XJ[(dr + a) * TC + dc + b] = d[a][b];
    __syncthreads();
    // update pass: rows i0 .. i1 - 1 of X minus (staged rows t of L^T / L) x X_J
    const int i0 = fwd ? (J + 1) * TB : 0, i1 = fwd ? kp : J * TB;
    const int strips = (i1 - i0) / (RG * TR);
    for (int st = warp; st < strips; st += RL_NT / 32) {
      const int r0 = st * RG * TR + ug * TR;  // row offset within the updated range
      T acc[TR][4] = {};
#pragma unroll 4
      for (int t = 0; t < TB; ++t) {
        const Vec4<T> x = lds4(XJ + t * TC + uc);
#pragma unroll
        for (int h = 0; h < TR / 4; ++h) {
          const Vec4<T> l = lds4(Lq + t * LP + r0 + 4 * h);
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[4 * h + a][b] = fma(l.v[a], x.v[b], acc[4 * h + a][b]);
        }
      }
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        T* xr = Xs + (size_t)(i0 + r0 + a) * TC + uc;
        const Vec4<T> cur = lds4(xr);
        xr[0] = cur.v[0] - acc[a][0];
        xr[1] = cur.v[1] - acc[a][1];
        xr[2] = cur.v[2] - acc[a][2];
        xr[3] = cur.v[3] - acc[a][3];
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int e = tid; e < k * TC; e += RL_NT) {
    const int i = e / TC, c = e % TC;
    if (c0 + c < n) B[(int64_t)i * ldb + c0 + c] = Xs[e];
  }
}

template <typename T>
static size_t trsm_rl_smem_bytes(int kp, int tc) {
  return sizeof(T) * ((size_t)kp * tc + 2 * (size_t)TB * rl_lpad<T>(kp) + 2 * (size_t)TB * LSP +
                      (size_t)kp);
}

template <typename T, int TC, int TR = 8>
static int32_t trsm_rl_launch(const LdlOut<T>& o, const T* C, int64_t ldc, int64_t n, T* B,
                              int64_t ldb, cudaStream_t s) {
  const size_t bytes = trsm_rl_smem_bytes<T>(o.kp, TC);
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_trsm_rl<T, TC, TR>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  k_trsm_rl<T, TC, TR><<<(unsigned)ceil_div(n, TC), RL_NT, bytes, s>>>(o, C, ldc, n, B, ldb);
  return last_launch_status();
}

template <typename T>
static size_t trsm_smem_bytes(int kp, int tc) {
  return sizeof(T) * ((size_t)kp * tc + (size_t)TSTAGES * TB * LSP + 2 * (size_t)TB * tc);
}

template <typename T, int TC>
static int32_t trsm_launch(const LdlOut<T>& o, const T* C, int64_t ldc, int64_t n, T* B,
                           int64_t ldb, size_t bytes, cudaStream_t s) {
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_trsm_ldl<T, TC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  k_trsm_ldl<T, TC><<<(unsigned)ceil_div(n, TC), TB / 2 * TC / 4, bytes, s>>>(o, C, ldc, n, B,
                                                                              ldb);
  return last_launch_status();
}

template <typename T>
int32_t trsm_ldl(const LdlOut<T>& o, const T* C, int64_t ldc, int64_t n, T* B, int64_t ldb,
                 cudaStream_t s, bool narrow) {
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (!narrow && trsm_rl_smem_bytes<T>(o.kp, 64) <= (size_t)optin)
    return trsm_rl_launch<T, 64>(o, C, ldc, n, B, ldb, s);
  if (trsm_rl_smem_bytes<T>(o.kp, 32) <= (size_t)optin)
    return trsm_rl_launch<T, 32>(o, C, ldc, n, B, ldb, s);
  if (narrow && trsm_smem_bytes<T>(o.kp, 32) <= (size_t)optin)
    return trsm_launch<T, 32>(o, C, ldc, n, B, ldb, trsm_smem_bytes<T>(o.kp, 32), s);
  if (trsm_smem_bytes<T>(o.kp, 64) <= (size_t)optin)
    return trsm_launch<T, 64>(o, C, ldc, n, B, ldb, trsm_smem_bytes<T>(o.kp, 64), s);
  if (trsm_smem_bytes<T>(o.kp, 32) <= (size_t)optin)
    return trsm_launch<T, 32>(o, C, ldc, n, B, ldb, trsm_smem_bytes<T>(o.kp, 32), s);
  return RLU_EUNSUPPORTED;
}
template int32_t trsm_ldl<float>(const LdlOut<float>&, const float*, int64_t, int64_t, float*,
                                 int64_t, cudaStream_t, bool);
template int32_t trsm_ldl<double>(const LdlOut<double>&, const double*, int64_t, int64_t, double*,
                                  int64_t, cudaStream_t, bool);

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
template int32_t copy_cm<__nv_bfloat16>(const __nv_bfloat16*, int64_t, __nv_bfloat16*, int64_t,
                                        int64_t, int64_t, cudaStream_t);

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

// ---- batched launchers --------------------------------------------------------------------
// CTA (problem blockIdx.x, column group blockIdx.y): columns c = y, y + gridDim.y, ... of
// L_y / L~ (m rows each) in a loop, so that the grid holds no CTAs for the rows small
// problems do not have. The CTA first inverts the permutation in shared memory
// (pinv[perm[p]] = p), so that it walks the rows of L~ = P^T L_y (and of Y and the TF32
// split) in order: only the writes of L_y in pivot order are scattered.
__global__ void k_build_ly_batched(const BuildJob* __restrict__ jobs) {
  extern __shared__ int bl_pinv[];  // [m]
  const BuildJob& j = jobs[blockIdx.x];
  const int64_t m = j.m;
  const int k = j.k;
  // entries outside [0, m) (an LU that stopped early) leave -1 and are skipped
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) bl_pinv[r] = -1;
  __syncthreads();
  for (int64_t p = threadIdx.x; p < m; p += blockDim.x) {
    const int q = j.perm[p];
    if (q >= 0 && q < m) bl_pinv[q] = (int)p;
  }
  __syncthreads();
  for (int c = blockIdx.y; c < k; c += gridDim.y) {
#pragma unroll 4
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const int p = bl_pinv[r];
      if (p < 0) continue;
      const float v = (c < p) ? j.Y[(int64_t)c * j.ldy + r] : (c == p ? 1.f : 0.f);
      j.Lt[(int64_t)c * j.ldl + r] = v;
      if (j.Lhi) tf32_split(v, j.Lhi, j.Llo, (int64_t)c * j.ldl + r);
      j.Lp[(int64_t)c * j.ldl + p] = v;
    }
  }
}

int32_t build_ly_batched(const BuildJob* jobs_dev, int count, int64_t max_m, int max_k,
                         cudaStream_t s) {
  if (count <= 0) return RLU_OK;
  (void)max_k;
  const size_t smem = (size_t)max_m * sizeof(int);
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_build_ly_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_build_ly_batched<<<dim3((unsigned)count, 8), 256, smem, s>>>(jobs_dev);
  return last_launch_status();
}

// Gram M = L~^T L~ (k x k, FP64 out, FP32 accumulation) for k <= 64: one CTA per problem;
// thread t holds the 4 x 4 block (4 (t / 16), 4 (t % 16)) of M; 32-row chunks of L~ are
// staged row-major in shared memory.
static constexpr int GS_CHUNK = 32;
static constexpr int GS_KMAX = 64;
__global__ void __launch_bounds__(256) k_gram_small_batched(const GemmArgs* __restrict__ jobs) {
  __shared__ __align__(16) float S[GS_CHUNK][GS_KMAX + 4];
  const GemmArgs& g = jobs[blockIdx.x];
  const int k = (int)g.N;
  const int64_t m = g.K;
  const float* Lt = static_cast<const float*>(g.A);
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  const bool active = 4 * ti < k && 4 * tj < k;
  float acc[4][4] = {};
  constexpr int PER = GS_CHUNK * GS_KMAX / 256;  // staged values per thread and chunk
  float nxt[PER];                                // the next chunk, loaded ahead
  auto load_chunk = [&](int64_t r0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int c = e / GS_CHUNK, rr = e % GS_CHUNK;  // column c, row r0 + rr (coalesced in rr)
      nxt[u] = (c < k && r0 + rr < m) ? Lt[(int64_t)c * g.lda + r0 + rr] : 0.f;
    }
  };
  load_chunk(0);
  for (int64_t r0 = 0; r0 < m; r0 += GS_CHUNK) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + 256 * u;
      S[e % GS_CHUNK][e / GS_CHUNK] = nxt[u];
    }
    __syncthreads();
    if (r0 + GS_CHUNK < m) load_chunk(r0 + GS_CHUNK);
    if (active) {
#pragma unroll 8
      for (int rr = 0; rr < GS_CHUNK; ++rr) {
        const float4 a = *reinterpret_cast<const float4*>(&S[rr][4 * ti]);
        const float4 b = *reinterpret_cast<const float4*>(&S[rr][4 * tj]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
      }
    }
  }
  if (!active) return;
  double* M = static_cast<double*>(g.C);
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = 4 * ti + x, jj = 4 * tj + y;
      if (i < k && jj < k) M[(int64_t)i * g.ldc + jj] = (double)acc[x][y];
    }
}

int32_t gram_small_batched(const GemmArgs* jobs_dev, int count, cudaStream_t s) {
  if (count <= 0) return RLU_OK;
  k_gram_small_batched<<<(unsigned)count, 256, 0, s>>>(jobs_dev);
  return last_launch_status();
}

int32_t ldl32_batched(const Ldl32Job* jobs_dev, int count, int max_k, cudaStream_t s) {
  if (count <= 0) return RLU_OK;
  if (max_k > L32_MAXB * LB) return RLU_EUNSUPPORTED;
  const size_t bytes = ldl32_smem_bytes(max_k);
  if (max_k <= 4 * LB) {
    RLU_CUDA_TRY(cudaFuncSetAttribute(k_ldl32_batched<128>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k_ldl32_batched<128><<<(unsigned)count, 128, bytes, s>>>(jobs_dev);
  } else {
    RLU_CUDA_TRY(cudaFuncSetAttribute(k_ldl32_batched<L32_NT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k_ldl32_batched<L32_NT><<<(unsigned)count, L32_NT, bytes, s>>>(jobs_dev);
  }
  return last_launch_status();
}

// Batched form for k <= 64: one thread per column of C over a tile list of (problem,
// 128-column block) entries. L (unit lower, from LR) sits in shared memory, zero-padded to
// the problem's bucket KB in {16, 32, 48, 64} (padded rows and columns change nothing), and
// the column in registers: forward substitution x_i -= sum_{j<i} L[i][j] x_j, scaling by
// 1/D, backward substitution x_i -= sum_{j>i} L[j][i] x_j. The bucket is chosen per CTA from
// its problem's k, so small problems do not pay for the largest k of the batch.
static constexpr int TS_KMAX = 64;
static constexpr int TS_LD = TS_KMAX + 4;  // 16-byte rows
static constexpr int TS_COLS = 128;

template <int KB>
__device__ __forceinline__ void trsm_small_body(const float (*Ls)[TS_LD], const float* dv,
                                                const float* __restrict__ C, int64_t ldc,
                                                float* __restrict__ B, int64_t ldb, int k,
                                                int64_t c) {
  float x[KB];
#pragma unroll
  for (int i = 0; i < KB; ++i) x[i] = i < k ? C[(int64_t)i * ldc + c] : 0.f;
#pragma unroll
  for (int i = 1; i < KB; ++i) {
    if (i < k) {
      float acc = x[i];
#pragma unroll
      for (int j = 0; j < i; ++j) acc = fmaf(-Ls[i][j], x[j], acc);
      x[i] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < KB; ++i) x[i] *= dv[i];
#pragma unroll
  for (int i = KB - 2; i >= 0; --i) {
    if (i < k - 1) {
      float acc = x[i];
#pragma unroll
      for (int j = i + 1; j < KB; ++j)
        if (j < k) acc = fmaf(-Ls[j][i], x[j], acc);
      x[i] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < KB; ++i)
    if (i < k) B[(int64_t)i * ldb + c] = x[i];
}

template <int KB>
__global__ void __launch_bounds__(TS_COLS) k_trsm_small_batched(const TrsmJob* __restrict__ jobs,
                                                                const int2* __restrict__ tiles) {
  __shared__ __align__(16) float Ls[TS_KMAX][TS_LD];
  __shared__ float dv[TS_KMAX];
  const int2 t = tiles[blockIdx.x];
  const TrsmJob& jb = jobs[t.x];
  const int k = jb.o.k, kp = jb.o.kp;
  for (int e = threadIdx.x; e < KB * KB; e += TS_COLS) {
    const int i = e / KB, j = e % KB;
    Ls[i][j] = (i < k && j < k) ? jb.o.LR[(int64_t)i * kp + j] : 0.f;
  }
  for (int i = threadIdx.x; i < KB; i += TS_COLS) dv[i] = i < k ? (float)jb.o.dinv[i] : 0.f;
  __syncthreads();
  const int64_t c = (int64_t)t.y * TS_COLS + threadIdx.x;
  if (c >= jb.n) return;
  trsm_small_body<KB>(Ls, dv, jb.C, jb.ldc, jb.B, jb.ldb, k, c);
}

int trsm_small_bucket(int k) { return k <= 16 ? 0 : k <= 32 ? 1 : k <= 48 ? 2 : 3; }

int32_t trsm_small_batched(const TrsmJob* jobs_dev, const int2* tiles_dev, const int* first,
                           const int* count, cudaStream_t s) {
  int launches = 0;
  for (int bkt = 0; bkt < 4; ++bkt) {
    if (count[bkt] <= 0) continue;
    const int2* tl = tiles_dev + first[bkt];
    const unsigned g = (unsigned)count[bkt];
    if (bkt == 0) k_trsm_small_batched<16><<<g, TS_COLS, 0, s>>>(jobs_dev, tl);
    else if (bkt == 1) k_trsm_small_batched<32><<<g, TS_COLS, 0, s>>>(jobs_dev, tl);
    else if (bkt == 2) k_trsm_small_batched<48><<<g, TS_COLS, 0, s>>>(jobs_dev, tl);
    else k_trsm_small_batched<64><<<g, TS_COLS, 0, s>>>(jobs_dev, tl);
    ++launches;
  }
  return launches ? last_launch_status(launches) : RLU_OK;
}

// L (m x k, column-major) = L_y (m x k, column-major, pivot order) L_b (k x k, column-major,
// unit lower) for k <= 64: one thread per row over a tile list of (problem, 256-row block)
// entries, L_b (zero-padded to the problem's bucket KB) in shared memory, the row of L_y in
// registers.
static constexpr int LM_ROWS = 256;

template <int KB>
__device__ __forceinline__ void lmul_body(const float* Lbs, const float* __restrict__ Ly,
                                          int64_t lda, float* __restrict__ L, int64_t ldc,
                                          int k, int64_t i) {
  float y[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) y[c] = c < k ? Ly[(int64_t)c * lda + i] : 0.f;
  for (int j = 0; j < k; ++j) {
    const float* bcol = Lbs + j * TS_LD;  // column j of L_b
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < KB; c += 4) {
      const float4 b4 = *reinterpret_cast<const float4*>(bcol + c);
      acc = fmaf(y[c], b4.x, acc);
      acc = fmaf(y[c + 1], b4.y, acc);
      acc = fmaf(y[c + 2], b4.z, acc);
      acc = fmaf(y[c + 3], b4.w, acc);
    }
    L[(int64_t)j * ldc + i] = acc;
  }
}

__global__ void __launch_bounds__(LM_ROWS) k_lmul_batched(const GemmArgs* __restrict__ jobs,
                                                          const int2* __restrict__ tiles) {
  __shared__ __align__(16) float Lbs[TS_KMAX * TS_LD];
  const int2 t = tiles[blockIdx.x];
  const GemmArgs& g = jobs[t.x];
  const int k = (int)g.N;
  const int kb = k <= 16 ? 16 : k <= 32 ? 32 : k <= 48 ? 48 : 64;
  const float* Lb = static_cast<const float*>(g.B);
  for (int e = threadIdx.x; e < k * kb; e += LM_ROWS) {
    const int j = e / kb, c = e % kb;  // column j, entry c
    Lbs[j * TS_LD + c] = c < k ? Lb[(int64_t)j * g.ldb + c] : 0.f;
  }
  __syncthreads();
  const int64_t i = (int64_t)t.y * LM_ROWS + threadIdx.x;
  if (i >= g.M) return;
  const float* Ly = static_cast<const float*>(g.A);
  float* L = static_cast<float*>(g.C);
  if (kb == 16) lmul_body<16>(Lbs, Ly, g.lda, L, g.ldc, k, i);
  else if (kb == 32) lmul_body<32>(Lbs, Ly, g.lda, L, g.ldc, k, i);
  else if (kb == 48) lmul_body<48>(Lbs, Ly, g.lda, L, g.ldc, k, i);
  else lmul_body<64>(Lbs, Ly, g.lda, L, g.ldc, k, i);
}

int32_t lmul_batched(const GemmArgs* jobs_dev, const int2* tiles_dev, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return RLU_OK;
  k_lmul_batched<<<(unsigned)ntiles, LM_ROWS, 0, s>>>(jobs_dev, tiles_dev);
  return last_launch_status();
}

int32_t trsm_batched(const TrsmJob* jobs_dev, const int2* tiles_dev, int ntiles, int max_kp,
                     cudaStream_t s) {
  if (ntiles <= 0) return RLU_OK;
  const size_t bytes = trsm_smem_bytes<float>(max_kp, 64);
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (bytes > (size_t)optin) return RLU_EUNSUPPORTED;
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_trsm_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes));
  k_trsm_batched<<<(unsigned)ntiles, TB / 2 * 64 / 4, bytes, s>>>(jobs_dev, tiles_dev);
  return last_launch_status();
}

// One CTA per problem: U (k rows of n) and L_b (k x k) in loops.
__global__ void k_gather_batched(const GatherJob* __restrict__ jobs) {
  const GatherJob& j = jobs[blockIdx.x];
  const int k = j.k;
  const int64_t n = j.n;
  for (int i = 0; i < k; ++i) {
#pragma unroll 4
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x)
      j.U[(int64_t)i * j.ldu + c] = c >= i ? j.B[(int64_t)i * j.ldb + j.Q[c]] : 0.f;
    // L_b column i: rows r > i from B's row r at the pivot column Q[i]
    for (int r = threadIdx.x; r < k; r += blockDim.x)
      j.Lb[(int64_t)i * k + r] = r > i ? j.B[(int64_t)r * j.ldb + j.Q[i]] : (r == i ? 1.f : 0.f);
  }
}

int32_t gather_batched(const GatherJob* jobs_dev, int count, int max_k, int64_t max_n,
                       cudaStream_t s) {
  if (count <= 0) return RLU_OK;
  (void)max_k;
  (void)max_n;
  k_gather_batched<<<(unsigned)count, 256, 0, s>>>(jobs_dev);
  return last_launch_status();
}

}  // namespace rlu
