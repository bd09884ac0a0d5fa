// Algorithm 2 (alg:randomized_orth, Section 4.3) on the GPU, in FP64: the randomized range
// finder with an orthogonal basis that Section 5 uses as the accuracy comparator of the
// randomized LU (the "randomized SVD" of its error experiment).
//
//   step 1  G = gaussian(seed)                       gauss.cu (the generator of Algorithm 1)
//   step 2  Y = A G                                  gemm_simt.cu
//   step 3  the left singular vectors of Y, from the eigenpairs of M = Y^T Y (FP64 Gram):
//           M = V diag(lambda) V^T by cyclic Jacobi (k_jacobi_sym, below), then
//           U_y = Y V diag(lambda)^{-1/2}
//   step 4  Q = the k columns of U_y with the largest lambda: Q = Y W with
//           W = V_k diag(lambda_k)^{-1/2} (k_jacobi_select, gemm_simt.cu)
//   and B = Q^T A, so that Q B = Q Q^T A is the rank-k approximation whose error
//   ||Q Q^T A - A|| Section 5 compares with the randomized LU's.
//
// The Jacobi eigensolver (parallel two-sided Jacobi): the l x l matrix (l rounded up to an
// even l2; a padding index stays decoupled) is swept by the round-robin (circle) schedule:
// each round pairs every index with one other, and the l2 / 2 rotations of a round commute,
// so M <- J^T M J updates every 2 x 2 block (pair i, pair j) independently from the old
// values: M and V are double buffered and a round costs one grid barrier. Every CTA computes
// the round's rotations itself (3 reads each) into shared memory. A pair is rotated while
// |m_pq| > 1e-15 sqrt(|m_pp m_qq|); the sweeps stop after one without rotations (or 30).
// The barrier is a counter in global memory whose waits give up after 2 s (RLU_ETIMEOUT).
#include <cooperative_groups.h>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "small.cuh"

namespace rlu {

int32_t launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, int64_t l, int32_t dtype,
                        void* G, int64_t ldg, cudaStream_t s);

static constexpr int JAC_T = 256;
static constexpr int JAC_MAX_SWEEPS = 30;

struct JacArgs {
  double* M0;        // l2 x l2 row-major (symmetric), the Gram matrix on entry
  double* M1;
  double* V0;        // l2 x l2 column-major, the identity on entry
  double* V1;
  int l2;
  unsigned* bar;     // grid barrier counter (zero on entry)
  unsigned* nrot;    // [JAC_MAX_SWEEPS] rotations per sweep (zero on entry)
  int* result;       // [0] buffer holding the result, [1] sweeps run
  int32_t* status;
};

__device__ __forceinline__ unsigned jac_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t jac_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// Every CTA's writes so far, then wait until all gridDim.x CTAs arrived for the n-th time.
__device__ bool jac_barrier(unsigned* bar, unsigned n, int32_t* status, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = n * gridDim.x;
    bool ok = true;
    if (jac_ld_acquire(bar) < target) {
      const uint64_t t0 = jac_now();
      while (jac_ld_acquire(bar) < target)
        if (jac_now() - t0 > 2000000000ull) {
          ok = false;
          break;
        }
    }
    __threadfence();
    if (!ok && status) atomicExch(status, RLU_ETIMEOUT);
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Pair i of round r of the circle schedule for l2 players: player 0 is fixed, players
// 1..l2-1 rotate; (p, q) with p < q.
__device__ __forceinline__ void jac_pair(int i, int r, int l2, int& p, int& q) {
  const int n1 = l2 - 1;
  int a, b;
  if (i == 0) {
    a = 0;
    b = 1 + (r % n1);
  } else {
    a = 1 + ((i + r) % n1);
    b = 1 + ((n1 - i + r) % n1);
  }
  p = min(a, b);
  q = max(a, b);
}

__global__ void __launch_bounds__(JAC_T) k_jacobi_sym(JacArgs a) {
  extern __shared__ __align__(16) unsigned char jac_smem[];
  const int l2 = a.l2, P = l2 / 2;
  double2* cs = reinterpret_cast<double2*>(jac_smem);       // [P] (c, s)
  int2* pq = reinterpret_cast<int2*>(cs + P);                // [P] (p, q)
  __shared__ int s_ok, s_cnt;
  unsigned nbar = 0;
  int buf = 0, sweep = 0;
  const int64_t gthreads = (int64_t)gridDim.x * JAC_T;
  const int64_t gtid = (int64_t)blockIdx.x * JAC_T + threadIdx.x;
  bool alive = true;
  for (sweep = 0; sweep < JAC_MAX_SWEEPS && alive; ++sweep) {
    for (int r = 0; r < l2 - 1 && alive; ++r) {
      const double* Mc = buf ? a.M1 : a.M0;
      double* Mn = buf ? a.M0 : a.M1;
      const double* Vc = buf ? a.V1 : a.V0;
      double* Vn = buf ? a.V0 : a.V1;
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
      int cnt = 0;
      for (int i = threadIdx.x; i < P; i += JAC_T) {
        int p, q;
        jac_pair(i, r, l2, p, q);
        const double app = Mc[(int64_t)p * l2 + p], aqq = Mc[(int64_t)q * l2 + q];
        const double apq = Mc[(int64_t)p * l2 + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-15 * sqrt(fabs(app) * fabs(aqq)) && apq != 0.0) {
          // t = tan(phi), the smaller root of t^2 + 2 theta t - 1 = 0, zeroes m'_pq
          const double theta = (aqq - app) / (2.0 * apq);
          const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
          ++cnt;
        }
        cs[i] = make_double2(c, s);
        pq[i] = make_int2(p, q);
      }
      if (blockIdx.x == 0 && cnt) atomicAdd(&s_cnt, cnt);
      __syncthreads();
      if (blockIdx.x == 0 && threadIdx.x == 0 && s_cnt) atomicAdd(&a.nrot[sweep], (unsigned)s_cnt);
      // M' = J^T M J, block (pair i, pair j) by block
      for (int64_t it = gtid; it < (int64_t)P * P; it += gthreads) {
        const int i = (int)(it / P), j = (int)(it % P);
        const double2 ri = cs[i], rj = cs[j];
        const int pi = pq[i].x, qi = pq[i].y, pj = pq[j].x, qj = pq[j].y;
        const double x00 = Mc[(int64_t)pi * l2 + pj], x01 = Mc[(int64_t)pi * l2 + qj];
        const double x10 = Mc[(int64_t)qi * l2 + pj], x11 = Mc[(int64_t)qi * l2 + qj];
        // columns: p <- c x_p - s x_q, q <- s x_p + c x_q
        const double y00 = rj.x * x00 - rj.y * x01, y01 = rj.y * x00 + rj.x * x01;
        const double y10 = rj.x * x10 - rj.y * x11, y11 = rj.y * x10 + rj.x * x11;
        // rows, the same rotation of pair i
        double z00 = ri.x * y00 - ri.y * y10, z10 = ri.y * y00 + ri.x * y10;
        double z01 = ri.x * y01 - ri.y * y11, z11 = ri.y * y01 + ri.x * y11;
        if (i == j && ri.y != 0.0) {  // the annihilated pair
          z01 = 0.0;
          z10 = 0.0;
        }
        Mn[(int64_t)pi * l2 + pj] = z00;
        Mn[(int64_t)pi * l2 + qj] = z01;
        Mn[(int64_t)qi * l2 + pj] = z10;
        Mn[(int64_t)qi * l2 + qj] = z11;
      }
      // V' = V J: the columns of each pair
      for (int64_t it = gtid; it < (int64_t)P * l2; it += gthreads) {
        const int j = (int)(it / l2), row = (int)(it % l2);
        const double2 rj = cs[j];
        const int pj = pq[j].x, qj = pq[j].y;
        const double vp = Vc[(int64_t)pj * l2 + row], vq = Vc[(int64_t)qj * l2 + row];
        Vn[(int64_t)pj * l2 + row] = rj.x * vp - rj.y * vq;
        Vn[(int64_t)qj * l2 + row] = rj.y * vp + rj.x * vq;
      }
      buf ^= 1;
      alive = jac_barrier(a.bar, ++nbar, a.status, &s_ok);
    }
    if (alive && jac_ld_acquire(&a.nrot[sweep]) == 0u) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.result[0] = buf;
    a.result[1] = sweep;
  }
}

// M (l x l FP64, row-major, ld l2) padded to l2 with a decoupled unit entry; V = I (l2 x l2).
__global__ void k_jacobi_init(double* M, double* V, int l, int l2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)l2 * l2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / l2), c = (int)(e % l2);
    V[e] = r == c ? 1.0 : 0.0;
    if (r >= l || c >= l) M[e] = (r == c) ? 1.0 : 0.0;
  }
}

// Ranks the eigenvalues lambda_j = M[j][j] (j < l) in decreasing order (ties by index):
// sigma[rank] = sqrt(lambda), and for rank < k, W[:, rank] = V[:l, j] / sqrt(lambda). An
// eigenvalue at or below 64 eps lambda_max is rounding noise of the Gram matrix (singular
// values of Y below about 1e-7 sigma_1 are not resolved by this route): its sigma is 0 and,
// for rank < k, its column of W is zero and status is RLU_EINVAL.
__global__ void k_jacobi_select(const double* M, const double* V, const int* result, int l,
                                int l2, int k, double* W, int64_t ldw, double* sigma,
                                int32_t* status) {
  const double* Mf = result[0] ? M + (int64_t)l2 * l2 : M;
  const double* Vf = result[0] ? V + (int64_t)l2 * l2 : V;
  __shared__ double s_max;
  __shared__ int s_rank;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < l; ++i) mx = fmax(mx, Mf[(int64_t)i * l2 + i]);
    s_max = mx;
  }
  __syncthreads();
  const double floor_ = 64.0 * 2.220446049250313e-16 * s_max;
  for (int j = blockIdx.x; j < l; j += gridDim.x) {
    const double lj_raw = Mf[(int64_t)j * l2 + j];
    const double lj = lj_raw > floor_ ? lj_raw : 0.0;
    if (threadIdx.x == 0) s_rank = 0;
    __syncthreads();
    int cnt = 0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
      const double li = Mf[(int64_t)i * l2 + i];
      if (li > lj_raw || (li == lj_raw && i < j)) ++cnt;
    }
    atomicAdd(&s_rank, cnt);
    __syncthreads();
    const int rank = s_rank;
    if (threadIdx.x == 0 && sigma) sigma[rank] = sqrt(lj > 0.0 ? lj : 0.0);
    if (rank < k) {
      const double inv = lj > 0.0 ? 1.0 / sqrt(lj) : 0.0;
      if (lj <= 0.0 && threadIdx.x == 0 && status) atomicExch(status, RLU_EINVAL);
      for (int r = threadIdx.x; r < l; r += blockDim.x)
        W[(int64_t)rank * ldw + r] = Vf[(int64_t)j * l2 + r] * inv;
    }
    __syncthreads();
  }
}

struct RsvdPlan {
  int64_t m = 0, n = 0;
  int k = 0, l = 0, l2 = 0;
  int64_t ldg = 0, ldy = 0, ldw = 0;
  int split_y = 1, split_g = 1, split_q = 1, split_b = 1;
  size_t off_G = 0, off_Y = 0, off_M = 0, off_V = 0, off_W = 0, off_hdr = 0, off_part = 0,
         total = 0;
};

static size_t rs_carve(size_t& cur, size_t bytes) {
  const size_t at = cur;
  cur += (size_t)round_up((int64_t)bytes, 256);
  return at;
}

static int rs_split(int64_t M, int64_t N, int64_t K) {
  const int bm = gemm_tile_m(RLU_F64), bn = gemm_tile_n(RLU_F64);
  const int64_t tiles = ceil_div(M, bm) * ceil_div(N, bn);
  int64_t s = ceil_div(2 * (int64_t)sm_count(), tiles);
  const int64_t kmax = K / 64 > 1 ? K / 64 : 1;
  return (int)(s < 1 ? 1 : (s > kmax ? kmax : s));
}

static bool rsvd_plan(int64_t m, int64_t n, int k, int l, RsvdPlan& p) {
  if (!(k >= 1 && k <= l && l <= m && l <= n) || l > 4096) return false;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return false;
  p.m = m; p.n = n; p.k = k; p.l = l;
  p.l2 = l + (l & 1);
  if (p.l2 < 2) p.l2 = 2;
  p.ldg = round_up(n, 8);
  p.ldy = round_up(m, 8);
  p.ldw = l;
  p.split_y = rs_split(m, l, n);
  p.split_g = rs_split(l, l, m);
  p.split_q = rs_split(m, k, l);
  p.split_b = rs_split(k, n, m);
  size_t part = 0;
  auto upd = [&](size_t b) { part = b > part ? b : part; };
  upd(gemm_partial_bytes<double>(m, l, p.split_y));
  upd(gemm_partial_bytes<double>(l, l, p.split_g));
  upd(gemm_partial_bytes<double>(m, k, p.split_q));
  upd(gemm_partial_bytes<double>(k, n, p.split_b));
  size_t cur = 0;
  p.off_G = rs_carve(cur, (size_t)p.ldg * l * 8);
  p.off_Y = rs_carve(cur, (size_t)p.ldy * l * 8);
  p.off_M = rs_carve(cur, 2 * (size_t)p.l2 * p.l2 * 8);
  p.off_V = rs_carve(cur, 2 * (size_t)p.l2 * p.l2 * 8);
  p.off_W = rs_carve(cur, (size_t)l * k * 8);
  p.off_hdr = rs_carve(cur, 512);  // barrier, rotation counts, result
  p.off_part = rs_carve(cur, part);
  p.total = cur;
  return true;
}

}  // namespace rlu

using namespace rlu;

extern "C" size_t rlu_rsvd_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l) {
  RsvdPlan p;
  return rsvd_plan(m, n, k, l, p) ? p.total : 0;
}

extern "C" int32_t rlu_rsvd(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                            int32_t k, int32_t l, uint64_t seed, void* Q, int64_t ldq, void* B,
                            int64_t ldb, double* sigma, rlu_info* info, void* workspace,
                            size_t ws_bytes, void* stream) {
  if (!A || !Q || !B) return RLU_EINVAL;
  if (dtype != RLU_F64) return RLU_EUNSUPPORTED;
  if (m < 1 || n < 1 || lda < n || ldq < m || ldb < n) return RLU_EINVAL;
  RsvdPlan p;
  if (!rsvd_plan(m, n, k, l, p)) return RLU_EINVAL;
  if (workspace == nullptr || ws_bytes < p.total) return RLU_ENOMEM;
  if (((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = static_cast<char*>(workspace);
  double* G = reinterpret_cast<double*>(ws + p.off_G);
  double* Y = reinterpret_cast<double*>(ws + p.off_Y);
  double* M = reinterpret_cast<double*>(ws + p.off_M);
  double* V = reinterpret_cast<double*>(ws + p.off_V);
  double* W = reinterpret_cast<double*>(ws + p.off_W);
  unsigned* hdr = reinterpret_cast<unsigned*>(ws + p.off_hdr);
  void* part = ws + p.off_part;
  const double* Ad = static_cast<const double*>(A);
  const int l2 = p.l2;
  int32_t* status = info ? &info->status : nullptr;
  if (info) RLU_TRY(info_init(info, s));
  // steps 1-2
  RLU_TRY(launch_gaussian(seed, 0, n, l, RLU_F64, G, p.ldg, s));
  {
    GemmOp op{Ad, lda, true, G, p.ldg, true, Y, p.ldy, false, m, l, n, p.split_y, part, false};
    RLU_TRY((gemm_simt<double, double>(op, s)));
  }
  // step 3: M = Y^T Y (l x l, ld l2), then its eigenpairs
  {
    GemmOp op{Y, p.ldy, true, Y, p.ldy, true, M, l2, true, l, l, m, p.split_g, part, false};
    RLU_TRY((gemm_simt<double, double>(op, s)));
  }
  k_jacobi_init<<<(unsigned)ceil_div((int64_t)l2 * l2, 256) > 1024 ? 1024
                      : (unsigned)ceil_div((int64_t)l2 * l2, 256), 256, 0, s>>>(M, V, l, l2);
  RLU_TRY(last_launch_status());
  RLU_CUDA_TRY(cudaMemsetAsync(hdr, 0, 512, s));
  JacArgs ja{};
  ja.M0 = M;
  ja.M1 = M + (size_t)l2 * l2;
  ja.V0 = V;
  ja.V1 = V + (size_t)l2 * l2;
  ja.l2 = l2;
  ja.bar = hdr;
  ja.nrot = hdr + 32;
  ja.result = reinterpret_cast<int*>(hdr + 96);
  ja.status = status;
  {
    const int P = l2 / 2;
    const size_t smem = (size_t)P * (sizeof(double2) + sizeof(int2));
    const void* fn = reinterpret_cast<const void*>(&k_jacobi_sym);
    RLU_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, JAC_T, smem));
    if (per_sm < 1) return RLU_EUNSUPPORTED;
    int64_t want = ceil_div((int64_t)P * (P > l2 ? P : l2), 4 * JAC_T);
    int grid = (int)(want < 1 ? 1 : (want > sm_count() ? sm_count() : want));
    void* args[] = {&ja};
    RLU_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(JAC_T), args, smem, s));
    RLU_TRY(last_launch_status());
  }
  // step 4: W = V_k diag(lambda_k)^{-1/2}, Q = Y W, B = Q^T A
  k_jacobi_select<<<(unsigned)(l < 1024 ? l : 1024), 128, 0, s>>>(M, V, ja.result, l, l2, k, W,
                                                                 p.ldw, sigma, status);
  RLU_TRY(last_launch_status());
  {
    GemmOp op{Y, p.ldy, false, W, p.ldw, true, Q, ldq, false, m, k, l, p.split_q, part, false};
    RLU_TRY((gemm_simt<double, double>(op, s)));
  }
  {
    GemmOp op{Q, ldq, true, Ad, lda, false, B, ldb, true, k, n, m, p.split_b, part, false};
    RLU_TRY((gemm_simt<double, double>(op, s)));
  }
  return RLU_OK;
}
