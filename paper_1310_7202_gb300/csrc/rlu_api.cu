// C ABI and host orchestration of Algorithm 1 (randomized LU) on one GB300.
//
// rlu_factor enqueues, on the caller's stream:
//   step 1  G = gaussian(seed)                                   gauss.cu
//   step 2  Y = A G                                              gemm_simt.cu
//   step 3  P Y = L_y U_y, partial pivoting, all l steps        panel_lu.cu (Doolittle)
//   step 4  L_y = first k columns; L~ = P^T L_y                  small.cu build_ly
//   step 5  M = L~^T L~ (FP64 sum of partial products); fork: R = chol(M), R^{-1} on a
//           helper stream while C = L~^T A runs; join; B = R^{-1} (R^{-T} C)
//   step 6  B Q = L_b U_b, column pivoting (LU of B^T)           panel_lu.cu (Crout)
//   step 7  L = L_y L_b                                          gemm_simt.cu
//   step 8  U = U_b                                              small.cu gather_lb_u
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "panel_lu.cuh"
#include "residual.cuh"
#include "small.cuh"
#include "umma.cuh"

namespace rlu {

int32_t launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, int64_t l, int32_t dtype,
                        void* G, int64_t ldg, cudaStream_t s);

static std::atomic<uint64_t> g_launches{0};
void note_launches(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

static const char* kStepNames[RLU_NUM_TIMED_STEPS] = {
    "gaussian", "gemm_Y", "lu_Y", "build_Ly", "gram", "ldl", "gemm_C", "trsm_B", "lu_B",
    "gather_Lb_U", "gemm_L"};

// Records the start/end event of timed step i when the caller asked for events.
struct StepTimer {
  const rlu_stage_outputs* st;
  int32_t rec(int i, bool end, cudaStream_t s) const {
    if (!st || !st->events || st->n_events < 2 * RLU_NUM_TIMED_STEPS) return RLU_OK;
    RLU_CUDA_TRY(cudaEventRecord((cudaEvent_t)st->events[2 * i + (end ? 1 : 0)], s));
    return RLU_OK;
  }
};

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int n = 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

// Helper stream and fork/join events of one caller stream on one device (created on first
// use), so that concurrent factorizations on different streams keep separate helpers.
struct SideStream {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::mutex mu;
};

static int32_t side_stream(cudaStream_t main, SideStream** out) {
  static std::mutex table_mu;
  static std::map<std::pair<int, cudaStream_t>, SideStream*> table;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  SideStream* ss = nullptr;
  {
    std::lock_guard<std::mutex> lock(table_mu);
    SideStream*& slot = table[{dev, main}];
    if (slot == nullptr) slot = new SideStream();
    ss = slot;
  }
  std::lock_guard<std::mutex> lock(ss->mu);
  if (ss->side == nullptr) {
    // highest priority: the factorization's CTA(s) must get their SMs before the
    // concurrent GEMM fills the GPU, otherwise they only start when that GEMM drains
    int lo = 0, hi = 0;
    RLU_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    RLU_CUDA_TRY(cudaStreamCreateWithPriority(&ss->side, cudaStreamNonBlocking, hi));
    RLU_CUDA_TRY(cudaEventCreateWithFlags(&ss->fork, cudaEventDisableTiming));
    RLU_CUDA_TRY(cudaEventCreateWithFlags(&ss->join, cudaEventDisableTiming));
  }
  *out = ss;
  return RLU_OK;
}

static int split_for(int64_t M, int64_t N, int64_t K, int bm, int bn, int kmin = 64) {
  const int64_t tiles = ceil_div(M, bm) * ceil_div(N, bn);
  const int64_t target = 2 * (int64_t)sm_count();
  int64_t s = ceil_div(target, tiles);
  const int64_t kmax = K / kmin > 1 ? K / kmin : 1;  // at least kmin of K per split
  if (s > kmax) s = kmax;
  if (s < 1) s = 1;
  return (int)s;
}

// Workspace layout of rlu_factor for one size / precision.
struct Plan {
  int32_t prec = RLU_PREC_F32;
  int32_t dt = RLU_F32;
  size_t esz = 4;
  int64_t m = 0, n = 0;
  int k = 0, l = 0;
  int64_t ldg = 0, ldy = 0, ldl = 0, ldb = 0, ldu12 = 0;
  int split_y = 1, split_g = 1, split_c = 1;
  int q = 0;                      // power iterations (Section 5)
  bool normalized = false;        // LU-normalised rounds
  int split_z = 1, split_y3 = 1;  // their products Z = A^T Y and Y = A Z
  size_t off_Ln = 0;              // the normalised block (FP64 / plain FP32 paths)
  // FP8 projection: e4m3 A and G with their UE8M0 scales
  size_t off_A8 = 0, off_SA = 0, off_G8 = 0, off_SG = 0;
  int64_t ld8 = 0, lds = 0, lsg = 0;
  size_t off_Z = 0, off_Yh = 0, off_Yl = 0, off_Zh = 0, off_Zl = 0, off_Yb[3] = {0, 0, 0},
         off_Zb[3] = {0, 0, 0};
  size_t off_Lbh = 0, off_Lbl = 0;  // TF32 split of L_b (k x k, ld round_up(k, 4))
  size_t off_G = 0, off_Y = 0, off_Lt = 0, off_Lp = 0, off_M = 0, off_dinv = 0, off_LT = 0,
         off_LR = 0, off_W = 0, off_WT = 0,
         off_C = 0, off_T = 0, off_B = 0, off_Lb = 0, off_part = 0, off_Lhi = 0, off_Llo = 0,
         off_pos = 0, off_ps = 0, off_u12 = 0, off_u12t = 0, off_Bh = 0, off_Bm = 0, off_Bl = 0, total = 0;
};

static size_t carve(size_t& cur, size_t bytes) {
  const size_t at = cur;
  cur += (size_t)round_up((int64_t)bytes, 256);
  return at;
}

static bool make_plan(int64_t m, int64_t n, int k, int l, int32_t prec, Plan& p, int q = 0,
                      bool normalized = false) {
  p.prec = prec;
  if (q < 0 || q > 16) return false;
  p.q = q;
  p.normalized = normalized && q > 0;
  if (prec == RLU_PREC_F64) {
    p.dt = RLU_F64;
    p.esz = 8;
  } else if (prec == RLU_PREC_F32 || prec == RLU_PREC_MIXED || prec == RLU_PREC_BF16 ||
             prec == RLU_PREC_FP8) {
    p.dt = RLU_F32;  // the path's type: Y, L~, the LUs, L and U (A may be BF16)
    p.esz = 4;
  } else {
    return false;
  }
  if (!(k >= 1 && k <= l && l <= m && l <= n)) return false;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return false;
  p.m = m; p.n = n; p.k = k; p.l = l;
  p.ldg = round_up(n, 8);
  p.ldy = round_up(m, 8);
  p.ldl = round_up(m, 8);
  p.ldb = round_up(n, 8);
  const int bm = gemm_tile_m(p.dt), bn = gemm_tile_n(p.dt);
  // FP64: a few tiles of FP64 multiply-adds (1/64 of the FP32 rate) would leave most SMs'
  // FP64 units idle, so split K down to one 16-deep k-step per split
  const int kmin = p.dt == RLU_F64 ? 16 : 64;
  p.split_y = split_for(m, l, n, bm, bn, kmin);
  if (prec == RLU_PREC_MIXED) {  // tensor-core products: 128-row tiles, split-K fills the SMs
    p.split_y = umma3_splits(m, n, l);
  }
  if (prec == RLU_PREC_BF16) p.split_y = umma_bf16_splits(m, n, l, 256);
  if (prec == RLU_PREC_FP8) p.split_y = umma_fp8_splits(m, n, l);
  const bool bf16_like = prec == RLU_PREC_BF16 || prec == RLU_PREC_FP8;
  p.split_g = split_for(k, k, m, bm, bn, kmin);
  if (p.dt == RLU_F32 && p.split_g < 2) p.split_g = 2;  // FP32 partials, FP64 reduction
  p.split_c = split_for(k, n, m, bm, bn, kmin);
  if (prec == RLU_PREC_MIXED || bf16_like) {
    p.split_g = umma3_splits(k, m, k);
    p.split_c = umma3_splits(n, m, k);
  }
  if (bf16_like) p.split_c = umma_bf16_splits(k, m, n, 256);
  // power iterations: Z = A^T Y (as C, with l columns of Y) and Y = A Z (as Y)
  p.split_z = split_for(l, n, m, bm, bn);
  p.split_y3 = p.split_y;
  if (prec == RLU_PREC_MIXED) p.split_z = umma3_splits(n, m, l);
  if (bf16_like) {
    p.split_z = umma_bf16_splits(l, m, n, 256);
    p.split_y3 = umma_bf16_splits(m, n, l, 128);
  }
  size_t part = 0;
  auto upd = [&](size_t b) { part = b > part ? b : part; };
  if (q > 0) {
    if (p.split_z > 1) upd((size_t)p.split_z * l * n * p.esz);
    if (p.split_y3 > 1) upd((size_t)p.split_y3 * m * l * p.esz);
  }
  if (p.split_y > 1) upd((size_t)p.split_y * m * l * p.esz);
  upd((size_t)(p.split_g + 1) * k * k * p.esz);
  if (p.split_c > 1) upd((size_t)p.split_c * k * n * p.esz);
  size_t cur = 0;
  const size_t e = p.esz;
  p.off_G = carve(cur, (size_t)p.ldg * l * e);
  p.off_Y = carve(cur, (size_t)p.ldy * l * e);
  p.off_Lt = carve(cur, (size_t)p.ldl * k * e);
  p.off_Lp = carve(cur, (size_t)p.ldl * k * e);
  p.off_M = carve(cur, (size_t)k * k * 8);
  const size_t kp = (size_t)round_up(k, 32);  // M = L D L^T: L padded to kp x kp
  p.off_dinv = carve(cur, (size_t)k * 8);
  p.off_LT = carve(cur, kp * kp * e);
  p.off_LR = carve(cur, kp * kp * e);
  p.off_W = carve(cur, kp * 32 * e);   // inverses of L's 32 x 32 diagonal blocks
  p.off_WT = carve(cur, kp * 32 * e);
  p.off_C = carve(cur, (size_t)k * p.ldb * e);
  p.off_B = carve(cur, (size_t)k * p.ldb * e);
  p.off_Lb = carve(cur, (size_t)k * k * e);
  p.off_part = carve(cur, part);
  p.off_pos = carve(cur, (size_t)(m > n ? m : n) * sizeof(int32_t));  // LU position state
  p.off_ps = carve(cur, (size_t)l * sizeof(int32_t));
  p.ldu12 = round_up(l, 4);  // the LUs' solved pivot rows, dense (<= 96 rows of <= l columns)
  p.off_u12 = carve(cur, (size_t)96 * p.ldu12 * e);
  if (prec == RLU_PREC_MIXED || bf16_like)  // the LUs' trailing updates on the tensor cores
    p.off_u12t = carve(cur, (size_t)2 * 96 * p.ldu12 * sizeof(float));
  if (prec == RLU_PREC_MIXED || bf16_like) {
    p.off_Lhi = carve(cur, (size_t)p.ldl * k * e);
    p.off_Llo = carve(cur, (size_t)p.ldl * k * e);
    p.off_Lbh = carve(cur, (size_t)round_up(k, 4) * k * 4);
    p.off_Lbl = carve(cur, (size_t)round_up(k, 4) * k * 4);
  }
  if (bf16_like) {  // L~ in three BF16 parts for the products with BF16 A
    p.off_Bh = carve(cur, (size_t)p.ldl * k * 2);
    p.off_Bm = carve(cur, (size_t)p.ldl * k * 2);
    p.off_Bl = carve(cur, (size_t)p.ldl * k * 2);
  }
  if (q > 0) {  // Z (n x l, ld ldg) and the splits of Y and Z for the accurate products
    p.off_Z = carve(cur, (size_t)p.ldg * l * e);
    // the normalised block P^T L of the LU of Y (ld ldy) or of Z (ld ldg), read by the
    // SIMT products (the tensor-core paths read its splits instead)
    p.off_Ln = carve(cur, (size_t)(p.ldy > p.ldg ? p.ldy : p.ldg) * l * e);
    if (prec == RLU_PREC_MIXED) {
      p.off_Yh = carve(cur, (size_t)p.ldy * l * 4);
      p.off_Yl = carve(cur, (size_t)p.ldy * l * 4);
      p.off_Zh = carve(cur, (size_t)p.ldg * l * 4);
      p.off_Zl = carve(cur, (size_t)p.ldg * l * 4);
    }
    if (bf16_like)
      for (int t = 0; t < 3; ++t) {
        p.off_Yb[t] = carve(cur, (size_t)p.ldy * l * 2);
        p.off_Zb[t] = carve(cur, (size_t)p.ldg * l * 2);
      }
  }
  if (prec == RLU_PREC_FP8) {  // e4m3 A (m rows) and G (l rows) with their scales
    p.ld8 = fp8_ld(n);
    p.lds = ceil_div(n, 128);
    p.lsg = ceil_div(l, 128);
    p.off_A8 = carve(cur, (size_t)m * p.ld8);
    p.off_SA = carve(cur, (size_t)m * p.lds);
    p.off_G8 = carve(cur, (size_t)l * p.ld8);
    p.off_SG = carve(cur, (size_t)p.lds * p.lsg);
  }
  p.total = cur;
  return true;
}

template <typename T>
static int32_t factor_t(const Plan& p, const void* Av, int64_t lda, uint64_t seed, int32_t* P,
                        int32_t* Q, T* L, int64_t ldl_out, T* U, int64_t ldu, rlu_info* info,
                        char* ws, const rlu_stage_outputs* st, cudaStream_t s) {
  T* G = reinterpret_cast<T*>(ws + p.off_G);
  T* Y = reinterpret_cast<T*>(ws + p.off_Y);
  T* Lt = reinterpret_cast<T*>(ws + p.off_Lt);
  T* Lp = reinterpret_cast<T*>(ws + p.off_Lp);
  double* M = reinterpret_cast<double*>(ws + p.off_M);
  LdlOut<T> ldl{};
  ldl.LT = reinterpret_cast<T*>(ws + p.off_LT);
  ldl.LR = reinterpret_cast<T*>(ws + p.off_LR);
  ldl.W = reinterpret_cast<T*>(ws + p.off_W);
  ldl.WT = reinterpret_cast<T*>(ws + p.off_WT);
  ldl.dinv = reinterpret_cast<double*>(ws + p.off_dinv);
  ldl.k = p.k;
  ldl.kp = (int)round_up(p.k, 32);
  T* Cb = reinterpret_cast<T*>(ws + p.off_C);
  T* Bb = reinterpret_cast<T*>(ws + p.off_B);
  T* Lb = reinterpret_cast<T*>(ws + p.off_Lb);
  void* part = ws + p.off_part;
  const T* A = static_cast<const T*>(Av);  // FP32/FP64 storage (BF16: only Av is read)
  // the FP8 form shares the BF16 form's products after step 2
  const bool fp8 = p.prec == RLU_PREC_FP8;
  const bool bf16 = p.prec == RLU_PREC_BF16 || fp8;
  const int64_t m = p.m, n = p.n;
  const int k = p.k, l = p.l;

  const StepTimer tm{st};
  if (info) RLU_TRY(info_init(info, s));
  // step 1
  RLU_TRY(tm.rec(0, false, s));
  RLU_TRY(launch_gaussian(seed, 0, n, l, (bf16 && !fp8) ? RLU_BF16 : p.dt, G, p.ldg, s));
  if (fp8)  // e4m3 G with one scale per 128 x 128 block
    RLU_TRY(fp8_quantize_g(reinterpret_cast<const float*>(G), p.ldg, n, l,
                           reinterpret_cast<uint8_t*>(ws + p.off_G8), p.ld8,
                           reinterpret_cast<uint8_t*>(ws + p.off_SG), p.lsg, s));
  RLU_TRY(tm.rec(0, true, s));
  if (st && st->G) {
    if (bf16 && !fp8)
      RLU_TRY(copy_cm<__nv_bfloat16>(reinterpret_cast<const __nv_bfloat16*>(G), p.ldg,
                                     static_cast<__nv_bfloat16*>(st->G), n, n, l, s));
    else
      RLU_TRY(copy_cm<T>(G, p.ldg, static_cast<T*>(st->G), n, n, l, s));
  }
  // step 2: Y (m x l, col-major) = A (row-major) * G (col-major)
  RLU_TRY(tm.rec(1, false, s));
  // the tensor-core projection reads A with TMA: rows must start on 16-byte boundaries
  const bool tma_ok = ((uintptr_t)A & 15u) == 0 && (lda * (int64_t)sizeof(T)) % 16 == 0;
  if (fp8) {  // e4m3 A (one scale per row and 128 columns) times e4m3 G, FP32 accumulation
    uint8_t* A8 = reinterpret_cast<uint8_t*>(ws + p.off_A8);
    uint8_t* SA = reinterpret_cast<uint8_t*>(ws + p.off_SA);
    RLU_TRY(fp8_quantize_a(Av, lda, m, n, A8, p.ld8, SA, p.lds, s));
    Fp8Op op{};
    op.A8 = A8;
    op.lda8 = p.ld8;
    op.SA = SA;
    op.lds = p.lds;
    op.G8 = reinterpret_cast<const uint8_t*>(ws + p.off_G8);
    op.ldg8 = p.ld8;
    op.SG = reinterpret_cast<const uint8_t*>(ws + p.off_SG);
    op.lsg = p.lsg;
    op.M = m;
    op.N = l;
    op.K = n;
    op.out = reinterpret_cast<float*>(Y);
    op.ldo = p.ldy;
    op.out_colmajor = true;
    op.splits = p.split_y;
    op.partial = reinterpret_cast<float*>(part);
    op.status = info ? &info->status : nullptr;
    RLU_TRY(umma_fp8_y(op, s));
  } else if (bf16) {  // BF16 A and G, FP32 accumulation (validated: A rows 16-byte aligned)
    UmmaBf16Op op{};
    op.A = Av;
    op.lda = lda;
    op.B0 = G;
    op.ldb = p.ldg;
    op.M = m;
    op.N = l;
    op.K = n;
    op.out = reinterpret_cast<float*>(Y);
    op.ldo = p.ldy;
    op.out_colmajor = true;
    op.splits = p.split_y;
    op.partial = reinterpret_cast<float*>(part);
    op.status = info ? &info->status : nullptr;
    RLU_TRY(umma_bf16_gemm(UB_MODE_Y, op, s));
  } else if (p.prec == RLU_PREC_MIXED && tma_ok) {
    Umma3Op op{};
    op.A0 = reinterpret_cast<const float*>(A);
    op.lda = lda;
    op.B0 = reinterpret_cast<const float*>(G);
    op.ldb = p.ldg;
    op.M = m;
    op.N = l;
    op.K = n;
    op.out = reinterpret_cast<float*>(Y);
    op.ldo = p.ldy;
    op.out_colmajor = true;
    op.splits = p.split_y;
    op.partial = reinterpret_cast<float*>(part);
    op.status = info ? &info->status : nullptr;
    RLU_TRY(umma3_gemm(U3_MODE_Y2, op, s));
  } else {
    GemmOp op{A, lda, true, G, p.ldg, true, Y, p.ldy, false, m, l, n, p.split_y, part, false};
    RLU_TRY((gemm_simt<T, T>(op, s)));
  }
  // power iterations (Section 5): Y <- A (A^T Y), q times, with FP32-accurate products on
  // the reduced-precision paths (Z and Y are not random matrices whose rounding is harmless)
  // LU normalisation of a block X (rows x l, column-major, ld): X is factored in place with
  // partial pivoting (its permutation into perm, an output buffer overwritten later) and
  // replaced, for the next product, by P^T L (unit lower factor, rows put back): in FP32 /
  // FP64 into Ln, or straight into the splits the tensor-core products read.
  auto normalize = [&](T* X, int64_t ld, int64_t rows, int32_t* perm, T* Ln, T* hi, T* lo,
                       Bf16Parts parts) -> int32_t {
    LuArgs a{};
    a.X = X; a.ldx = ld; a.R = (int)rows; a.C = l; a.perm = perm;
    a.zero_step = nullptr;  // a zero pivot of a round is not one of the factorization's
    a.nonfinite = info ? &info->nonfinite : nullptr;
    a.status = info ? &info->status : nullptr;
    a.posg = reinterpret_cast<int32_t*>(ws + p.off_pos);
    a.psg = reinterpret_cast<int32_t*>(ws + p.off_ps);
    a.u12 = ws + p.off_u12;
    a.ldu = p.ldu12;
    a.u12t = p.off_u12t ? ws + p.off_u12t : nullptr;
    RLU_TRY(launch_cluster_lu(p.dt, false, a, s));
    return build_ly<T>(X, ld, rows, l, perm, Ln, nullptr, ld, s, hi, lo, parts);
  };
  for (int it = 0; it < p.q; ++it) {
    T* Z = reinterpret_cast<T*>(ws + p.off_Z);  // n x l, column-major, ld ldg
    T* Ln = reinterpret_cast<T*>(ws + p.off_Ln);
    if (bf16) {
      Bf16Parts yp{}, zp{};
      yp.hi = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Yb[0]);
      yp.mid = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Yb[1]);
      yp.lo = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Yb[2]);
      zp.hi = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Zb[0]);
      zp.mid = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Zb[1]);
      zp.lo = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Zb[2]);
      if (p.normalized)
        RLU_TRY(normalize(Y, p.ldy, m, P, nullptr, nullptr, nullptr, yp));
      else
        RLU_TRY(split_parts(reinterpret_cast<const float*>(Y), p.ldy, m, l, nullptr, nullptr, yp, s));
      UmmaBf16Op zo{};  // Z^T (l x n, row-major = Z column-major) = Y^T A
      zo.A = Av;
      zo.lda = lda;
      zo.B0 = yp.hi;
      zo.B1 = yp.mid;
      zo.B2 = yp.lo;
      zo.ldb = p.ldy;
      zo.M = l;
      zo.N = n;
      zo.K = m;
      zo.out = reinterpret_cast<float*>(Z);
      zo.ldo = p.ldg;
      zo.out_colmajor = false;
      zo.splits = p.split_z;
      zo.partial = reinterpret_cast<float*>(part);
      zo.status = info ? &info->status : nullptr;
      RLU_TRY(umma_bf16_gemm(UB_MODE_C3, zo, s));
      if (p.normalized)
        RLU_TRY(normalize(Z, p.ldg, n, Q, nullptr, nullptr, nullptr, zp));
      else
        RLU_TRY(split_parts(reinterpret_cast<const float*>(Z), p.ldg, n, l, nullptr, nullptr, zp, s));
      UmmaBf16Op yo{};  // Y = A Z, Z in three BF16 parts
      yo.A = Av;
      yo.lda = lda;
      yo.B0 = zp.hi;
      yo.B1 = zp.mid;
      yo.B2 = zp.lo;
      yo.ldb = p.ldg;
      yo.M = m;
      yo.N = l;
      yo.K = n;
      yo.out = reinterpret_cast<float*>(Y);
      yo.ldo = p.ldy;
      yo.out_colmajor = true;
      yo.splits = p.split_y3;
      yo.partial = reinterpret_cast<float*>(part);
      yo.status = info ? &info->status : nullptr;
      RLU_TRY(umma_bf16_gemm(UB_MODE_Y3, yo, s));
    } else if (p.prec == RLU_PREC_MIXED && tma_ok) {
      float* Yh = reinterpret_cast<float*>(ws + p.off_Yh);
      float* Yl = reinterpret_cast<float*>(ws + p.off_Yl);
      float* Zh = reinterpret_cast<float*>(ws + p.off_Zh);
      float* Zl = reinterpret_cast<float*>(ws + p.off_Zl);
      if (p.normalized)
        RLU_TRY(normalize(Y, p.ldy, m, P, nullptr, reinterpret_cast<T*>(Yh),
                          reinterpret_cast<T*>(Yl), Bf16Parts{}));
      else
        RLU_TRY(split_parts(reinterpret_cast<const float*>(Y), p.ldy, m, l, Yh, Yl, Bf16Parts{}, s));
      Umma3Op zo{};  // Z (n x l, column-major) = A^T Y, three TF32 products
      zo.A0 = reinterpret_cast<const float*>(A);
      zo.lda = lda;
      zo.B0 = Yh;
      zo.B1 = Yl;
      zo.ldb = p.ldy;
      zo.M = n;
      zo.N = l;
      zo.K = m;
      zo.out = reinterpret_cast<float*>(Z);
      zo.ldo = p.ldg;
      zo.out_colmajor = true;
      zo.splits = p.split_z;
      zo.partial = reinterpret_cast<float*>(part);
      zo.status = info ? &info->status : nullptr;
      RLU_TRY(umma3_gemm(U3_MODE_C3, zo, s));
      if (p.normalized)
        RLU_TRY(normalize(Z, p.ldg, n, Q, nullptr, reinterpret_cast<T*>(Zh),
                          reinterpret_cast<T*>(Zl), Bf16Parts{}));
      else
        RLU_TRY(split_parts(reinterpret_cast<const float*>(Z), p.ldg, n, l, Zh, Zl, Bf16Parts{}, s));
      Umma3Op yo{};  // Y = A Z, three TF32 products
      yo.A0 = reinterpret_cast<const float*>(A);
      yo.lda = lda;
      yo.B0 = Zh;
      yo.B1 = Zl;
      yo.ldb = p.ldg;
      yo.M = m;
      yo.N = l;
      yo.K = n;
      yo.out = reinterpret_cast<float*>(Y);
      yo.ldo = p.ldy;
      yo.out_colmajor = true;
      yo.splits = p.split_y3;
      yo.partial = reinterpret_cast<float*>(part);
      yo.status = info ? &info->status : nullptr;
      RLU_TRY(umma3_gemm(U3_MODE_Y3, yo, s));
    } else {
      const T* Yin = Y;
      if (p.normalized) {
        RLU_TRY(normalize(Y, p.ldy, m, P, Ln, nullptr, nullptr, Bf16Parts{}));
        Yin = Ln;
      }
      GemmOp zo{Yin, p.ldy, true, A, lda, false, Z, p.ldg, true, l, n, m, p.split_z, part, false};
      RLU_TRY((gemm_simt<T, T>(zo, s)));
      const T* Zin = Z;
      if (p.normalized) {
        RLU_TRY(normalize(Z, p.ldg, n, Q, Ln, nullptr, nullptr, Bf16Parts{}));
        Zin = Ln;
      }
      GemmOp yo{A, lda, true, Zin, p.ldg, true, Y, p.ldy, false, m, l, n, p.split_y3, part, false};
      RLU_TRY((gemm_simt<T, T>(yo, s)));
    }
  }
  RLU_TRY(tm.rec(1, true, s));
  if (st && st->Y) RLU_TRY(copy_cm<T>(Y, p.ldy, static_cast<T*>(st->Y), m, m, l, s));
  // step 3
  RLU_TRY(tm.rec(2, false, s));
  {
    LuArgs a{};
    a.X = Y; a.ldx = p.ldy; a.R = (int)m; a.C = l; a.perm = P;
    a.zero_step = info ? &info->first_zero_pivot_y : nullptr;
    a.nonfinite = info ? &info->nonfinite : nullptr;
    a.status = info ? &info->status : nullptr;
    a.posg = reinterpret_cast<int32_t*>(ws + p.off_pos);
    a.psg = reinterpret_cast<int32_t*>(ws + p.off_ps);
    a.u12 = ws + p.off_u12;
    a.ldu = p.ldu12;
    a.u12t = p.off_u12t ? ws + p.off_u12t : nullptr;
    RLU_TRY(launch_cluster_lu(p.dt, false, a, s));
  }
  RLU_TRY(tm.rec(2, true, s));
  // step 4
  RLU_TRY(tm.rec(3, false, s));
  T* Lhi = p.off_Lhi ? reinterpret_cast<T*>(ws + p.off_Lhi) : nullptr;
  T* Llo = p.off_Llo ? reinterpret_cast<T*>(ws + p.off_Llo) : nullptr;
  Bf16Parts bp{};
  if (bf16) {
    bp.hi = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Bh);
    bp.mid = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Bm);
    bp.lo = reinterpret_cast<__nv_bfloat16*>(ws + p.off_Bl);
  }
  RLU_TRY(build_ly<T>(Y, p.ldy, m, k, P, Lt, Lp, p.ldl, s, Lhi, Llo, bp));
  RLU_TRY(tm.rec(3, true, s));
  if (st && st->Ly) RLU_TRY(copy_cm<T>(Lp, p.ldl, static_cast<T*>(st->Ly), m, m, k, s));
  // step 5: Gram M = L~^T L~ in FP64
  RLU_TRY(tm.rec(4, false, s));
  if (Lhi) {  // tensor cores, 3 TF32 products; FP32 partials summed in FP64
    Umma3Op op{};
    op.A0 = reinterpret_cast<const float*>(Lhi);
    op.A1 = reinterpret_cast<const float*>(Llo);
    op.lda = p.ldl;
    op.B0 = op.A0;
    op.B1 = op.A1;
    op.ldb = p.ldl;
    op.M = k;
    op.N = k;
    op.K = m;
    op.out = nullptr;
    op.splits = p.split_g;
    op.partial = reinterpret_cast<float*>(part);
    op.status = info ? &info->status : nullptr;
    RLU_TRY(umma3_gemm(U3_MODE_G3, op, s));
    const int kc = (int)round_up(ceil_div(m, p.split_g), 32);
    RLU_TRY(splitk_reduce_f64(reinterpret_cast<const float*>(part), (int)ceil_div(m, kc), k, k,
                              M, k, s));
  } else {
    GemmOp op{Lt, p.ldl, true, Lt, p.ldl, true, M, k, true, k, k, m, p.split_g, part, false};
    RLU_TRY((gemm_simt<T, double>(op, s)));
  }
  RLU_TRY(tm.rec(4, true, s));
  SideStream* ss = nullptr;
  RLU_TRY(side_stream(s, &ss));
  {
    std::lock_guard<std::mutex> lock(ss->mu);
    RLU_CUDA_TRY(cudaEventRecord(ss->fork, s));
    RLU_CUDA_TRY(cudaStreamWaitEvent(ss->side, ss->fork, 0));
    RLU_TRY(tm.rec(5, false, ss->side));
    RLU_TRY(ldl_factor<T>(M, k, ldl, info ? &info->status : nullptr, ss->side));
    RLU_TRY(tm.rec(5, true, ss->side));
    RLU_CUDA_TRY(cudaEventRecord(ss->join, ss->side));
    // C = L~^T A (k x n, row-major)
    RLU_TRY(tm.rec(6, false, s));
    if (bf16) {  // C = L~^T A with L~ in three BF16 parts and BF16 A
      UmmaBf16Op op{};
      op.A = Av;
      op.lda = lda;
      op.B0 = bp.hi;
      op.B1 = bp.mid;
      op.B2 = bp.lo;
      op.ldb = p.ldl;
      op.M = k;
      op.N = n;
      op.K = m;
      op.out = reinterpret_cast<float*>(Cb);
      op.ldo = p.ldb;
      op.out_colmajor = false;
      op.splits = p.split_c;
      op.partial = reinterpret_cast<float*>(part);
      op.status = info ? &info->status : nullptr;
      RLU_TRY(umma_bf16_gemm(UB_MODE_C3, op, s));
    } else if (Lhi && tma_ok) {  // C^T = A^T L~ on the tensor cores, 3 TF32 products
      Umma3Op op{};
      op.A0 = reinterpret_cast<const float*>(A);
      op.lda = lda;
      op.B0 = reinterpret_cast<const float*>(Lhi);
      op.B1 = reinterpret_cast<const float*>(Llo);
      op.ldb = p.ldl;
      op.M = n;
      op.N = k;
      op.K = m;
      op.out = reinterpret_cast<float*>(Cb);
      op.ldo = p.ldb;
      op.out_colmajor = true;  // D row = column of A, D column = row of C
      op.splits = p.split_c;
      op.partial = reinterpret_cast<float*>(part);
      op.status = info ? &info->status : nullptr;
      RLU_TRY(umma3_gemm(U3_MODE_C3, op, s));
    } else {
      GemmOp op{Lt, p.ldl, true, A, lda, false, Cb, p.ldb, true, k, n, m, p.split_c, part, false};
      RLU_TRY((gemm_simt<T, T>(op, s)));
    }
    RLU_TRY(tm.rec(6, true, s));
    RLU_CUDA_TRY(cudaStreamWaitEvent(s, ss->join, 0));
  }
  // B = M^{-1} C = L^{-T} D^{-1} L^{-1} C
  RLU_TRY(tm.rec(7, false, s));
  RLU_TRY(trsm_ldl<T>(ldl, Cb, p.ldb, n, Bb, p.ldb, s));
  RLU_TRY(tm.rec(7, true, s));
  if (st && st->B) RLU_TRY(copy_cm<T>(Bb, p.ldb, static_cast<T*>(st->B), n, n, k, s));
  // step 6: LU of B^T (n x k, col-major = B row-major), Crout form
  RLU_TRY(tm.rec(8, false, s));
  {
    LuArgs a{};
    a.X = Bb; a.ldx = p.ldb; a.R = (int)n; a.C = k; a.perm = Q;
    a.zero_step = info ? &info->first_zero_pivot_b : nullptr;
    a.nonfinite = info ? &info->nonfinite : nullptr;
    a.status = info ? &info->status : nullptr;
    a.posg = reinterpret_cast<int32_t*>(ws + p.off_pos);
    a.psg = reinterpret_cast<int32_t*>(ws + p.off_ps);
    a.u12 = ws + p.off_u12;
    a.ldu = p.ldu12;
    a.u12t = p.off_u12t ? ws + p.off_u12t : nullptr;
    RLU_TRY(launch_cluster_lu(p.dt, true, a, s));
  }
  RLU_TRY(tm.rec(8, true, s));
  // step 8 (and L_b for step 7)
  RLU_TRY(tm.rec(9, false, s));
  RLU_TRY(gather_lb_u<T>(Bb, p.ldb, Q, k, n, Lb, U, ldu, s));
  RLU_TRY(tm.rec(9, true, s));
  // step 7: L = L_y L_b
  RLU_TRY(tm.rec(10, false, s));
  if (p.off_Lbh) {  // three TF32 products: L_y (column-major, i.e. K x M row-major) is
                    // transposed and split on chip as in the C product; L_b pre-split
    float* Lbh = reinterpret_cast<float*>(ws + p.off_Lbh);
    float* Lbl = reinterpret_cast<float*>(ws + p.off_Lbl);
    const int64_t kb = round_up(k, 4);
    RLU_TRY(split_parts(reinterpret_cast<const float*>(Lb), k, k, k, Lbh, Lbl, Bf16Parts{}, s,
                        kb));
    Umma3Op op{};
    op.A0 = reinterpret_cast<const float*>(Lp);
    op.lda = p.ldl;
    op.B0 = Lbh;
    op.B1 = Lbl;
    op.ldb = kb;
    op.M = m;
    op.N = k;
    op.K = k;
    op.out = reinterpret_cast<float*>(L);
    op.ldo = ldl_out;
    op.out_colmajor = true;
    op.splits = 1;
    op.status = info ? &info->status : nullptr;
    RLU_TRY(umma3_gemm(U3_MODE_C3, op, s));
  } else {
    GemmOp op{Lp, p.ldl, false, Lb, k, true, L, ldl_out, false, m, k, k, 1, nullptr, false};
    RLU_TRY((gemm_simt<T, T>(op, s)));
  }
  RLU_TRY(tm.rec(10, true, s));
  return RLU_OK;
}

int32_t validate(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                        int32_t k, int32_t l, int32_t prec, const int32_t* P, const int32_t* Q,
                        const void* L, int64_t ldl, const void* U, int64_t ldu) {
  if (!A || !P || !Q || !L || !U) return RLU_EINVAL;
  if (m < 1 || n < 1 || k < 1 || k > l || l > m || l > n) return RLU_EINVAL;
  if (lda < n || ldl < m || ldu < n) return RLU_EINVAL;
  if (prec == RLU_PREC_F64 && dtype != RLU_F64) return RLU_EUNSUPPORTED;
  if ((prec == RLU_PREC_F32 || prec == RLU_PREC_MIXED) && dtype != RLU_F32)
    return RLU_EUNSUPPORTED;
  if (prec == RLU_PREC_BF16 || prec == RLU_PREC_FP8) {
    if (dtype != RLU_BF16) return RLU_EUNSUPPORTED;
    // the BF16 products read A with TMA: rows on 16-byte boundaries
    if (((uintptr_t)A & 15u) != 0 || lda % 8 != 0) return RLU_EINVAL;
  }
  if (prec != RLU_PREC_F64 && prec != RLU_PREC_F32 && prec != RLU_PREC_MIXED &&
      prec != RLU_PREC_BF16 && prec != RLU_PREC_FP8)
    return RLU_EUNSUPPORTED;
  return RLU_OK;
}

}  // namespace rlu

using namespace rlu;

extern "C" int32_t rlu_version(void) { return 100; }

extern "C" const char* rlu_timed_step_name(int32_t i) {
  return (i >= 0 && i < RLU_NUM_TIMED_STEPS) ? kStepNames[i] : nullptr;
}

extern "C" uint64_t rlu_launch_count(void) { return g_launches.load(); }

extern "C" const char* rlu_status_string(int32_t status) {
  switch (status) {
    case RLU_OK: return "ok";
    case RLU_EINVAL: return "invalid argument";
    case RLU_ENOMEM: return "workspace too small";
    case RLU_EUNSUPPORTED: return "unsupported dtype/precision/size";
    case RLU_ECUDA: return "CUDA runtime error";
    case RLU_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

extern "C" size_t rlu_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l, int32_t prec) {
  Plan p;
  if (!make_plan(m, n, k, l, prec, p)) return 0;
  return p.total;
}

extern "C" size_t rlu_workspace_size_power(int64_t m, int64_t n, int32_t k, int32_t l,
                                           int32_t prec, int32_t q) {
  Plan p;
  if (!make_plan(m, n, k, l, prec, p, q)) return 0;
  return p.total;
}

extern "C" int32_t rlu_factor_power(const void* A, int32_t dtype, int64_t m, int64_t n,
                                    int64_t lda, int32_t k, int32_t l, uint64_t seed,
                                    int32_t prec, int32_t q, int32_t normalized, int32_t* P,
                                    int32_t* Q, void* L, int64_t ldl, void* U, int64_t ldu,
                                    rlu_info* info, void* workspace, size_t ws_bytes,
                                    const rlu_stage_outputs* stages, void* stream) {
  RLU_TRY(validate(A, dtype, m, n, lda, k, l, prec, P, Q, L, ldl, U, ldu));
  if (normalized != 0 && normalized != 1) return RLU_EINVAL;
  Plan p;
  if (!make_plan(m, n, k, l, prec, p, q, normalized != 0)) return RLU_EINVAL;
  if (workspace == nullptr || ws_bytes < p.total) return RLU_ENOMEM;
  if (((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (p.dt == RLU_F64)
    return factor_t<double>(p, A, lda, seed, P, Q, (double*)L, ldl, (double*)U, ldu, info,
                            (char*)workspace, stages, s);
  return factor_t<float>(p, A, lda, seed, P, Q, (float*)L, ldl, (float*)U, ldu, info,
                         (char*)workspace, stages, s);
}

extern "C" int32_t rlu_factor_stages(const void* A, int32_t dtype, int64_t m, int64_t n,
                                     int64_t lda, int32_t k, int32_t l, uint64_t seed,
                                     int32_t prec, int32_t* P, int32_t* Q, void* L, int64_t ldl,
                                     void* U, int64_t ldu, rlu_info* info, void* workspace,
                                     size_t ws_bytes, const rlu_stage_outputs* stages,
                                     void* stream) {
  return rlu_factor_power(A, dtype, m, n, lda, k, l, seed, prec, 0, 0, P, Q, L, ldl, U, ldu,
                          info, workspace, ws_bytes, stages, stream);
}

extern "C" int32_t rlu_factor(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                              int32_t k, int32_t l, uint64_t seed, int32_t prec, int32_t* P,
                              int32_t* Q, void* L, int64_t ldl, void* U, int64_t ldu,
                              rlu_info* info, void* workspace, size_t ws_bytes, void* stream) {
  return rlu_factor_stages(A, dtype, m, n, lda, k, l, seed, prec, P, Q, L, ldl, U, ldu, info,
                           workspace, ws_bytes, nullptr, stream);
}

extern "C" size_t rlu_reconstruct_workspace_size(int64_t m, int64_t n, int32_t k) {
  if (m < 1 || n < 1 || k < 1) return 0;
  return residual_workspace_bytes(m, n, k);
}

extern "C" int32_t rlu_reconstruct_error(const void* A, int32_t dtype, int64_t m, int64_t n,
                                         int64_t lda, int32_t k, const int32_t* P,
                                         const int32_t* Q, const void* L, int64_t ldl,
                                         const void* U, int64_t ldu, int32_t lu_dtype,
                                         double* err_fro, double* err_spec, int32_t power_iters,
                                         void* workspace, size_t ws_bytes, void* stream) {
  if (!A || !P || !Q || !L || !U || !err_fro) return RLU_EINVAL;
  if (m < 1 || n < 1 || k < 1 || lda < n || ldl < m || ldu < n || power_iters < 0)
    return RLU_EINVAL;
  if (workspace == nullptr || ws_bytes < residual_workspace_bytes(m, n, k)) return RLU_ENOMEM;
  ResidualArgs a{A, lda, P, Q, L, ldl, U, ldu, m, n, k};
  return residual_error(dtype, lu_dtype, a, err_fro, err_spec, power_iters, (double*)workspace,
                        (cudaStream_t)stream);
}
