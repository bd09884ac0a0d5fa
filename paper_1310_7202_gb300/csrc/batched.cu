// Batched form (include/rlu_batch.h): the steps of Algorithm 1 for many independent problems
// of uneven sizes, each step one launch over the whole batch (per-problem argument records
// in device memory, entry z = problem z), so the launch count does not grow with the batch
// and the sequence can be captured in a CUDA graph.
//
//   info init, step 1 G (batched Philox/Box-Muller), step 2 Y = A G (batched SIMT GEMM, or
//   the tcgen05 TF32-split GEMM with per-problem tensor maps for RLU_PREC_MIXED),
//   step 3 LU(Y) (one thread-block cluster per problem, launches grouped by cluster size),
//   step 4 L_y and L~, step 5 Gram (FP32 products stored in FP64) -> LDL^T (one CTA per
//   problem) and C = L~^T A (SIMT, or tcgen05 for RLU_PREC_MIXED) -> blocked triangular
//   solves, step 6 LU(B^T) (clusters), steps
//   7-8 L_b, U gathers and L = L_y L_b.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "batched.cuh"
#include "gemm_simt.cuh"
#include "panel_lu.cuh"
#include "umma.cuh"
#include "../../include/rlu_batch.h"

namespace rlu {

namespace {

constexpr int kMaxL = 76;   // one register panel per LU (FP32)
constexpr int kMaxK = 256;  // one-CTA LDL^T
constexpr int64_t kMaxRows = 16 * 512;

size_t carve(size_t& cur, size_t bytes) {
  const size_t at = cur;
  cur += (size_t)round_up((int64_t)std::max<size_t>(bytes, 1), 256);
  return at;
}

struct ProblemLayout {
  int64_t ldg, ldy, ldl, ldb;
  int kp;
  size_t G, Y, Lt, Lp, Mg, dinv, LT, LR, W, WT, C, B, Lb, pos, ps, Lhi, Llo;
};

struct Tables {
  size_t info, gauss, gemm_y, lu_y, build, gemm_g, ldl, gemm_c, trsm, lu_b, gather, gemm_l,
      u3y, u3c, u3y_tiles, u3c_tiles, trsm_tiles, lmul_tiles, u3_counter;
  int n_tiles_y, n_tiles_c;  // 128-row tiles of the two tensor-core products
  int n_tiles_t;             // column blocks of the substitution B = M^{-1} C
  int n_tiles_l;             // 256-row blocks of L = L_y L_b (small k only)
  bool small_k;              // every k <= 64: register kernels for the solve and L
};

constexpr int kSmallK = 64;

// LU group of a problem with R rows (see rlu_batch) and its rows per CTA: small problems
// take one narrow CTA, so that several of them share an SM.
int lu_group(int64_t R, int rows_per_cta, int* rpc) {
  if (R <= 128) {
    *rpc = 128;
    return 17;
  }
  if (R <= 256 && rows_per_cta == 512) {
    *rpc = 256;
    return 18;
  }
  *rpc = rows_per_cta;
  return (int)ceil_div(R, rows_per_cta);
}

bool valid_problem(const rlu_problem& p, int32_t prec) {
  if (!p.A || !p.P || !p.Q || !p.L || !p.U) return false;
  // the tensor-core products read A with TMA: rows on 16-byte boundaries
  if (prec == RLU_PREC_MIXED && (((uintptr_t)p.A & 15u) != 0 || p.lda % 4 != 0)) return false;
  if (p.m < 1 || p.n < 1 || p.k < 1 || p.k > p.l || p.l > p.m || p.l > p.n) return false;
  if (p.l > kMaxL || p.k > kMaxK || p.m > kMaxRows || p.n > kMaxRows) return false;
  if (p.lda < p.n || p.ldl < p.m || p.ldu < p.n) return false;
  return true;
}

// Layout of everything: the argument tables first, then each problem's buffers.
size_t plan_layout(const rlu_problem* probs, int count, int32_t prec, Tables& t,
                   std::vector<ProblemLayout>* lay) {
  size_t cur = 0;
  const size_t c = (size_t)count;
  t.info = carve(cur, c * sizeof(rlu_info*));
  t.gauss = carve(cur, c * sizeof(GaussJob));
  t.gemm_y = carve(cur, c * sizeof(GemmArgs));
  t.lu_y = carve(cur, c * sizeof(LuArgs));
  t.build = carve(cur, c * sizeof(BuildJob));
  t.gemm_g = carve(cur, c * sizeof(GemmArgs));
  t.ldl = carve(cur, c * sizeof(Ldl32Job));
  t.gemm_c = carve(cur, c * sizeof(GemmArgs));
  t.trsm = carve(cur, c * sizeof(TrsmJob));
  t.small_k = true;
  for (int i = 0; i < count; ++i) t.small_k = t.small_k && probs[i].k <= kSmallK;
  t.n_tiles_t = t.n_tiles_l = 0;
  for (int i = 0; i < count; ++i) {
    t.n_tiles_t += (int)ceil_div(probs[i].n, t.small_k ? 128 : 64);
    if (t.small_k) t.n_tiles_l += (int)ceil_div(probs[i].m, 256);
  }
  t.trsm_tiles = carve(cur, (size_t)t.n_tiles_t * sizeof(int2));
  t.lmul_tiles = carve(cur, (size_t)t.n_tiles_l * sizeof(int2));
  t.lu_b = carve(cur, c * sizeof(LuArgs));
  t.gather = carve(cur, c * sizeof(GatherJob));
  t.gemm_l = carve(cur, c * sizeof(GemmArgs));
  t.u3y = t.u3c = t.u3y_tiles = t.u3c_tiles = 0;
  t.n_tiles_y = t.n_tiles_c = 0;
  if (prec == RLU_PREC_MIXED) {
    t.u3y = carve(cur, c * sizeof(U3Job));
    t.u3c = carve(cur, c * sizeof(U3Job));
    for (int i = 0; i < count; ++i) {
      t.n_tiles_y += (int)ceil_div(probs[i].m, 128);
      t.n_tiles_c += (int)ceil_div(probs[i].n, 128);
    }
    t.u3y_tiles = carve(cur, (size_t)t.n_tiles_y * sizeof(int2));
    t.u3c_tiles = carve(cur, (size_t)t.n_tiles_c * sizeof(int2));
    t.u3_counter = carve(cur, 256);  // tile counter of the persistent products
  }
  for (int i = 0; i < count; ++i) {
    const rlu_problem& p = probs[i];
    ProblemLayout L{};
    L.ldg = round_up(p.n, 4);
    L.ldy = round_up(p.m, 4);
    L.ldl = round_up(p.m, 4);
    L.ldb = round_up(p.n, 4);
    L.kp = (int)round_up(p.k, 32);
    const size_t kp = (size_t)L.kp;
    L.G = carve(cur, (size_t)L.ldg * p.l * 4);
    L.Y = carve(cur, (size_t)L.ldy * p.l * 4);
    L.Lt = carve(cur, (size_t)L.ldl * p.k * 4);
    L.Lp = carve(cur, (size_t)L.ldl * p.k * 4);
    L.Mg = carve(cur, (size_t)p.k * p.k * 8);
    L.dinv = carve(cur, (size_t)p.k * 8);
    L.LT = carve(cur, kp * kp * 4);
    L.LR = carve(cur, kp * kp * 4);
    L.W = carve(cur, kp * 32 * 4);
    L.WT = carve(cur, kp * 32 * 4);
    L.C = carve(cur, (size_t)p.k * L.ldb * 4);
    L.B = carve(cur, (size_t)p.k * L.ldb * 4);
    L.Lb = carve(cur, (size_t)p.k * p.k * 4);
    L.pos = carve(cur, (size_t)std::max(p.m, p.n) * 4);
    L.ps = carve(cur, (size_t)p.l * 4);
    L.Lhi = L.Llo = 0;
    if (prec == RLU_PREC_MIXED) {
      L.Lhi = carve(cur, (size_t)L.ldl * p.k * 4);
      L.Llo = carve(cur, (size_t)L.ldl * p.k * 4);
    }
    if (lay) lay->push_back(L);
  }
  return cur;
}

__global__ void k_info_init_batched(rlu_info* const* __restrict__ infos, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    rlu_info* p = infos[i];
    if (p) {
      p->status = RLU_OK;
      p->first_zero_pivot_y = -1;
      p->first_zero_pivot_b = -1;
      p->nonfinite = 0;
    }
  }
}

}  // namespace
}  // namespace rlu

struct rlu_batch {
  char* ws = nullptr;
  int count = 0;
  int32_t prec = RLU_PREC_F32;
  rlu::Tables t{};
  int64_t max_m = 0, max_n = 0;
  int max_k = 0, max_l = 0, max_kp = 0;
  // LU groups: 1..16 = clusters of that many CTAs of lu_rows_per_cta rows; 17 / 18 = one CTA
  // of 128 / 256 threads for problems of at most 128 / 256 rows
  int first_y[rlu::kLuGroups] = {}, count_y[rlu::kLuGroups] = {}, first_b[rlu::kLuGroups] = {},
      count_b[rlu::kLuGroups] = {};
  int launches = 0;
  // tensor-core rings of the mixed precision (Y = A G, C = L~^T A)
  int u3y_stages = 0, u3y_stage_bytes = 0, u3c_stages = 0, u3c_stage_bytes = 0;
  int ts_first[4] = {}, ts_count[4] = {};  // small-k substitution tiles per bucket of k
  rlu_batch_options opt{};
  rlu::LuFork lu_fork{};  // helper streams: the LU groups run side by side
  bool have_fork = false;
  rlu_batch() = default;
  rlu_batch(const rlu_batch&) = delete;
  rlu_batch& operator=(const rlu_batch&) = delete;
  ~rlu_batch() {  // streams with work pending are released once it completes
    if (lu_fork.fork) cudaEventDestroy(lu_fork.fork);
    for (int i = 0; i < rlu::kLuSide; ++i) {
      if (lu_fork.hs[i]) cudaStreamDestroy(lu_fork.hs[i]);
      if (lu_fork.join[i]) cudaEventDestroy(lu_fork.join[i]);
    }
  }
};

extern "C" size_t rlu_batch_workspace_size(const rlu_problem* problems, int32_t count,
                                           int32_t prec) {
  using namespace rlu;
  if (!problems || count < 1 || count > 65535) return 0;
  if (prec != RLU_PREC_F32 && prec != RLU_PREC_MIXED) return 0;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(problems[i], prec)) return 0;
  Tables t{};
  return plan_layout(problems, count, prec, t, nullptr);
}

extern "C" int32_t rlu_batch_create(const rlu_problem* problems, int32_t count, int32_t prec,
                                    const rlu_batch_options* options, void* workspace,
                                    size_t ws_bytes, rlu_batch** out) {
  using namespace rlu;
  if (!out || !problems || count < 1 || count > 65535) return RLU_EINVAL;
  *out = nullptr;
  rlu_batch_options opt{};
  if (options) opt = *options;
  if (opt.lu_rows_per_cta == 0) opt.lu_rows_per_cta = 512;
  if (opt.lu_rows_per_cta != 512 && opt.lu_rows_per_cta != 256) return RLU_EINVAL;
  for (int t : {opt.gemm_tile_y, opt.gemm_tile_c, opt.gemm_tile_l})
    if (t != 0 && t != 1) return RLU_EINVAL;
  for (int u : {opt.umma_ctas_y, opt.umma_ctas_c})
    if (u < 0 || u > 2) return RLU_EINVAL;
  for (int i = 0; i < count; ++i)
    if (std::max(problems[i].m, problems[i].n) > 16 * (int64_t)opt.lu_rows_per_cta)
      return RLU_EINVAL;
  if (prec != RLU_PREC_F32 && prec != RLU_PREC_MIXED) return RLU_EUNSUPPORTED;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(problems[i], prec)) return RLU_EINVAL;
  if (workspace == nullptr || ((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  Tables t{};
  std::vector<ProblemLayout> lay;
  const size_t need = plan_layout(problems, count, prec, t, &lay);
  if (ws_bytes < need) return RLU_ENOMEM;
  char* ws = static_cast<char*>(workspace);
  rlu_batch* b = new rlu_batch();
  {
    bool ok = cudaEventCreateWithFlags(&b->lu_fork.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kLuSide; ++i)
      ok = cudaStreamCreateWithFlags(&b->lu_fork.hs[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->lu_fork.join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      delete b;  // the destructor releases what was created
      return RLU_ECUDA;
    }
    b->have_fork = true;
  }
  b->ws = ws;
  b->count = count;
  b->prec = prec;
  b->t = t;
  b->opt = opt;

  const size_t c = (size_t)count;
  std::vector<rlu_info*> infos(c);
  std::vector<GaussJob> gauss(c);
  std::vector<GemmArgs> gy(c), gg(c), gc(c), gl(c);
  std::vector<LuArgs> luy_all(c), lub_all(c);
  std::vector<BuildJob> build(c);
  std::vector<Ldl32Job> ldl(c);
  std::vector<TrsmJob> trsm(c);
  std::vector<GatherJob> gather(c);
  std::vector<int> gy_of(c), gb_of(c);
  const bool mixed = prec == RLU_PREC_MIXED;
  std::vector<U3Job> u3y(mixed ? c : 0), u3c(mixed ? c : 0);
  int max_stage_y = 0, max_stage_c = 0;
  for (int i = 0; i < count; ++i) {
    const rlu_problem& p = problems[i];
    const ProblemLayout& L = lay[(size_t)i];
    float* G = reinterpret_cast<float*>(ws + L.G);
    float* Y = reinterpret_cast<float*>(ws + L.Y);
    float* Lt = reinterpret_cast<float*>(ws + L.Lt);
    float* Lp = reinterpret_cast<float*>(ws + L.Lp);
    double* Mg = reinterpret_cast<double*>(ws + L.Mg);
    float* Cb = reinterpret_cast<float*>(ws + L.C);
    float* Bb = reinterpret_cast<float*>(ws + L.B);
    float* Lb = reinterpret_cast<float*>(ws + L.Lb);
    int32_t* pos = reinterpret_cast<int32_t*>(ws + L.pos);
    int32_t* ps = reinterpret_cast<int32_t*>(ws + L.ps);
    LdlOut<float> o{};
    o.LT = reinterpret_cast<float*>(ws + L.LT);
    o.LR = reinterpret_cast<float*>(ws + L.LR);
    o.W = reinterpret_cast<float*>(ws + L.W);
    o.WT = reinterpret_cast<float*>(ws + L.WT);
    o.dinv = reinterpret_cast<double*>(ws + L.dinv);
    o.k = p.k;
    o.kp = L.kp;
    infos[(size_t)i] = p.info;
    gauss[(size_t)i] = GaussJob{p.seed, p.n, p.l, G, L.ldg};
    GemmArgs a{};
    a.split_stride = 0;
    a.alpha_neg = false;
    // step 2: Y (m x l, column-major) = A (row-major) G (column-major)
    a.A = p.A; a.lda = p.lda; a.B = G; a.ldb = L.ldg; a.C = Y; a.ldc = L.ldy;
    a.M = p.m; a.N = p.l; a.K = p.n; a.kchunk = p.n;
    gy[(size_t)i] = a;
    // step 5: Gram M (k x k, FP64) = L~^T L~ ; C (k x n, row-major) = L~^T A
    a.A = Lt; a.lda = L.ldl; a.B = Lt; a.ldb = L.ldl; a.C = Mg; a.ldc = p.k;
    a.M = p.k; a.N = p.k; a.K = p.m; a.kchunk = p.m;
    gg[(size_t)i] = a;
    a.A = Lt; a.lda = L.ldl; a.B = p.A; a.ldb = p.lda; a.C = Cb; a.ldc = L.ldb;
    a.M = p.k; a.N = p.n; a.K = p.m; a.kchunk = p.m;
    gc[(size_t)i] = a;
    // step 7: L (m x k, column-major) = L_y (pivot order) L_b
    a.A = Lp; a.lda = L.ldl; a.B = Lb; a.ldb = p.k; a.C = p.L; a.ldc = p.ldl;
    a.M = p.m; a.N = p.k; a.K = p.k; a.kchunk = p.k;
    gl[(size_t)i] = a;
    LuArgs u{};
    u.X = Y; u.ldx = L.ldy; u.R = (int)p.m; u.C = p.l; u.perm = p.P;
    u.zero_step = p.info ? &p.info->first_zero_pivot_y : nullptr;
    u.nonfinite = p.info ? &p.info->nonfinite : nullptr;
    u.status = p.info ? &p.info->status : nullptr;
    u.posg = pos; u.psg = ps; u.p0 = 0; u.pw = p.l; u.nb = kMaxL;
    gy_of[(size_t)i] = lu_group(p.m, opt.lu_rows_per_cta, &u.rpc);
    luy_all[(size_t)i] = u;
    u.X = Bb; u.ldx = L.ldb; u.R = (int)p.n; u.C = p.k; u.perm = p.Q;
    u.zero_step = p.info ? &p.info->first_zero_pivot_b : nullptr;
    u.pw = p.k;
    gb_of[(size_t)i] = lu_group(p.n, opt.lu_rows_per_cta, &u.rpc);
    lub_all[(size_t)i] = u;
    float* Lhi = mixed ? reinterpret_cast<float*>(ws + L.Lhi) : nullptr;
    float* Llo = mixed ? reinterpret_cast<float*>(ws + L.Llo) : nullptr;
    build[(size_t)i] = BuildJob{Y, L.ldy, p.m, p.k, p.P, Lt, Lp, L.ldl, Lhi, Llo};
    if (mixed) {  // tensor-core records of Y = A G and C^T = A^T L~
      Umma3Op op{};
      op.A0 = static_cast<const float*>(p.A);
      op.lda = p.lda;
      op.B0 = G;
      op.ldb = L.ldg;
      op.M = p.m;
      op.N = p.l;
      op.K = p.n;
      op.out = Y;
      op.ldo = L.ldy;
      op.out_colmajor = true;
      op.status = p.info ? &p.info->status : nullptr;
      int sb = 0;
      int32_t st = umma3_make_job(U3_MODE_Y2, op, &u3y[(size_t)i], &sb, opt.umma_ctas_y != 2);
      max_stage_y = std::max(max_stage_y, sb);
      op = Umma3Op{};
      op.A0 = static_cast<const float*>(p.A);
      op.lda = p.lda;
      op.B0 = Lhi;
      op.B1 = Llo;
      op.ldb = L.ldl;
      op.M = p.n;
      op.N = p.k;
      op.K = p.m;
      op.out = Cb;
      op.ldo = L.ldb;
      op.out_colmajor = true;
      op.status = p.info ? &p.info->status : nullptr;
      if (st == RLU_OK)
        st = umma3_make_job(U3_MODE_C3, op, &u3c[(size_t)i], &sb, opt.umma_ctas_c != 2);
      max_stage_c = std::max(max_stage_c, sb);
      if (st != RLU_OK) {
        delete b;
        return st;
      }
    }
    ldl[(size_t)i] = Ldl32Job{Mg, p.k, o, p.info ? &p.info->status : nullptr};
    trsm[(size_t)i] = TrsmJob{o, Cb, L.ldb, p.n, Bb, L.ldb};
    gather[(size_t)i] = GatherJob{Bb, L.ldb, p.Q, p.k, p.n, Lb, static_cast<float*>(p.U), p.ldu};
    b->max_m = std::max(b->max_m, p.m);
    b->max_n = std::max(b->max_n, p.n);
    b->max_k = std::max(b->max_k, p.k);
    b->max_l = std::max(b->max_l, p.l);
    b->max_kp = std::max(b->max_kp, L.kp);
  }
  // LU records grouped by cluster size
  auto group = [&](const std::vector<LuArgs>& all, const std::vector<int>& gof, int* first,
                   int* cnt, std::vector<LuArgs>& sorted) {
    for (int g = 0; g < kLuGroups; ++g) cnt[g] = 0;
    for (int v : gof) ++cnt[v];
    int acc = 0;
    for (int g = 0; g < kLuGroups; ++g) {
      first[g] = acc;
      acc += cnt[g];
    }
    std::vector<int> fill(first, first + kLuGroups);
    sorted.resize(all.size());
    for (size_t i = 0; i < all.size(); ++i) sorted[(size_t)fill[gof[i]]++] = all[i];
  };
  std::vector<LuArgs> luy, lub;
  group(luy_all, gy_of, b->first_y, b->count_y, luy);
  group(lub_all, gb_of, b->first_b, b->count_b, lub);

  auto up = [&](size_t off, const void* src, size_t bytes) -> int32_t {
    RLU_CUDA_TRY(cudaMemcpy(ws + off, src, bytes, cudaMemcpyHostToDevice));
    return RLU_OK;
  };
  int32_t st = RLU_OK;
  if (st == RLU_OK) st = up(t.info, infos.data(), c * sizeof(rlu_info*));
  if (st == RLU_OK) st = up(t.gauss, gauss.data(), c * sizeof(GaussJob));
  if (st == RLU_OK) st = up(t.gemm_y, gy.data(), c * sizeof(GemmArgs));
  if (st == RLU_OK) st = up(t.lu_y, luy.data(), c * sizeof(LuArgs));
  if (st == RLU_OK) st = up(t.build, build.data(), c * sizeof(BuildJob));
  if (st == RLU_OK) st = up(t.gemm_g, gg.data(), c * sizeof(GemmArgs));
  if (st == RLU_OK) st = up(t.ldl, ldl.data(), c * sizeof(Ldl32Job));
  if (st == RLU_OK) st = up(t.gemm_c, gc.data(), c * sizeof(GemmArgs));
  if (st == RLU_OK) st = up(t.trsm, trsm.data(), c * sizeof(TrsmJob));
  if (st == RLU_OK) st = up(t.lu_b, lub.data(), c * sizeof(LuArgs));
  if (st == RLU_OK) st = up(t.gather, gather.data(), c * sizeof(GatherJob));
  if (st == RLU_OK) st = up(t.gemm_l, gl.data(), c * sizeof(GemmArgs));
  {  // tile lists of the substitution (problem, column block) and of L (problem, row
     // block), the blocks of a problem next to each other
    std::vector<int2> tt, tl;
    tt.reserve((size_t)t.n_tiles_t);
    tl.reserve((size_t)t.n_tiles_l);
    const int cw = t.small_k ? 128 : 64;
    // small k: the substitution's tiles grouped by the bucket of k (one launch each)
    for (int bkt = 0; bkt < (t.small_k ? 4 : 1); ++bkt) {
      if (t.small_k) b->ts_first[bkt] = (int)tt.size();
      for (int i = 0; i < count; ++i) {
        if (t.small_k && trsm_small_bucket(problems[i].k) != bkt) continue;
        for (int cb = 0; cb < (int)ceil_div(problems[i].n, cw); ++cb) tt.push_back(make_int2(i, cb));
      }
      if (t.small_k) b->ts_count[bkt] = (int)tt.size() - b->ts_first[bkt];
    }
    for (int i = 0; i < count && t.small_k; ++i)
      for (int rb = 0; rb < (int)ceil_div(problems[i].m, 256); ++rb) tl.push_back(make_int2(i, rb));
    if (st == RLU_OK) st = up(t.trsm_tiles, tt.data(), tt.size() * sizeof(int2));
    if (st == RLU_OK && !tl.empty()) st = up(t.lmul_tiles, tl.data(), tl.size() * sizeof(int2));
  }
  if (mixed && st == RLU_OK) {
    // ring depth: the deepest for one CTA per SM, else a ring that lets two CTAs share an
    // SM when two slots still fit that way
    auto ring = [&](int stage_bytes, int ctas) {
      int d = ctas == 2 ? umma3_stages_for(stage_bytes, 2) : 0;
      if (d < 2) d = umma3_stages_for(stage_bytes, 1);
      return d;
    };
    const int sy = ring(max_stage_y, opt.umma_ctas_y), sc = ring(max_stage_c, opt.umma_ctas_c);
    if (sy < 2 || sc < 2) st = RLU_EUNSUPPORTED;
    for (auto& j : u3y) j.a.stages = sy;
    for (auto& j : u3c) j.a.stages = sc;
    b->u3y_stages = sy;
    b->u3y_stage_bytes = max_stage_y;
    b->u3c_stages = sc;
    b->u3c_stage_bytes = max_stage_c;
    if (st == RLU_OK) st = up(t.u3y, u3y.data(), c * sizeof(U3Job));
    if (st == RLU_OK) st = up(t.u3c, u3c.data(), c * sizeof(U3Job));
    // tile lists: the tiles of one problem next to each other
    std::vector<int2> ty, tc;
    ty.reserve((size_t)t.n_tiles_y);
    tc.reserve((size_t)t.n_tiles_c);
    for (int i = 0; i < count; ++i) {
      for (int mt = 0; mt < (int)ceil_div(problems[i].m, 128); ++mt) ty.push_back(make_int2(i, mt));
      for (int mt = 0; mt < (int)ceil_div(problems[i].n, 128); ++mt) tc.push_back(make_int2(i, mt));
    }
    if (st == RLU_OK) st = up(t.u3y_tiles, ty.data(), ty.size() * sizeof(int2));
    if (st == RLU_OK) st = up(t.u3c_tiles, tc.data(), tc.size() * sizeof(int2));
  }
  if (st != RLU_OK) {
    delete b;
    return st;
  }
  int groups = 0;
  for (int g = 1; g < kLuGroups; ++g) groups += (b->count_y[g] > 0) + (b->count_b[g] > 0);
  int buckets = 0;  // the small-k substitution: one launch per nonempty bucket of k
  for (int bkt = 0; bkt < 4; ++bkt) buckets += b->ts_count[bkt] > 0;
  b->launches = 10 + groups + (t.small_k && buckets > 1 ? buckets - 1 : 0);
  *out = b;
  return RLU_OK;
}

extern "C" int32_t rlu_factor_batched(rlu_batch* b, void* stream) {
  using namespace rlu;
  if (!b) return RLU_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = b->ws;
  const Tables& t = b->t;
  const int c = b->count;
  k_info_init_batched<<<(unsigned)ceil_div(c, 256), 256, 0, s>>>(
      reinterpret_cast<rlu_info* const*>(ws + t.info), c);
  RLU_TRY(last_launch_status());
  RLU_TRY(launch_gaussian_batched(reinterpret_cast<const GaussJob*>(ws + t.gauss), c, s));
  if (b->prec == RLU_PREC_MIXED)
    RLU_TRY(umma3_batched(U3_MODE_Y2, reinterpret_cast<const U3Job*>(ws + t.u3y),
                          reinterpret_cast<const int2*>(ws + t.u3y_tiles), t.n_tiles_y,
                          b->u3y_stages, b->u3y_stage_bytes,
                          reinterpret_cast<unsigned*>(ws + t.u3_counter), s,
                          b->opt.umma_ctas_y != 2));
  else
    RLU_TRY((gemm_simt_batched<float, float>(reinterpret_cast<const GemmArgs*>(ws + t.gemm_y),
                                             c, b->max_m, b->max_l, true, true, false, s,
                                             b->opt.gemm_tile_y)));
  RLU_TRY(launch_lu_reg_batched(false, b->opt.lu_rows_per_cta,
                                reinterpret_cast<const LuArgs*>(ws + t.lu_y), b->first_y,
                                b->count_y, s, b->have_fork ? &b->lu_fork : nullptr));
  RLU_TRY(build_ly_batched(reinterpret_cast<const BuildJob*>(ws + t.build), c, b->max_m,
                           b->max_k, s));
  if (t.small_k)  // the Gram is k x k with k <= 64: one CTA per problem
    RLU_TRY(gram_small_batched(reinterpret_cast<const GemmArgs*>(ws + t.gemm_g), c, s));
  else
    RLU_TRY((gemm_simt_batched<float, double>(reinterpret_cast<const GemmArgs*>(ws + t.gemm_g),
                                              c, b->max_k, b->max_k, true, true, true, s, 1)));
  RLU_TRY(ldl32_batched(reinterpret_cast<const Ldl32Job*>(ws + t.ldl), c, b->max_k, s));
  if (b->prec == RLU_PREC_MIXED)
    RLU_TRY(umma3_batched(U3_MODE_C3, reinterpret_cast<const U3Job*>(ws + t.u3c),
                          reinterpret_cast<const int2*>(ws + t.u3c_tiles), t.n_tiles_c,
                          b->u3c_stages, b->u3c_stage_bytes,
                          reinterpret_cast<unsigned*>(ws + t.u3_counter), s,
                          b->opt.umma_ctas_c != 2));
  else
    RLU_TRY((gemm_simt_batched<float, float>(reinterpret_cast<const GemmArgs*>(ws + t.gemm_c),
                                             c, b->max_k, b->max_n, true, false, true, s,
                                             b->opt.gemm_tile_c)));
  if (t.small_k)
    RLU_TRY(trsm_small_batched(reinterpret_cast<const TrsmJob*>(ws + t.trsm),
                               reinterpret_cast<const int2*>(ws + t.trsm_tiles), b->ts_first,
                               b->ts_count, s));
  else
    RLU_TRY(trsm_batched(reinterpret_cast<const TrsmJob*>(ws + t.trsm),
                         reinterpret_cast<const int2*>(ws + t.trsm_tiles), t.n_tiles_t, b->max_kp,
                         s));
  RLU_TRY(launch_lu_reg_batched(true, b->opt.lu_rows_per_cta,
                                reinterpret_cast<const LuArgs*>(ws + t.lu_b), b->first_b,
                                b->count_b, s, b->have_fork ? &b->lu_fork : nullptr));
  RLU_TRY(gather_batched(reinterpret_cast<const GatherJob*>(ws + t.gather), c, b->max_k,
                         b->max_n, s));
  if (t.small_k)
    RLU_TRY(lmul_batched(reinterpret_cast<const GemmArgs*>(ws + t.gemm_l),
                         reinterpret_cast<const int2*>(ws + t.lmul_tiles), t.n_tiles_l, s));
  else
    RLU_TRY((gemm_simt_batched<float, float>(reinterpret_cast<const GemmArgs*>(ws + t.gemm_l), c,
                                             b->max_m, b->max_k, false, true, false, s,
                                             b->opt.gemm_tile_l)));
  return RLU_OK;
}

extern "C" int32_t rlu_batch_launches(const rlu_batch* b) { return b ? b->launches : 0; }

extern "C" int32_t rlu_batch_destroy(rlu_batch* b) {
  if (!b) return RLU_EINVAL;
  delete b;
  return RLU_OK;
}
