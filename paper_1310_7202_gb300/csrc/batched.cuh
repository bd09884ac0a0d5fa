// Per-problem argument records of the batched kernels (one device array per step, built on
// the host by the batch plan in batched.cu; entry z is problem z unless stated otherwise).
#pragma once

#include "common.cuh"
#include "gemm_simt.cuh"
#include "small.cuh"

namespace rlu {

struct GaussJob {  // step 1: G (n x l, column-major, ld ldg) from the problem's seed
  uint64_t seed;
  int64_t n, l;
  float* G;
  int64_t ldg;
};

struct BuildJob {  // step 4: L_y (pivot order, Lp) and L~ = P^T L_y (Lt), both m x k, ld ldl;
                   // with Lhi non-null also L~'s exact TF32 split (Lhi + Llo)
  const float* Y;
  int64_t ldy, m;
  int k;
  const int32_t* perm;
  float* Lt;
  float* Lp;
  int64_t ldl;
  float* Lhi;
  float* Llo;
};

struct Ldl32Job {  // step 5: M (k x k FP64) = L D L^T on one CTA
  const double* M;
  int k;
  LdlOut<float> o;
  int32_t* status;
};

struct TrsmJob {  // step 5: B = L^{-T} D^{-1} L^{-1} C (k x n, row-major)
  LdlOut<float> o;
  const float* C;
  int64_t ldc, n;
  float* B;
  int64_t ldb;
};

struct GatherJob {  // steps 6-8: L_b (k x k, column-major) and U (k x n, row-major)
  const float* B;
  int64_t ldb;
  const int32_t* Q;
  int k;
  int64_t n;
  float* Lb;
  float* U;
  int64_t ldu;
};

int32_t launch_gaussian_batched(const GaussJob* jobs_dev, int count, cudaStream_t s);
int32_t build_ly_batched(const BuildJob* jobs_dev, int count, int64_t max_m, int max_k,
                         cudaStream_t s);
int32_t ldl32_batched(const Ldl32Job* jobs_dev, int count, int max_k, cudaStream_t s);
// over a tile list of (problem, 64-column block) pairs
int32_t trsm_batched(const TrsmJob* jobs_dev, const int2* tiles_dev, int ntiles, int max_kp,
                     cudaStream_t s);
int32_t gather_batched(const GatherJob* jobs_dev, int count, int max_k, int64_t max_n,
                       cudaStream_t s);
// k <= 64: the substitution one thread per column over (problem, 128-column block) tiles,
// grouped by the bucket of k (trsm_small_bucket: 0..3 for k <= 16, 32, 48, 64; tiles of
// bucket b at first[b] .. first[b] + count[b] - 1, one launch per nonempty bucket), and
// L = L_y L_b one thread per row over (problem, 256-row block) tiles
int trsm_small_bucket(int k);
int32_t trsm_small_batched(const TrsmJob* jobs_dev, const int2* tiles_dev, const int* first,
                           const int* count, cudaStream_t s);
int32_t lmul_batched(const GemmArgs* jobs_dev, const int2* tiles_dev, int ntiles, cudaStream_t s);
// k <= 64: the Gram M = L~^T L~ (FP64 out, FP32 accumulation), one CTA per problem
int32_t gram_small_batched(const GemmArgs* jobs_dev, int count, cudaStream_t s);

}  // namespace rlu
