// Interface of the SIMT GEMM family (see gemm_simt.cu).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace rlu {

// Kernel arguments (by value).
struct GemmArgs {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  int64_t M, N, K;
  int64_t kchunk;        // K range per split
  int64_t split_stride;  // elements between partial slices
  bool alpha_neg;        // store -A*B instead of A*B
};

// One product C = op(A) * op(B).
//   a_kmajor: A(i, kk) at A[i*lda + kk] (true) or A[kk*lda + i] (false)
//   b_kmajor: B(kk, j) at B[j*ldb + kk] (true) or B[kk*ldb + j] (false)
//   c_rowmajor: C(i, j) at C[i*ldc + j] (true) or C[j*ldc + i] (false)
//   splits > 1: split-K into ``partial`` (splits*M*N elements of the input type), then a
//   fixed-order reduction into C (of the output type).
struct GemmOp {
  const void* A;
  int64_t lda;
  bool a_kmajor;
  const void* B;
  int64_t ldb;
  bool b_kmajor;
  void* C;
  int64_t ldc;
  bool c_rowmajor;
  int64_t M, N, K;
  int splits;
  void* partial;
  bool negate;
};

template <typename T, typename OutT>
int32_t gemm_simt(const GemmOp& op, cudaStream_t s);

template <typename T>
size_t gemm_partial_bytes(int64_t M, int64_t N, int splits);

// Batched products: table_dev[z] (device array of count GemmArgs with kchunk = K and
// split_stride = 0) is problem z; layouts as for GemmOp, the same for every problem;
// max_m / max_n bound the problems' M and N (grid size). tile 0: 128 x 128 output tiles
// (FP32), 1: 64 x 64.
template <typename T, typename OutT>
int32_t gemm_simt_batched(const GemmArgs* table_dev, int count, int64_t max_m, int64_t max_n,
                          bool a_kmajor, bool b_kmajor, bool c_rowmajor, cudaStream_t s,
                          int tile = 0);

int gemm_tile_m(int32_t dtype);
int gemm_tile_n(int32_t dtype);

}  // namespace rlu
