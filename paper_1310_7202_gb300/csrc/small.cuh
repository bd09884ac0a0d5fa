// Interface of the small kernels (see small.cu).
#pragma once

#include "common.cuh"

namespace rlu {

// Three BF16 parts (hi + mid + lo) of L~, same layout as L~ (ld ldl); all null when unused.
struct Bf16Parts {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* mid = nullptr;
  __nv_bfloat16* lo = nullptr;
};

// Exact TF32 pairs (hi, lo) and/or three BF16 parts of a column-major FP32 matrix (the
// operands of FP32-accurate tensor-core products), written with ld ldo (0: the input's ld);
// null outputs are skipped.
int32_t split_parts(const float* X, int64_t ld, int64_t rows, int cols, float* hi, float* lo,
                    Bf16Parts bp, cudaStream_t s, int64_t ldo = 0);

template <typename T>
int32_t build_ly(const T* Y, int64_t ldy, int64_t m, int k, const int32_t* perm, T* Lt, T* Lp,
                 int64_t ldl, cudaStream_t s, T* Lhi = nullptr, T* Llo = nullptr,
                 Bf16Parts bp = Bf16Parts{});

// Outputs of the LDL^T factorization M = L D L^T that the triangular solves read, in the
// path's type and zero-padded to kp = 32 * ceil(k / 32) (identity on the padded diagonal):
// L column-major (LT[c * kp + i] = L[i][c]) and row-major (LR[i * kp + c]); the inverses
// W_b of L's 32 x 32 diagonal blocks, row-major (W) and transposed (WT); 1/D (k doubles).
template <typename T>
struct LdlOut {
  T* LT;
  T* LR;
  T* W;
  T* WT;
  double* dinv;
  int k;
  int kp;
};

// M (k x k FP64, row-major; overwritten) = L D L^T.
template <typename T>
int32_t ldl_factor(double* M, int k, const LdlOut<T>& o, int32_t* status, cudaStream_t s);

// Whether ldl_factor handles a k x k Gram (FP32 outputs: f32).
bool ldl_factor_supported(int k, bool f32);

// B (k x n, row-major) = L^{-T} D^{-1} L^{-1} C (C k x n row-major). narrow: 32 columns per
// CTA (twice the CTAs of the default 64, for right-hand sides too few to fill the GPU).
template <typename T>
int32_t trsm_ldl(const LdlOut<T>& o, const T* C, int64_t ldc, int64_t n, T* B, int64_t ldb,
                 cudaStream_t s, bool narrow = false);

template <typename T>
int32_t gather_lb_u(const T* B, int64_t ldb, const int32_t* Q, int k, int64_t n, T* Lb, T* U,
                    int64_t ldu, cudaStream_t s);

template <typename T>
int32_t copy_cm(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                cudaStream_t s);

int32_t info_init(rlu_info* info, cudaStream_t s);

}  // namespace rlu
