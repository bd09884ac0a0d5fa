// Interface of the small kernels (see small.cu).
#pragma once

#include "common.cuh"

namespace rlu {

template <typename T>
int32_t build_ly(const T* Y, int64_t ldy, int64_t m, int k, const int32_t* perm, T* Lt, T* Lp,
                 int64_t ldl, cudaStream_t s, T* Lhi = nullptr, T* Llo = nullptr);

template <typename T>
int32_t chol_inv(double* M, int k, double* Rinv, T* RinvT, int32_t* status, cudaStream_t s);

template <typename T>
int32_t gather_lb_u(const T* B, int64_t ldb, const int32_t* Q, int k, int64_t n, T* Lb, T* U,
                    int64_t ldu, cudaStream_t s);

template <typename T>
int32_t copy_cm(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                cudaStream_t s);

int32_t info_init(rlu_info* info, cudaStream_t s);

}  // namespace rlu
