// Interface of the reconstruction-error kernels (see residual.cu).
#pragma once

#include "common.cuh"

namespace rlu {

struct ResidualArgs {
  const void* A;
  int64_t lda;
  const int32_t* P;
  const int32_t* Q;
  const void* L;
  int64_t ldl;
  const void* U;
  int64_t ldu;
  int64_t m, n;
  int k;
};

size_t residual_workspace_bytes(int64_t m, int64_t n, int k);

int32_t residual_error(int32_t dtA, int32_t dtLU, const ResidualArgs& a, double* err_fro,
                       double* err_spec, int iters, double* ws, cudaStream_t s);

}  // namespace rlu
