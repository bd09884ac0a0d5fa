// Fixed-scratch variant of rlu_reconstruct_error.
//
// Some callers cannot allocate device memory themselves: code that runs inside a host
// framework which owns every byte of the device through its own memory pool, or a latency-
// critical path where a cudaMalloc/cudaFree (which may synchronise the device) is not
// allowed. rlu_reconstruct_error_static lets them measure ||P A Q - L U|| without passing a
// workspace: its scratch is the file-scope array below, which every GPU that loads this
// library holds until the process exits.
//
// Properties a caller relies on:
//  * no cudaMalloc, cudaFree or other allocating call is made;
//  * the first call on a device looks up the array's device address (cudaGetSymbolAddress,
//    with that device current) and caches it; make that first call before any stream
//    capture;
//  * problems whose scratch need exceeds kStaticScratchBytes are rejected with RLU_ENOMEM
//    before anything is enqueued;
//  * all calls share the one array and it keeps the previous call's contents; the kernels
//    write every scratch word before reading it, so nothing needs clearing; calls that
//    overlap on the GPU (different streams, no ordering between them) race on the array.
#include <mutex>

#include "common.cuh"
#include "residual.cuh"

namespace rlu {

static constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device (looked up once per device).
static int32_t static_scratch(void** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RLU_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
      return RLU_ECUDA;
    addr[dev] = p;
  }
  *out = addr[dev];
  return RLU_OK;
}

}  // namespace rlu

extern "C" int32_t rlu_reconstruct_error_static(const void* A, int32_t dtype, int64_t m,
                                                int64_t n, int64_t lda, int32_t k,
                                                const int32_t* P, const int32_t* Q,
                                                const void* L, int64_t ldl, const void* U,
                                                int64_t ldu, int32_t lu_dtype, double* err_fro,
                                                double* err_spec, int32_t power_iters,
                                                void* stream) {
  using namespace rlu;
  if (!A || !P || !Q || !L || !U || !err_fro) return RLU_EINVAL;
  if (m < 1 || n < 1 || k < 1 || lda < n || ldl < m || ldu < n || power_iters < 0)
    return RLU_EINVAL;
  if (residual_workspace_bytes(m, n, k) > kStaticScratchBytes) return RLU_ENOMEM;
  void* scratch = nullptr;
  RLU_TRY(static_scratch(&scratch));
  ResidualArgs a{A, lda, P, Q, L, ldl, U, ldu, m, n, k};
  return residual_error(dtype, lu_dtype, a, err_fro, err_spec, power_iters,
                        static_cast<double*>(scratch), (cudaStream_t)stream);
}
