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
//  * the array's device address is looked up (cudaGetSymbolAddress, with the device
//    current) on the first call in each CUDA context of a device and cached together with
//    that context's id; a later call in another context (after cudaDeviceReset, or once
//    the primary context was released and created again) looks it up again. A lookup is
//    never made while the caller's stream is capturing: such a call returns RLU_EINVAL,
//    so make the first call on a device (and the first after a reset) outside any stream
//    capture;
//  * problems whose scratch need exceeds kStaticScratchBytes are rejected with RLU_ENOMEM
//    before anything is enqueued;
//  * all calls share the one array and it keeps the previous call's contents; the kernels
//    write every scratch word before reading it, so nothing needs clearing; calls that
//    overlap on the GPU (different streams, no ordering between them) race on the array.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "residual.cuh"

namespace rlu {

static constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Id of the CUDA context current on this thread (0 when none is current, or when the
// driver does not export cuCtxGetId). Resolved through the runtime's driver entry points,
// so the library does not link the driver library itself.
static unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    cudaGetLastError();  // a symbol this driver lacks is not an error of the caller's
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_static_scratch in the current device's current context. Cached per
// device together with the context id it was found in; looked up again when the context
// changed (never during a capture on s).
static int32_t static_scratch(cudaStream_t s, void** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  static unsigned long long ctx_of[64] = {0};
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RLU_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long ctx = current_context_id();
  if (addr[dev] != nullptr && ctx != 0 && ctx == ctx_of[dev]) {
    *out = addr[dev];
    return RLU_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();  // leave no sticky error behind for the caller's next call
    return RLU_ECUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return RLU_EINVAL;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return RLU_ECUDA;
  }
  addr[dev] = p;
  ctx_of[dev] = current_context_id();  // the lookup made the primary context current
  *out = p;
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
  RLU_TRY(static_scratch((cudaStream_t)stream, &scratch));
  ResidualArgs a{A, lda, P, Q, L, ldl, U, ldu, m, n, k};
  return residual_error(dtype, lu_dtype, a, err_fro, err_spec, power_iters,
                        static_cast<double*>(scratch), (cudaStream_t)stream);
}
