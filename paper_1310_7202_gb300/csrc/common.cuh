// Shared device/host helpers of the sm_103a randomized LU library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rlu.h"

namespace rlu {

#define RLU_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return RLU_ECUDA;                 \
  } while (0)

#define RLU_TRY(expr)                                        \
  do {                                                       \
    int32_t _s = (expr);                                     \
    if (_s != RLU_OK) return _s;                             \
  } while (0)

// Counts every kernel launch of the library (read by rlu_launch_count).
void note_launches(int count);

inline int32_t last_launch_status(int launches = 1) {
  note_launches(launches);
  return cudaGetLastError() == cudaSuccess ? RLU_OK : RLU_ECUDA;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

template <typename T> struct dtype_of;
template <> struct dtype_of<double> { static constexpr int32_t value = RLU_F64; };
template <> struct dtype_of<float> { static constexpr int32_t value = RLU_F32; };

// Number of SMs of the current device (cached per device ordinal).
int sm_count();

// Pivot-search candidate: larger |value| wins; equal magnitudes go to the smaller current
// position (the getf2 / i?amax "first maximum" rule). A NaN magnitude never wins.
template <typename T>
struct Cand {
  T mag;      // |value|, -1 when the candidate is empty
  int pos;    // current position of the row
  int row;    // row index (global)
};

template <typename T>
__device__ __forceinline__ bool cand_better(T mag_a, int pos_a, T mag_b, int pos_b) {
  return (mag_a > mag_b) || (mag_a == mag_b && pos_a < pos_b);
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T& mag, int& pos, int& row) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    T om = __shfl_xor_sync(0xffffffffu, mag, off);
    int op = __shfl_xor_sync(0xffffffffu, pos, off);
    int orow = __shfl_xor_sync(0xffffffffu, row, off);
    if (cand_better(om, op, mag, pos)) {
      mag = om;
      pos = op;
      row = orow;
    }
  }
}

__device__ __forceinline__ bool is_finite_val(double x) { return isfinite(x); }
__device__ __forceinline__ bool is_finite_val(float x) { return isfinite(x); }

// Complex FP32 element of the register LU (same memory layout as float2): arithmetic with
// fused multiply-adds, so that the LU's templates run on it as on float and double.
struct __align__(8) cf32 {
  float x, y;
  cf32() = default;
  __host__ __device__ constexpr cf32(float r) : x(r), y(0.f) {}
  __host__ __device__ constexpr cf32(float r, float i) : x(r), y(i) {}
};
__device__ __forceinline__ cf32 operator-(cf32 a) { return cf32(-a.x, -a.y); }
__device__ __forceinline__ cf32 operator*(cf32 a, cf32 b) {
  return cf32(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ bool operator!=(cf32 a, cf32 b) { return a.x != b.x || a.y != b.y; }
__device__ __forceinline__ bool operator==(cf32 a, cf32 b) { return a.x == b.x && a.y == b.y; }
// a b + c (the float and double overloads stay visible beside it)
using ::fma;
__device__ __forceinline__ cf32 fma(cf32 a, cf32 b, cf32 c) {
  return cf32(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ bool is_finite_val(cf32 v) { return isfinite(v.x) && isfinite(v.y); }

}  // namespace rlu
