// Interface of the cluster LU kernel (see panel_lu.cu).
#pragma once

#include "common.cuh"

namespace rlu {

struct LuArgs {
  void* X;             // R x C column-major, factored in place
  int64_t ldx;         // >= R
  int R, C;            // rows, steps (C <= R)
  int nb;              // panel width (set by the launcher)
  int rpc;             // rows per CTA (set by the launcher)
  int32_t* perm;       // [R] out: row at final position p
  int32_t* zero_step;  // out: first step with a zero pivot, -1 if none (may be NULL)
  int32_t* nonfinite;  // out: OR-ed with 1 when a NaN/Inf is met (may be NULL)
  int32_t* status;     // out: set to RLU_ETIMEOUT if a cluster wait gave up (may be NULL)
  // register kernel only: position state kept between its per-panel launches
  int32_t* posg;       // [R] current position of every row
  int32_t* psg;        // [C] row at each position < C
  int p0;              // first column of the panel of this launch
  int pw;              // its width
  int cu;              // the launch solves the pivot rows of columns [p0 + pw, cu) (0: C)
  void* u12;           // [96][ldu] the solved pivot rows of the current panel or block,
  int64_t ldu;         //   dense (row s = pivot p0 + s), read by the trailing update
  void* u12t;          // FP32 only, may be NULL: [2][96][ldu] floats of scratch; when set,
                       //   the trailing updates run on the tensor cores (three TF32 products)
};

// crout = false: Doolittle (step 3, LU of Y); crout = true: pivot row scaled (step 6 on B^T).
int32_t launch_cluster_lu(int32_t dtype, bool crout, const LuArgs& a, cudaStream_t s);

// Register-resident variant (lu_reg.cu); *launched is false when the shape does not fit it.
// dtype RLU_F64, RLU_F32 or kLuC64 (complex FP32, interleaved (Re, Im) pairs; pivots by
// |Re| + |Im|; the fast randomized LU of Algorithm 4).
static constexpr int32_t kLuC64 = 64;
int32_t launch_lu_reg(int32_t dtype, bool crout, const LuArgs& a, cudaStream_t s, bool* launched);

// Batched FP32 LUs of single-panel problems (C <= 76, R <= 16 x rows_per_cta), one cluster
// each; the device table is grouped (entries first[g] .. first[g] + count[g] - 1; first and
// count are host arrays of kLuGroups entries): g = 1..16 is the cluster size ceil(R /
// rows_per_cta) with rows_per_cta-thread CTAs, g = 17 one 128-thread CTA (R <= 128), g = 18
// one 256-thread CTA (R <= 256). Each entry carries its rpc (rows per CTA), p0 = 0, pw = C
// and its own position state (posg, psg).
static constexpr int kLuGroups = 19;
// Helper streams for the groups: with fork != nullptr every non-empty group is launched on
// its own helper stream (fork / join events around them on s), so that the groups' CTAs
// share the GPU instead of running one launch after another; works under stream capture
// (parallel branches of the graph).
static constexpr int kLuSide = 6;
struct LuFork {
  cudaStream_t hs[kLuSide];
  cudaEvent_t fork;
  cudaEvent_t join[kLuSide];
};
int32_t launch_lu_reg_batched(bool crout, int rows_per_cta, const LuArgs* table_dev,
                              const int* first, const int* count, cudaStream_t s,
                              const LuFork* fork = nullptr);

}  // namespace rlu
