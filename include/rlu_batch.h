/* Batched form of the randomized LU (Algorithm 1 of "Randomized LU Decomposition", arXiv
 * 1310.7202): many independent factorizations of uneven sizes per launch. The paper has no
 * counterpart; it describes one factorization at a time.
 *
 * A batch plan is made once for a list of problems and a workspace (rlu_batch_create): it
 * computes every problem's workspace layout and writes the per-problem argument records of
 * each step into the workspace. rlu_factor_batched then only enqueues kernels (about a dozen
 * launches for the whole batch, independent of the problem count, no host synchronisation),
 * so it can be captured in a CUDA graph and replayed; each replay factors the current
 * contents of the problems' A into their P, Q, L, U, info.
 *
 * Problems: FP32 storage (RLU_F32), 1 <= k <= l <= min(m, n), l <= 76 (one register panel
 * for each LU), k <= 256, m <= 8192, n <= 8192, at most 65535 problems. Layouts and the
 * meaning of P, Q, L, U, info are those of rlu_factor; the caller owns every buffer.
 * Precision: RLU_PREC_F32 (plain FP32 SIMT products) or RLU_PREC_MIXED (the projection and
 * C = L~^T A on the tensor cores, FP32-accurate TF32 splits; A rows must then start on
 * 16-byte boundaries: lda a multiple of 4 and A 16-byte aligned). */
#ifndef RLU_BATCH_H
#define RLU_BATCH_H

#include <stddef.h>
#include <stdint.h>

#include "rlu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlu_batch rlu_batch;

typedef struct {
  const void* A;
  int64_t m, n, lda;
  int32_t k, l;
  uint64_t seed;
  int32_t* P;
  int32_t* Q;
  void* L;
  int64_t ldl;
  void* U;
  int64_t ldu;
  rlu_info* info;
} rlu_problem;

/* Kernel choices of a batch (the autotuner's knobs; zero-initialised = defaults).
 *   gemm_tile_y, gemm_tile_c, gemm_tile_l: SIMT output tile of the products Y = A G,
 *     C = L~^T A and L = L_y L_b: 0 = 128 x 128, 1 = 64 x 64 (Y and C use the tensor cores
 *     under RLU_PREC_MIXED; their knobs are then ignored; when every k <= 64, L = L_y L_b
 *     runs one thread per row and gemm_tile_l is ignored).
 *   lu_rows_per_cta: rows of an LU held by one CTA of a problem's cluster: 0 or 512 (512
 *     threads), 256 (256 threads, twice the CTAs per problem; m and n <= 4096).
 *   umma_ctas_y, umma_ctas_c: under RLU_PREC_MIXED, CTAs of the tensor-core product Y = A G
 *     (resp. C = L~^T A) meant to share an SM: 0 or 1 (one CTA per SM, which keeps A's TF32
 *     parts in tensor memory, with the deepest staging ring it can hold), 2 (A's parts
 *     through shared memory and a shallower ring, so that two CTAs share the SM; a product
 *     whose two-slot ring does not fit that way keeps one CTA per SM). Ignored under
 *     RLU_PREC_F32. */
typedef struct {
  int32_t gemm_tile_y;
  int32_t gemm_tile_c;
  int32_t gemm_tile_l;
  int32_t lu_rows_per_cta;
  int32_t umma_ctas_y;
  int32_t umma_ctas_c;
} rlu_batch_options;

/* Workspace bytes for the batch (0 if a problem is invalid for the batched form). */
size_t rlu_batch_workspace_size(const rlu_problem* problems, int32_t count, int32_t prec);

/* Plans the batch in the caller's workspace (256-byte aligned, at least
 * rlu_batch_workspace_size bytes) and uploads the argument records (synchronous copies).
 * options may be NULL (defaults). RLU_EINVAL for an invalid problem, option or argument
 * (including a problem too tall for lu_rows_per_cta), RLU_ENOMEM for a small workspace. */
int32_t rlu_batch_create(const rlu_problem* problems, int32_t count, int32_t prec,
                         const rlu_batch_options* options, void* workspace, size_t ws_bytes,
                         rlu_batch** out);

/* Enqueues the whole batch on stream (a cudaStream_t, NULL for the legacy stream). */
int32_t rlu_factor_batched(rlu_batch* batch, void* stream);

/* Kernel launches rlu_factor_batched enqueues for this batch. */
int32_t rlu_batch_launches(const rlu_batch* batch);

int32_t rlu_batch_destroy(rlu_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* RLU_BATCH_H */
