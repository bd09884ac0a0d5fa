/*
 * rlu.h - C ABI of the GB300 (sm_103a) randomized LU library.
 *
 * The library computes the randomized LU decomposition of Algorithm 1 of Shabat, Shmueli,
 * Aizenbud and Averbuch, "Randomized LU Decomposition" (Section 4): for an m x n matrix A
 * and integers k <= l it returns row and column permutations P, Q, a unit lower
 * trapezoidal L (m x k) and an upper trapezoidal U (k x n) with
 *     || P A Q - L U || = O(sigma_{k+1}(A))            (Eq. lu_error and theorem trm:rand_lu_err, Section 4).
 *
 * Conventions shared by every entry point
 *   - All matrix and vector pointers are DEVICE pointers owned by the caller. The library
 *     never allocates device memory inside a call; scratch space is the caller's
 *     ``workspace`` buffer, sized by the matching *_workspace_size() query.
 *   - ``stream`` is a cudaStream_t passed as void* (NULL = the legacy default stream). Every
 *     call only enqueues work on that stream (and on library-owned helper streams that
 *     fork from and join back into it) and returns without synchronising.
 *   - Argument errors are detected on the host and returned synchronously; nothing is
 *     enqueued then. Conditions found on the device (zero pivots, NaN/Inf) are written to
 *     the caller's device-resident rlu_info.
 *   - Permutations are 0-based gather vectors: (P A Q)[i][j] = A[P[i]][Q[j]].
 *   - A is row-major (element (i, j) at A[i*lda + j], lda >= n). L is column-major
 *     (element (i, t) at L[t*ldl + i], ldl >= m). U is row-major (U[t*ldu + j], ldu >= n).
 *   - Steps 1-8 below refer to the steps of Algorithm 1.
 */
#ifndef RLU_H
#define RLU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RLU_OK = 0,
  RLU_EINVAL = 1,        /* an argument is out of range, NULL or misaligned */
  RLU_ENOMEM = 2,        /* workspace smaller than *_workspace_size() */
  RLU_EUNSUPPORTED = 3,  /* dtype / precision combination not provided */
  RLU_ECUDA = 4,         /* a CUDA runtime call failed (launch, attribute, event) */
  RLU_ETIMEOUT = 5       /* device side only (rlu_info.status): a wait between the CTAs of
                            a cluster gave up after about one second; results are invalid */
} rlu_status;

typedef enum { RLU_F64 = 0, RLU_F32 = 1, RLU_BF16 = 2 } rlu_dtype;

/* Arithmetic of the whole path. In every precision the pseudo-inverse product of step 5
 * solves the normal equations M B = C with M = L~^T L~ reduced in FP64 and factored as
 * L D L^T (FP64 for RLU_PREC_F64 and for k > 256; FP32 otherwise), followed by blocked
 * triangular solves in the path's type.
 *   RLU_PREC_F64: A, G, Y, B, L, U in FP64, FP64 arithmetic everywhere. A must be RLU_F64.
 *   RLU_PREC_F32: "plain FP32". A, G, Y, B, L, U in FP32; FP32 SIMT GEMMs and LUs.
 *                 A must be RLU_F32.
 *   RLU_PREC_MIXED: as RLU_PREC_F32, but the three large products run on the tensor cores
 *                 from exact TF32 splits, FP32-accurate: Y = A G as hi(A) G + lo(A) G (G is
 *                 rounded to TF32, which only changes the Gaussian test matrix), the Gram
 *                 matrix and C = L~^T A with three products each. A must be RLU_F32. The
 *                 tensor-core products read A with TMA, which needs 16-byte aligned rows
 *                 (A aligned, lda a multiple of 4); otherwise they run on the FP32 SIMT
 *                 GEMM.
 *   RLU_PREC_BF16: the precision form for A stored in BF16 (A must be RLU_BF16, 16-byte
 *                 aligned, lda a multiple of 8, else RLU_EINVAL). G is generated in BF16 and
 *                 Y = A G runs on the BF16 tensor cores with FP32 accumulation; C = L~^T A
 *                 takes L~ in three BF16 parts (hi + mid + lo, FP32 accurate) against the
 *                 exact BF16 A; Y, L~, the Gram matrix (TF32 splits as in RLU_PREC_MIXED), the
 *                 LUs, L and U are FP32 (L and U are returned in FP32).
 *   RLU_PREC_FP8: as RLU_PREC_BF16, but Y = A G runs in FP8 e4m3 with per-tile power-of-two
 *                 (UE8M0) scales: A is quantised with one scale per row and 128-column
 *                 block (1 x 128 tiles), G with one scale per 128 x 128 block, each scale the
 *                 smallest power of two that keeps the tile's largest magnitude within e4m3's
 *                 448 (round to nearest even); the tensor cores apply the scales
 *                 (block-scaled MMA) and accumulate in FP32. The workspace adds the e4m3 A
 *                 (m x 128*ceil(n/128) bytes), G and the scales. E4m3 keeps 4 significant
 *                 bits, so A's quantisation adds about 3% relative noise to every entry: the
 *                 range finder tolerates it only while that noise stays well below
 *                 sigma_{k+1} (it does not at 32768 x 16384 with sigma_i = 0.99^i, k = 512). */
typedef enum {
  RLU_PREC_F64 = 0,
  RLU_PREC_F32 = 1,
  RLU_PREC_MIXED = 2,
  RLU_PREC_BF16 = 3,
  RLU_PREC_FP8 = 4
} rlu_precision;

/* Device-resident status written by rlu_factor (the caller reads it after the stream
 * completes). */
typedef struct {
  int32_t status;              /* RLU_OK, or a device-detected failure code            */
  int32_t first_zero_pivot_y;  /* first step of the LU of Y (step 3) with a zero pivot,
                                  -1 if none (not an error: getrf semantics)            */
  int32_t first_zero_pivot_b;  /* same for the column-pivoted LU of B (step 6)          */
  int32_t nonfinite;           /* nonzero if a NaN or Inf met a pivot search            */
} rlu_info;

/* Library version (major*10000 + minor*100 + patch). */
int32_t rlu_version(void);

/* Short static string for a status code. */
const char* rlu_status_string(int32_t status);

/* Raw Philox4x32-10 stream behind step 1 (Salmon et al., SC'11): for c = 0..n_counters-1
 * writes the four output words of counter index (first_counter + c) to out[4c .. 4c+3].
 * Counter words = (index lo32, index hi32, stream_id, 0); key = (seed lo32, seed hi32).
 * out: device, 4*n_counters uint32. Errors: RLU_EINVAL if out is NULL or n_counters < 0. */
int32_t rlu_philox_u32(uint64_t seed, uint32_t stream_id, uint64_t first_counter,
                       int64_t n_counters, uint32_t* out, void* stream);

/* Step 1: the Gaussian matrix G (n x l, column-major, ldg >= n) with i.i.d. N(0,1) entries.
 * Entry (i, j) is element e = j*n + i of the stream; counter e/4 gives elements
 * 4c..4c+3 as two Box-Muller pairs (x0,x1) and (x2,x3). dtype RLU_F64: the FP64 transform
 * (u = (x0+1)/2^32, series logarithm and sine/cosine in IEEE-rounded FP64 operations);
 * RLU_F32: the same transform in FP32 operations on u = (floor(x0/2^8)+1)/2^24 and the
 * top 27 bits of x1; RLU_BF16: the FP32 value rounded to nearest even.
 * Errors: RLU_EINVAL on NULL G, n or l < 0, or ldg < n. */
int32_t rlu_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, int64_t l,
                     int32_t dtype, void* G, int64_t ldg, void* stream);

/* Bytes of workspace rlu_factor needs for these sizes and precision (0 if invalid). */
size_t rlu_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l, int32_t prec);

/* Algorithm 1, steps 1-8: randomized LU of A (m x n, row-major, lda >= n).
 *   k, l      : 1 <= k <= l <= min(m, n) (Algorithm 1 input; l <= min(m, n) as in the
 *               lemmas behind theorem trm:rand_lu_err).
 *   seed      : Philox key for G (stream id 0).
 *   P (m), Q (n): int32 gather permutations (outputs).
 *   L (m x k, column-major, ldl >= m), U (k x n, row-major, ldu >= n): outputs, FP64 for
 *               RLU_PREC_F64 and FP32 for RLU_PREC_F32.
 *   info      : device rlu_info (output; may be NULL).
 *   workspace : device scratch of at least rlu_workspace_size() bytes, 256-byte aligned.
 * Step 3 is LU with partial pivoting over all l columns (getf2 tie rule: first maximum in
 * the current row order); step 5 uses the normal equations
 * L_y^+ = (L_y^T L_y)^{-1} L_y^T (remark after Algorithm 1) with an LDL^T (Cholesky)
 * factorization of the k x k Gram matrix: FP64 for RLU_PREC_F64 and for k > 512, FP32 on
 * the single-precision paths otherwise; step 6 pivots on the largest entry of row j of the
 * current Schur complement and keeps the unit diagonal on L_b.
 * Errors: RLU_EINVAL (dimensions, NULL pointers, strides), RLU_EUNSUPPORTED (dtype does
 * not match prec), RLU_ENOMEM (workspace too small), RLU_ECUDA (launch failure). */
int32_t rlu_factor(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                   int32_t k, int32_t l, uint64_t seed, int32_t prec,
                   int32_t* P, int32_t* Q, void* L, int64_t ldl, void* U, int64_t ldu,
                   rlu_info* info, void* workspace, size_t ws_bytes, void* stream);

/* Optional copies of the intermediates of Algorithm 1, for verification, and optional
 * per-step timing events. Every pointer may be NULL; types follow the path (FP64 or FP32).
 *   G  : n x l column-major (ld n)      step 1
 *   Y  : m x l column-major (ld m)      step 2, before the LU
 *   Ly : m x k column-major (ld m)      step 4, unit lower trapezoidal, pivot row order
 *   B  : k x n row-major    (ld n)      step 5, before its LU
 *   events: 2*RLU_NUM_TIMED_STEPS caller-created cudaEvent_t handles (as void*); when
 *           n_events is large enough, events[2i] and events[2i+1] are recorded right before
 *           and after timed step i, on the stream that runs it (see rlu_timed_step_name). */
typedef struct {
  void* G;
  void* Y;
  void* Ly;
  void* B;
  void** events;
  int32_t n_events;
} rlu_stage_outputs;

/* Timed steps of rlu_factor_stages, in order: 0 gaussian (step 1), 1 Y = A G (step 2),
 * 2 LU of Y (step 3), 3 L_y / L~ (step 4), 4 Gram (step 5), 5 Cholesky + inverse (step 5,
 * helper stream), 6 C = L~^T A (step 5), 7 B = R^-1 R^-T C (step 5), 8 LU of B (step 6),
 * 9 L_b / U gathers (steps 6, 8), 10 L = L_y L_b (step 7). */
#define RLU_NUM_TIMED_STEPS 11

/* Name of timed step i (static string), or NULL when out of range. */
const char* rlu_timed_step_name(int32_t i);

/* Number of kernels this library has enqueued since it was loaded (host-side counter,
 * all devices and threads). */
uint64_t rlu_launch_count(void);

/* rlu_factor that also writes the intermediates named in ``stages`` (may be NULL, then it
 * is rlu_factor). Same arguments, errors and workspace. */
int32_t rlu_factor_stages(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                          int32_t k, int32_t l, uint64_t seed, int32_t prec,
                          int32_t* P, int32_t* Q, void* L, int64_t ldl, void* U,
                          int64_t ldu, rlu_info* info, void* workspace, size_t ws_bytes,
                          const rlu_stage_outputs* stages, void* stream);

/* Power iterations (Section 5, "Power Iterations"): step 2 becomes
 * Y = (A A^T)^q A G, applied as q rounds of Z = A^T Y, Y = A Z.
 *   normalized = 0: unnormalised rounds, as the paper states them for small q. The scale of
 *              the top singular direction grows like sigma_1^(2q+1) against the others, so
 *              directions below (sigma_{k+1}/sigma_1)^(2q+1) of it drown in the rounding of
 *              the path's type (FP32: already at q = 1 for sigma_i = i^-2 and k = 200).
 *   normalized = 1: the normalised scheme the paper refers to for larger q, read as LU
 *              normalisation: before each product the block (Y, then Z) is factored with
 *              partial pivoting and replaced by P^T L (its unit lower factor with the rows
 *              put back). This multiplies the block on the right by an upper triangular
 *              matrix, so the column space, and in exact arithmetic the pivots and factors
 *              of steps 3-8, are those of the unnormalised rounds; each round costs two
 *              more pivoted LUs (m x l and n x l).
 * The products of the rounds are FP32 accurate on RLU_PREC_MIXED (three TF32 products) and
 * RLU_PREC_BF16 (three BF16 products against the exact BF16 A); plain FP32 / FP64 SIMT
 * otherwise. 0 <= q <= 16 (q = 0 is rlu_factor_stages). The normalisation LUs use P and Q
 * as scratch before the factorization writes them. Workspace: rlu_workspace_size_power
 * (either value of normalized), which adds Z (n x l), the normalised block and the splits
 * of Y and Z to rlu_workspace_size. Other arguments, outputs and errors as
 * rlu_factor_stages; RLU_EINVAL also for q outside [0, 16] or normalized not 0 or 1. */
size_t rlu_workspace_size_power(int64_t m, int64_t n, int32_t k, int32_t l, int32_t prec,
                                int32_t q);
int32_t rlu_factor_power(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                         int32_t k, int32_t l, uint64_t seed, int32_t prec, int32_t q,
                         int32_t normalized, int32_t* P, int32_t* Q, void* L, int64_t ldl,
                         void* U, int64_t ldu, rlu_info* info, void* workspace,
                         size_t ws_bytes, const rlu_stage_outputs* stages, void* stream);

/* Algorithm 3 (Section 5, "Rank Deficient Least Squares"): x minimising ||A x - b|| from
 * the factors of Algorithm 1 (A ~ P^T L U Q^T): c = P b (c[i] = b[P[i]]), y = L^+ c by the
 * normal equations (FP64 Gram, the LDL^T and blocked substitution of step 5),
 * z_1 = U_1^{-1} y with U_1 = U[:, 0:k], z = (z_1, 0), x = Q z (x[Q[j]] = z[j]): x has at
 * most k nonzero entries.
 *   dtype      : RLU_F32 or RLU_F64, the type of L, U, b and x (as rlu_factor wrote them).
 *   P (m), Q (n), L (m x k, column-major, ldl >= m), U (k x n, row-major, ldu >= n): the
 *              factors, device memory, unchanged.
 *   b          : m x nrhs column-major (ldb >= m); x: n x nrhs column-major (ldx >= n),
 *                output. nrhs >= 1.
 *   info       : device rlu_info (may be NULL): status RLU_EINVAL if L^T L is not positive
 *                definite; first_zero_pivot_b = a zero diagonal entry of U_1 (that entry
 *                of z_1 is set to 0).
 *   workspace  : rlu_lstsq_workspace_size bytes, 256-byte aligned.
 * Errors: RLU_EINVAL (NULL pointers, strides, k outside [1, min(m, n)]), RLU_EUNSUPPORTED
 * (dtype, k > 4096), RLU_ENOMEM, RLU_ECUDA. Asynchronous on stream. */
size_t rlu_lstsq_workspace_size(int64_t m, int64_t n, int32_t k, int32_t nrhs, int32_t dtype);
int32_t rlu_lstsq(int32_t dtype, int64_t m, int64_t n, int32_t k, const int32_t* P,
                  const int32_t* Q, const void* L, int64_t ldl, const void* U, int64_t ldu,
                  const void* b, int64_t ldb, int32_t nrhs, void* x, int64_t ldx,
                  rlu_info* info, void* workspace, size_t ws_bytes, void* stream);

/* Algorithm 2 (alg:randomized_orth, Section 4.3): the randomized range finder with an
 * orthogonal basis, the accuracy comparator ("randomized SVD") of the error experiment of
 * Section 5. Step 1 draws G (n x l) as step 1 of Algorithm 1 does (FP64 transform, stream
 * id 0), step 2 forms Y = A G, step 3 takes the left singular vectors of Y from the
 * eigenpairs of the FP64 Gram matrix Y^T Y (parallel cyclic Jacobi: U_y = Y V diag(lambda)^-1/2),
 * step 4 keeps the k with the largest singular values: Q (m x k, column-major, ldq >= m,
 * orthonormal columns). Also returns B = Q^T A (k x n, row-major, ldb >= n), so that
 * ||Q B - A|| = ||Q Q^T A - A|| is the comparator's rank-k error (rlu_reconstruct_error
 * with identity permutations, L = Q, U = B), and sigma (l doubles, may be NULL): the
 * singular values of Y in decreasing order.
 *   dtype: RLU_F64 only (the comparison runs in double precision, as the paper's does).
 *   1 <= k <= l <= min(m, n), l <= 4096.
 *   info: device rlu_info (may be NULL): status RLU_EINVAL when Y has fewer than k singular
 *         values above the resolution of the Gram route (an eigenvalue of Y^T Y at or below
 *         64 eps lambda_max, i.e. sigma_j(Y) below about 1e-7 sigma_1(Y), is rounding noise:
 *         its sigma is returned as 0 and its column of Q is zero); RLU_ETIMEOUT when a grid
 *         barrier of the eigensolver gave up.
 *   workspace: rlu_rsvd_workspace_size bytes, 256-byte aligned.
 * Errors: RLU_EINVAL (dimensions, NULL pointers, strides), RLU_EUNSUPPORTED (dtype),
 * RLU_ENOMEM, RLU_ECUDA. Asynchronous on stream. */
size_t rlu_rsvd_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l);
int32_t rlu_rsvd(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                 int32_t l, uint64_t seed, void* Q, int64_t ldq, void* B, int64_t ldb,
                 double* sigma, rlu_info* info, void* workspace, size_t ws_bytes,
                 void* stream);

/* Bytes of workspace rlu_reconstruct_error needs. */
size_t rlu_reconstruct_workspace_size(int64_t m, int64_t n, int32_t k);

/* Error of Eq. (1) / Eq. (relErr): R = P A Q - L U with A (m x n) of ``dtype`` and L, U of
 * ``lu_dtype`` (layouts as in rlu_factor). Writes ||R||_F to err_fro[0] (FP64 sum of
 * squares of residuals formed in FP64 from the stored values) and, if err_spec is not NULL,
 * a power-iteration estimate of ||R||_2 after ``power_iters`` steps of x <- R^T R x from a
 * fixed start vector (a lower bound that converges to ||R||_2) to err_spec[0].
 * err_fro, err_spec: device doubles. Errors: RLU_EINVAL, RLU_EUNSUPPORTED, RLU_ENOMEM. */
int32_t rlu_reconstruct_error(const void* A, int32_t dtype, int64_t m, int64_t n,
                              int64_t lda, int32_t k, const int32_t* P, const int32_t* Q,
                              const void* L, int64_t ldl, const void* U, int64_t ldu,
                              int32_t lu_dtype, double* err_fro, double* err_spec,
                              int32_t power_iters, void* workspace, size_t ws_bytes,
                              void* stream);

/* rlu_reconstruct_error without a workspace argument. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory themselves (a host
 * framework that owns all device memory through its own pool, or a path where a cudaMalloc
 * or cudaFree would synchronise the device). Its scratch is a fixed 8 MiB array in the
 * library's device memory, present on every GPU that loads the library until the process
 * exits; it makes no allocating call. The first call in a device's CUDA context looks up
 * that array's address (with the device current) and caches it with the context's id; a
 * call in a new context (after cudaDeviceReset, or once the primary context was released
 * and created again) looks it up again. No lookup is made while ``stream`` is capturing:
 * that call returns RLU_EINVAL, so make the first call on a device, and the first after a
 * reset, outside any stream capture. Problems needing
 * more than 8 MiB of scratch (rlu_reconstruct_workspace_size() > 8 MiB) return RLU_ENOMEM
 * before anything is enqueued. All calls share the array: calls that overlap on the GPU
 * race, so order them (one stream, or events). Other arguments, outputs and errors as in
 * rlu_reconstruct_error. */
int32_t rlu_reconstruct_error_static(const void* A, int32_t dtype, int64_t m, int64_t n,
                                     int64_t lda, int32_t k, const int32_t* P,
                                     const int32_t* Q, const void* L, int64_t ldl,
                                     const void* U, int64_t ldu, int32_t lu_dtype,
                                     double* err_fro, double* err_spec, int32_t power_iters,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RLU_H */
