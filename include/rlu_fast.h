/*
 * rlu_fast.h - C ABI of the fast randomized LU (Algorithm 4 of Shabat, Shmueli, Aizenbud and
 * Averbuch, "Randomized LU Decomposition", Section 4.1).
 *
 * Algorithm 4 replaces the Gaussian projection of Algorithm 1 by the subsampled random
 * Fourier transform R = D F S of Section 2 ("The SRFT matrix"), and the second pass over A
 * by an interpolative decomposition of Y ("Interpolative decomposition", Section 2):
 *   1-2  Y = A R (m x l, complex): d_c = exp(2 pi i theta_c), F[a][b] = n^{-1/2}
 *        exp(-2 pi i a b / n), S selects the columns s_0..s_{l-1} of D F;
 *   3-4  P Y = L_y U_y, partial pivoting (pivot: first maximum of |Re| + |Im|, the LAPACK
 *        rule for complex data), all l steps; L_y keeps its first k columns;
 *   5    the full-rank ID Y = X Y(J,:) from that LU: J = P[0..l-1] and
 *        P X = [L_1; L_2] L_1^{-1}, [L_1; L_2] the m x l unit lower factor of step 3;
 *   6    B = L_y^+ P X A(J,:) with L_y^+ = (L_y^H L_y)^{-1} L_y^H (normal equations);
 *   7    B Q = L_b U_b, column pivoting (pivot: first maximum of |Re| + |Im| of the row);
 *   8-9  L = L_y L_b, U = U_b.
 * so that || P A Q - L U || = O(sigma_{k+1}(A)) (the fast randomized LU error theorem,
 * Section 4.1). Only l rows of A are read after the projection.
 *
 * Conventions: those of rlu.h (device pointers owned by the caller, no allocation inside
 * the call, asynchronous on ``stream``, host-side argument checks, device-side conditions in
 * rlu_info, 0-based gather permutations (P A Q)[i][j] = A[P[i]][Q[j]]). Arithmetic is FP32:
 * A is real FP32, row-major (A[i*lda + j], lda >= n); L and U are complex FP32 stored as
 * interleaved (real, imaginary) pairs: L column-major m x k (element (i, t) at pair
 * t*ldl + i, ldl >= m, unit lower trapezoidal), U row-major k x n (pair t*ldu + j,
 * ldu >= n, upper trapezoidal). ldl and ldu count complex elements.
 *
 * The random numbers of R are inputs: theta (n FP32 values in [0, 1), device) and s (l
 * distinct int32 indices in [0, n), device). An index outside [0, n) sets info->status to
 * RLU_EINVAL on the device (the entry is taken as 0); repeated indices are not detected
 * (R then loses its orthonormal columns).
 *
 * Limits (RLU_EUNSUPPORTED beyond them): n <= 16384 with no prime factor other than 2, 3
 * and 5 (the row transform); l <= 512; the rows of Y (m x l) and of B^T (n x k) must fit
 * the shared memory of one CTA per SM, about m * l <= 152 * 27000 (the cooperative LU);
 * 2k within the LDL^T of the normal equations (the real 2k x 2k form of the Hermitian
 * k x k Gram: FP32 LDL^T up to 2k = 512, the FP64 cluster Cholesky of rlu.h's step 5 while
 * its column blocks fit shared memory, about 2k <= 640 on a GB300).
 * Device-side: info->first_zero_pivot_y / _b as in rlu.h; RLU_ETIMEOUT in info->status if a
 * grid barrier of the cooperative LU waits more than 2 s (the launch then ends early).
 */
#ifndef RLU_FAST_H
#define RLU_FAST_H

#include <stddef.h>
#include <stdint.h>

#include "rlu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Steps 1-2 alone: Y = A D F S (m x l complex FP32, row-major, pair i*ldy + j, ldy >= l).
 * Workspace: rlu_srft_workspace_size(n) bytes, 256-byte aligned (0 if n is outside the
 * limits above). The row transforms run one CTA per row of A. */
size_t rlu_srft_workspace_size(int64_t n);
int32_t rlu_srft_apply(const float* A, int64_t m, int64_t n, int64_t lda, const float* theta,
                       const int32_t* s, int32_t l, void* Y, int64_t ldy, rlu_info* info,
                       void* workspace, size_t ws_bytes, void* stream);

/* Workspace bytes for an m x n problem with rank k and l projections (0 if the sizes are
 * invalid, 1 <= k <= l <= min(m, n) violated, or outside the limits above). */
size_t rlu_fast_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l);

/* Algorithm 4 on stream. P (m), Q (n): int32 outputs. L, U: complex FP32 outputs (see
 * above). info: device rlu_info or NULL. workspace: 256-byte aligned, at least
 * rlu_fast_workspace_size bytes. Returns RLU_EINVAL (NULL pointer, leading dimension, sizes,
 * misaligned workspace), RLU_EUNSUPPORTED (limits), RLU_ENOMEM (workspace too small),
 * RLU_ECUDA (a launch failed), else RLU_OK. */
int32_t rlu_fast_factor(const float* A, int64_t m, int64_t n, int64_t lda, int32_t k, int32_t l,
                        const float* theta, const int32_t* s, int32_t* P, int32_t* Q, void* L,
                        int64_t ldl, void* U, int64_t ldu, rlu_info* info, void* workspace,
                        size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RLU_FAST_H */
