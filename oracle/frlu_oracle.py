"""Plain, slow, complex128 restatement of Algorithm 4 ("Fast Randomized LU Decomposition",
Section 4.1) of Shabat, Shmueli, Aizenbud and Averbuch, "Randomized LU Decomposition":
the Gaussian projection of Algorithm 1 is replaced by the SRFT R = D F S of Section 2
("The SRFT matrix"), and the second pass over A by an interpolative decomposition (ID,
Section 2, "Interpolative decomposition") of Y.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline; never by the product path. Shares no code with the CUDA implementation.

Readings taken here (the paper is silent or loose on each):
  * R = D F S: d_c = exp(2 pi i theta_c) with theta_c uniform on [0, 1) (the uniform
    distribution on the unit circle); F[a, b] = n^{-1/2} exp(-2 pi i a b / n) with 0-based
    indices; S holds a single 1 in each column j, in row s_j, and the s_j are distinct
    (sampling without replacement, so that R has orthonormal columns). The random numbers
    theta (n) and s (l) are inputs drawn by the seeded generator outside this module.
  * Step 3 uses partial pivoting, all l steps, LAPACK zgetf2 semantics: the pivot of step j
    is the first maximum of |Re| + |Im| in the current row order (izamax); a zero pivot
    skips the scaling and is reported.
  * Step 5, the full-rank ID of Y, is taken from the LU of step 3 (Section 2 notes that the
    ID can be computed with LU instead of QR): with P Y = L U, L = [L_1; L_2] (L_1 the
    leading l x l unit lower block), J = (P[0], ..., P[l-1]) and X = P^T [I_l; L_2 L_1^{-1}],
    so that Y = X Y(J,:) holds exactly. The entries of X are not bounded by 2 as those of a
    strong rank-revealing ID are.
  * Step 6, B = L_y^+ P X A(J,:), uses the normal equations of the remark after Algorithm 1
    with the Hermitian Gram: L_y^+ = (L_y^H L_y)^{-1} L_y^H, by a Cholesky factorization.
  * Step 7 is the column-pivoted LU of Algorithm 1 step 6 on complex B: the pivot of step j
    is the first maximum of |Re| + |Im| of row j of the current Schur complement; L_b has
    the unit diagonal.
  * P and Q are gather index vectors: (P A Q)[i, j] = A[P[i], Q[j]]. L and U are complex.

Parity unpinned: none; every function here has a pin in tests/test_oracle_frlu.py.
"""
from __future__ import annotations

import math

import numpy as np


def cabs1(z: np.ndarray) -> np.ndarray:
    """|Re z| + |Im z|, the magnitude LAPACK's complex pivot search (izamax) compares."""
    return np.abs(np.real(z)) + np.abs(np.imag(z))


# ---------------------------------------------------------------------------------------
# Steps 1-2: the SRFT matrix R = D F S (Section 2) and Y = A R.
# ---------------------------------------------------------------------------------------

def srft_matrix(n: int, theta: np.ndarray, s: np.ndarray) -> np.ndarray:
    """R = D F S (n x l), entry by entry from the definition: R[c, j] = d_c F[c, s_j] with
    d_c = exp(2 pi i theta_c) and F[c, b] = n^{-1/2} exp(-2 pi i c b / n). The exponent c b
    is reduced mod n in exact integer arithmetic before the angle is formed."""
    theta = np.asarray(theta, dtype=np.float64)
    s = np.asarray(s, dtype=np.int64)
    if theta.shape != (n,) or s.ndim != 1:
        raise ValueError("theta must have n entries and s must be a vector")
    if s.size and (s.min() < 0 or s.max() >= n or np.unique(s).size != s.size):
        raise ValueError("s must hold distinct indices in [0, n)")
    c = np.arange(n, dtype=np.int64)[:, None]
    e = (c * s[None, :]) % n                                   # c s_j mod n, exact
    F_cols = np.exp(-2j * np.pi * e / n) / math.sqrt(n)        # F[:, s_j]
    d = np.exp(2j * np.pi * theta)
    return d[:, None] * F_cols


def srft_apply(A: np.ndarray, theta: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Step 2 of Algorithm 4: Y = A R, a plain product with the explicit R."""
    A = np.asarray(A)
    return A @ srft_matrix(A.shape[1], theta, s)


# ---------------------------------------------------------------------------------------
# Steps 3 and 7: complex LU with partial (row) and column pivoting.
# ---------------------------------------------------------------------------------------

def clu_partial_pivot(Y: np.ndarray):
    """Step 3: P Y = L_y U_y on a complex copy of Y (m x l), all l steps. Step j: r = first
    index >= j of the largest |Re| + |Im| of Y[:, j] (current row order); if Y[r, j] != 0,
    swap full rows j and r, divide Y[j+1:, j] by Y[j, j] and subtract the outer product from
    Y[j+1:, j+1:]; otherwise record the first zero step. Returns (LU, perm, first_zero) with
    perm in gather form."""
    Y = np.array(Y, dtype=np.complex128, copy=True)
    m, l = Y.shape
    perm = np.arange(m, dtype=np.int64)
    first_zero = -1
    for j in range(min(m, l)):
        r = j + int(np.argmax(cabs1(Y[j:, j])))
        if Y[r, j] != 0:
            if r != j:
                Y[[j, r], :] = Y[[r, j], :]
                perm[[j, r]] = perm[[r, j]]
            Y[j + 1:, j] = Y[j + 1:, j] / Y[j, j]
            Y[j + 1:, j + 1:] -= np.outer(Y[j + 1:, j], Y[j, j + 1:])
        elif first_zero < 0:
            first_zero = j
    return Y, perm, first_zero


def clu_column_pivot(B: np.ndarray):
    """Step 7: B Q = L_b U_b with column pivoting, k steps on complex B (k x n). Step j:
    c = first index >= j of the largest |Re| + |Im| of B[j, j:] (current column order); swap
    columns j and c (of B and of q); if B[j, j] != 0, divide B[j+1:, j] by B[j, j] and
    subtract the outer product from B[j+1:, j+1:]. Returns (L_b, U_b, q, first_zero)."""
    B = np.array(B, dtype=np.complex128, copy=True)
    k, n = B.shape
    q = np.arange(n, dtype=np.int64)
    first_zero = -1
    for j in range(k):
        c = j + int(np.argmax(cabs1(B[j, j:])))
        if c != j:
            B[:, [j, c]] = B[:, [c, j]]
            q[[j, c]] = q[[c, j]]
        if B[j, j] != 0:
            B[j + 1:, j] = B[j + 1:, j] / B[j, j]
            B[j + 1:, j + 1:] -= np.outer(B[j + 1:, j], B[j, j + 1:])
        elif first_zero < 0:
            first_zero = j
    Lb = np.tril(B[:, :k], -1) + np.eye(k)
    Ub = np.triu(B)
    return Lb, Ub, q, first_zero


# ---------------------------------------------------------------------------------------
# Step 5: the full-rank ID Y = X Y(J,:) from the LU of step 3.
# ---------------------------------------------------------------------------------------

def _solve_right_unit_lower(Vm: np.ndarray, L1: np.ndarray) -> np.ndarray:
    """W with W L1 = Vm for a unit lower triangular L1, column by column from the last:
    W[:, b] = Vm[:, b] - sum_{c > b} W[:, c] L1[c, b]."""
    W = np.array(Vm, dtype=np.complex128, copy=True)
    l = L1.shape[0]
    for b in range(l - 1, -1, -1):
        W[:, b] -= W[:, b + 1:] @ L1[b + 1:, b]
    return W


def id_from_lu(Y_lu: np.ndarray, perm: np.ndarray, l: int):
    """J = perm[:l] and X (m x l) with X[perm] = [I_l; L_2 L_1^{-1}], where [L_1; L_2] is the
    unit lower factor of step 3 (strict lower part of Y_lu plus the identity)."""
    m = Y_lu.shape[0]
    Lfull = np.tril(Y_lu[:, :l], -1) + np.eye(m, l)
    L1 = Lfull[:l]
    PX = _solve_right_unit_lower(Lfull, L1)         # P X = L_full L_1^{-1} = [I; L_2 L_1^{-1}]
    X = np.empty_like(PX)
    X[perm] = PX                                    # undo P: row perm[i] of X = row i of P X
    return np.asarray(perm[:l], dtype=np.int64), X


# ---------------------------------------------------------------------------------------
# Step 6: B = L_y^+ (P X A(J,:)) by the normal equations.
# ---------------------------------------------------------------------------------------

def _csolve_lower(Lm, X):
    """Forward substitution, row by row (complex lower triangular Lm)."""
    Z = np.array(X, dtype=np.complex128, copy=True)
    for i in range(Lm.shape[0]):
        Z[i] = (Z[i] - Lm[i, :i] @ Z[:i]) / Lm[i, i]
    return Z


def _csolve_upper(Um, X):
    """Back substitution, row by row (complex upper triangular Um)."""
    Z = np.array(X, dtype=np.complex128, copy=True)
    for i in range(Um.shape[0] - 1, -1, -1):
        Z[i] = (Z[i] - Um[i, i + 1:] @ Z[i + 1:]) / Um[i, i]
    return Z


def cpinv_apply(Ly: np.ndarray, T: np.ndarray) -> np.ndarray:
    """L_y^+ T with M = L_y^H L_y = R^H R (Cholesky), C = L_y^H T, B = R^{-1} (R^{-H} C)."""
    M = Ly.conj().T @ Ly
    Rt = np.linalg.cholesky(M)                      # lower: M = Rt Rt^H
    C = Ly.conj().T @ T
    return _csolve_upper(Rt.conj().T, _csolve_lower(Rt, C))


def check_dims(m: int, n: int, k: int, l: int) -> None:
    """Algorithm 4 input: 1 <= k <= l <= min(m, n)."""
    if not (1 <= k <= l <= min(m, n)):
        raise ValueError(f"need 1 <= k <= l <= min(m, n); got m={m} n={n} k={k} l={l}")


def frlu_factor(A: np.ndarray, k: int, l: int, theta: np.ndarray, s: np.ndarray) -> dict:
    """Algorithm 4, steps 1-9, in complex128 (A real, upcast exactly to FP64). Returns P, Q
    (gather form), L (m x k complex, unit lower trapezoidal), U (k x n complex, upper
    trapezoidal) and the intermediates R, Y, Y_lu, L_y, J, X, B, L_b."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    check_dims(m, n, k, l)
    if len(s) != l:
        raise ValueError("s must hold l indices")
    R = srft_matrix(n, theta, s)                            # step 1
    Y = A @ R                                               # step 2
    Y_lu, P, zero_y = clu_partial_pivot(Y)                  # step 3
    Ly = np.tril(Y_lu[:, :k], -1) + np.eye(m, k)            # step 4: first k columns
    J, X = id_from_lu(Y_lu, P, l)                           # step 5
    PXA = (X @ A[J, :])[P, :]                               # P X A(J,:)
    B = cpinv_apply(Ly, PXA)                                # step 6
    Lb, Ub, Q, zero_b = clu_column_pivot(B)                 # step 7
    L = Ly @ Lb                                             # step 8
    U = Ub                                                  # step 9
    return dict(P=P, Q=Q, L=L, U=U, R=R, Y=Y, Y_lu=Y_lu, Ly=Ly, J=J, X=X, B=B, Lb=Lb,
                first_zero_y=zero_y, first_zero_b=zero_b)


def creconstruct_error(A, P, Q, L, U) -> tuple[float, float]:
    """(||P A Q - L U||_F, ||P A Q - L U||_2) for complex L, U, in complex128."""
    A = np.asarray(A, dtype=np.float64)
    Rm = A[np.asarray(P)][:, np.asarray(Q)] - (np.asarray(L, np.complex128)
                                               @ np.asarray(U, np.complex128))
    fro = float(np.linalg.norm(Rm))
    spec = float(np.linalg.norm(Rm, 2)) if Rm.size else 0.0
    return fro, spec
