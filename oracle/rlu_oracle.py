"""Plain, slow, FP64 restatement of Algorithm 1 ("Randomized LU Decomposition") of
Shabat, Shmueli, Aizenbud and Averbuch, plus the error measures of Eq. (1) / Eq. (relErr)
and the bound of the error theorem of Section 4 (trm:rand_lu_err).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline; never by the product path. Shares no code with the CUDA implementation.

Readings of the paper taken here (the paper is silent or loose on each):
  * Step 1 random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
    seed, one 128-bit counter per four consecutive entries of G in column-major order, and a
    Box-Muller transform whose logarithm and sine/cosine are evaluated by fixed series with
    IEEE-rounded +,-,*,/ only, so that every implementation that performs the same
    operations produces the same doubles.
  * Step 3 uses partial pivoting (the remark after Algorithm 1), all l steps, LAPACK getf2
    semantics: the pivot is the first maximum |value| in the current row order; a zero
    pivot skips the scaling and is reported.
  * Step 5 uses the normal equations of the remark after Algorithm 1:
    L_y^+ = (L_y^T L_y)^{-1} L_y^T, with a Cholesky factorization of the k x k Gram matrix.
  * Step 6 "LU with column pivoting" keeps the unit diagonal on L_b; the pivot of step j is
    the first maximum |value| of row j of the current Schur complement.
  * P and Q are returned as gather index vectors: (P A Q)[i, j] = A[P[i], Q[j]].

Parity unpinned: none; every function here has a pin in tests/test_oracle_*.py.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------------------
# Step 1 of Algorithm 1: Gaussian G (n x l), "i.i.d. Gaussian with zero mean and unit
# standard deviation". The generator below is a reading (the paper names none).
# ---------------------------------------------------------------------------------------

# Philox4x32 multipliers and Weyl key increments as published by Salmon et al. (SC'11).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (counter words c0..c3, key words k0, k1).

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit products, then
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is advanced by the
    Weyl constants between rounds.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + PHILOX_W1) & 0xFFFFFFFF)
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return tuple(x.astype(np.uint32) for x in c)


def philox_stream(seed: int, stream_id: int, first_counter: int, n_counters: int) -> np.ndarray:
    """Raw uint32 stream: counters first_counter .. first_counter+n_counters-1, four words
    each, in order. Counter = (index lo32, index hi32, stream_id, 0); key = (seed lo32,
    seed hi32)."""
    idx = np.arange(first_counter, first_counter + n_counters, dtype=np.uint64)
    out = philox4x32_10(idx & _MASK32, idx >> np.uint64(32),
                        np.full(idx.shape, stream_id & 0xFFFFFFFF, dtype=np.uint64),
                        np.zeros(idx.shape, dtype=np.uint64),
                        seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return np.stack(out, axis=1).reshape(-1)


_LN2 = float.fromhex("0x1.62e42fefa39efp-1")     # double nearest ln 2
_SQRT2 = float.fromhex("0x1.6a09e667f3bcdp+0")   # double nearest sqrt 2
_PI_4 = float.fromhex("0x1.921fb54442d18p-1")    # double nearest pi/4


def _ln_coefficients(count=12):
    # 1/(2n+1), each a correctly rounded IEEE division
    return [1.0 / float(2 * n + 1) for n in range(count)]


def _trig_coefficients(count=10):
    # a_n = a_{n-1} / ((2n)(2n+1)) for sin (a_0 = 1); b_n = b_{n-1} / ((2n-1)(2n)) for cos
    s, c = [1.0], [1.0]
    for n in range(1, count):
        s.append(s[-1] / float((2 * n) * (2 * n + 1)))
        c.append(c[-1] / float((2 * n - 1) * (2 * n)))
    s = [v if n % 2 == 0 else -v for n, v in enumerate(s)]
    c = [v if n % 2 == 0 else -v for n, v in enumerate(c)]
    return s, c


def series_ln(u: np.ndarray) -> np.ndarray:
    """ln u for u in (0, 1]: u = f * 2^e with f in [sqrt2/2, sqrt2] (exact split),
    ln f = 2 atanh(s) = 2 s sum_n s^(2n)/(2n+1) with s = (f-1)/(f+1), 12 terms by Horner,
    then e*ln2 + ln f. Every step is one IEEE-rounded operation."""
    u = np.asarray(u, dtype=np.float64)
    mant, ex = np.frexp(u)                 # u = mant * 2^ex, mant in [0.5, 1)
    f = mant * 2.0
    e = (ex - 1).astype(np.float64)
    big = f > _SQRT2
    f = np.where(big, mant, f)
    e = np.where(big, e + 1.0, e)
    s = (f - 1.0) / (f + 1.0)
    z = s * s
    coef = _ln_coefficients()
    p = np.full_like(z, coef[-1])
    for cf in reversed(coef[:-1]):
        p = p * z + cf
    lnf = (s * p) * 2.0
    return e * _LN2 + lnf


def series_sincos_2pi(x: np.ndarray):
    """(sin, cos) of 2*pi*x/2^32 for uint32 x. The octant q = x >> 29 is exact; the angle
    inside it, phi = (pi/4) * w with w = (x mod 2^29)/2^29 (or 1-w in odd octants), is
    reduced to [0, pi/4]; sin and cos of phi by 10-term Taylor series (Horner in phi^2);
    the octant symmetries give the result."""
    x = np.asarray(x, dtype=np.uint64)
    q = (x >> np.uint64(29)).astype(np.int64)
    wi = (x & np.uint64((1 << 29) - 1)).astype(np.float64)
    odd = (q & 1) == 1
    wi = np.where(odd, float(1 << 29) - wi, wi)
    phi = _PI_4 * (wi * float.fromhex("0x1p-29"))
    z = phi * phi
    sc, cc = _trig_coefficients()
    sp = np.full_like(z, sc[-1])
    for cf in reversed(sc[:-1]):
        sp = sp * z + cf
    sin_phi = phi * sp
    cp = np.full_like(z, cc[-1])
    for cf in reversed(cc[:-1]):
        cp = cp * z + cf
    cos_phi = cp
    # octant table: q -> (sin theta, cos theta) in terms of (sin phi, cos phi)
    sin_t = np.select([q == 0, q == 1, q == 2, q == 3, q == 4, q == 5, q == 6, q == 7],
                      [sin_phi, cos_phi, cos_phi, sin_phi, -sin_phi, -cos_phi, -cos_phi,
                       -sin_phi])
    cos_t = np.select([q == 0, q == 1, q == 2, q == 3, q == 4, q == 5, q == 6, q == 7],
                      [cos_phi, sin_phi, -sin_phi, -cos_phi, -cos_phi, -sin_phi, sin_phi,
                       cos_phi])
    return sin_t, cos_t


def box_muller(xa: np.ndarray, xb: np.ndarray):
    """Box-Muller: u = (xa+1)/2^32 in (0,1], r = sqrt(-2 ln u), theta = 2 pi xb/2^32;
    returns (r cos theta, r sin theta)."""
    u = (np.asarray(xa, dtype=np.float64) + 1.0) * float.fromhex("0x1p-32")
    r = np.sqrt(series_ln(u) * -2.0)
    s, c = series_sincos_2pi(xb)
    return r * c, r * s


def gaussian(seed: int, stream_id: int, n: int, l: int) -> np.ndarray:
    """Step 1 of Algorithm 1: G (n x l), N(0,1) entries. Entry G[i, j] is element
    e = j*n + i of the stream; counter e//4 yields elements 4c..4c+3 as
    (z0, z1) = BoxMuller(x0, x1), (z2, z3) = BoxMuller(x2, x3)."""
    total = n * l
    nc = (total + 3) // 4
    words = philox_stream(seed, stream_id, 0, nc).reshape(nc, 4)
    z0, z1 = box_muller(words[:, 0], words[:, 1])
    z2, z3 = box_muller(words[:, 2], words[:, 3])
    flat = np.stack([z0, z1, z2, z3], axis=1).reshape(-1)[:total]
    return flat.reshape(l, n).T.copy()        # column j holds elements j*n .. j*n+n-1


_F32 = np.float32
_LN2_F = np.float32(float.fromhex("0x1.62e430p-1"))    # float nearest ln 2
_SQRT2_F = np.float32(float.fromhex("0x1.6a09e6p+0"))  # float nearest sqrt 2
_PI_4_F = np.float32(float.fromhex("0x1.921fb6p-1"))   # float nearest pi/4


def _series_coefficients_f32(n_ln=6, n_trig=7):
    """FP32 coefficient tables, every entry one IEEE-rounded FP32 division:
    1/(2n+1) for the logarithm; a_n = a_{n-1}/((2n)(2n+1)) (sine) and
    b_n = b_{n-1}/((2n-1)(2n)) (cosine), signs alternating."""
    ln = [_F32(1.0) / _F32(2 * n + 1) for n in range(n_ln)]
    s, c = [_F32(1.0)], [_F32(1.0)]
    for n in range(1, n_trig):
        s.append(s[-1] / _F32((2 * n) * (2 * n + 1)))
        c.append(c[-1] / _F32((2 * n - 1) * (2 * n)))
    s = [v if n % 2 == 0 else -v for n, v in enumerate(s)]
    c = [v if n % 2 == 0 else -v for n, v in enumerate(c)]
    return ln, s, c


def box_muller_f32(xa: np.ndarray, xb: np.ndarray):
    """Box-Muller in FP32 operations only (the generator of the FP32 and BF16 paths):
    u = (floor(xa/2^8) + 1)/2^24 in (0, 1]; ln u by the atanh series (6 terms);
    octant q = xb >> 29 and 24-bit fraction (xb >> 5) mod 2^24 (complemented in odd
    octants) give phi in [0, pi/4]; sine and cosine by 7-term Taylor series.
    Returns (r cos theta, r sin theta) as float32."""
    ln_c, sin_c, cos_c = _series_coefficients_f32()
    xa = np.asarray(xa, dtype=np.uint64)
    xb = np.asarray(xb, dtype=np.uint64)
    u = ((xa >> np.uint64(8)).astype(_F32) + _F32(1.0)) * _F32(2.0**-24)
    mant, ex = np.frexp(u)
    f = mant * _F32(2.0)
    e = (ex - 1).astype(_F32)
    big = f > _SQRT2_F
    f = np.where(big, mant, f).astype(_F32)
    e = np.where(big, e + _F32(1.0), e).astype(_F32)
    s = (f - _F32(1.0)) / (f + _F32(1.0))
    z = s * s
    p = np.full_like(z, ln_c[-1])
    for cf in reversed(ln_c[:-1]):
        p = p * z + cf
    lnu = e * _LN2_F + (s * p) * _F32(2.0)
    r = np.sqrt(lnu * _F32(-2.0))
    q = (xb >> np.uint64(29)).astype(np.int64)
    wi = ((xb >> np.uint64(5)) & np.uint64((1 << 24) - 1)).astype(_F32)
    wi = np.where((q & 1) == 1, _F32(1 << 24) - wi, wi).astype(_F32)
    phi = _PI_4_F * (wi * _F32(2.0**-24))
    z = phi * phi
    sp = np.full_like(z, sin_c[-1])
    for cf in reversed(sin_c[:-1]):
        sp = sp * z + cf
    sin_phi = phi * sp
    cp = np.full_like(z, cos_c[-1])
    for cf in reversed(cos_c[:-1]):
        cp = cp * z + cf
    cos_phi = cp
    conds = [q == i for i in range(8)]
    sin_t = np.select(conds, [sin_phi, cos_phi, cos_phi, sin_phi, -sin_phi, -cos_phi,
                              -cos_phi, -sin_phi]).astype(_F32)
    cos_t = np.select(conds, [cos_phi, sin_phi, -sin_phi, -cos_phi, -cos_phi, -sin_phi,
                              sin_phi, cos_phi]).astype(_F32)
    return r * cos_t, r * sin_t


def gaussian_f32(seed: int, stream_id: int, n: int, l: int) -> np.ndarray:
    """Step 1 for the FP32 / BF16 paths: same stream and element layout as gaussian(),
    transform box_muller_f32. Returns float32 (n x l)."""
    total = n * l
    nc = (total + 3) // 4
    words = philox_stream(seed, stream_id, 0, nc).reshape(nc, 4)
    z0, z1 = box_muller_f32(words[:, 0], words[:, 1])
    z2, z3 = box_muller_f32(words[:, 2], words[:, 3])
    flat = np.stack([z0, z1, z2, z3], axis=1).reshape(-1)[:total]
    return flat.reshape(l, n).T.copy()


# ---------------------------------------------------------------------------------------
# Steps 3 and 6 of Algorithm 1: LU with partial (row) and column pivoting.
# ---------------------------------------------------------------------------------------

def _top_two_gap(v: np.ndarray) -> float:
    """Relative gap (top1 - top2)/top1 between the two largest magnitudes of a candidate
    set (1.0 when there is one candidate, 0.0 when the top is zero)."""
    if v.size < 2:
        return 1.0
    a = np.abs(v)
    two = np.partition(a, a.size - 2)[-2:]
    top1, top2 = max(two), min(two)
    return 0.0 if top1 == 0 else float((top1 - top2) / top1)


def lu_partial_pivot(Y: np.ndarray):
    """Step 3 (with the remark after Algorithm 1: partial pivoting): P Y = L_y U_y.

    In place on a copy of Y (m x l). For j = 0..l-1: r = first index >= j of the largest
    |Y[:, j]| (current row order); if Y[r, j] != 0, swap full rows j and r, divide
    Y[j+1:, j] by Y[j, j] and subtract the outer product from Y[j+1:, j+1:]; otherwise
    record the first zero step. Returns (LU, perm, first_zero, gaps) with perm in gather
    form (row i of P Y is row perm[i] of Y) and gaps[j] the relative gap of step j."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    m, l = Y.shape
    perm = np.arange(m, dtype=np.int64)
    first_zero = -1
    gaps = np.ones(l)
    for j in range(l):
        col = Y[j:, j]
        gaps[j] = _top_two_gap(col)
        r = j + int(np.argmax(np.abs(col)))
        if Y[r, j] != 0.0:
            if r != j:
                Y[[j, r], :] = Y[[r, j], :]
                perm[[j, r]] = perm[[r, j]]
            Y[j + 1:, j] = Y[j + 1:, j] / Y[j, j]
            Y[j + 1:, j + 1:] -= np.outer(Y[j + 1:, j], Y[j, j + 1:])
        elif first_zero < 0:
            first_zero = j
    return Y, perm, first_zero, gaps


def lu_column_pivot(B: np.ndarray):
    """Step 6: B Q = L_b U_b with column pivoting, k steps on B (k x n).

    Step j: c = first index >= j of the largest |B[j, :]| (current column order); swap
    columns j and c (of B and of q); if B[j, j] != 0, divide B[j+1:, j] by B[j, j] and
    subtract the outer product from B[j+1:, j+1:]. L_b = unit lower k x k part,
    U_b = upper trapezoidal k x n part including the diagonal.
    Returns (L_b, U_b, q, first_zero, gaps); q is in gather form."""
    B = np.array(B, dtype=np.float64, copy=True)
    k, n = B.shape
    q = np.arange(n, dtype=np.int64)
    first_zero = -1
    gaps = np.ones(k)
    for j in range(k):
        row = B[j, j:]
        gaps[j] = _top_two_gap(row)
        c = j + int(np.argmax(np.abs(row)))
        if c != j:
            B[:, [j, c]] = B[:, [c, j]]
            q[[j, c]] = q[[c, j]]
        if B[j, j] != 0.0:
            B[j + 1:, j] = B[j + 1:, j] / B[j, j]
            B[j + 1:, j + 1:] -= np.outer(B[j + 1:, j], B[j, j + 1:])
        elif first_zero < 0:
            first_zero = j
    Lb = np.tril(B[:, :k], -1) + np.eye(k)
    Ub = np.triu(B)
    return Lb, Ub, q, first_zero, gaps


# ---------------------------------------------------------------------------------------
# Step 5: B = L_y^+ P A with L_y^+ = (L_y^T L_y)^{-1} L_y^T (remark after Algorithm 1).
# ---------------------------------------------------------------------------------------

def pinv_apply(Ly: np.ndarray, PA: np.ndarray) -> np.ndarray:
    """Normal equations: M = L_y^T L_y, M = R^T R (Cholesky), C = L_y^T PA,
    B = R^{-1} (R^{-T} C) by two triangular solves."""
    M = Ly.T @ Ly
    Rt = np.linalg.cholesky(M)          # lower: M = Rt Rt^T, R = Rt^T
    C = Ly.T @ PA
    T = _solve_lower(Rt, C)
    return _solve_upper(Rt.T, T)


def _solve_lower(Lm, X):
    """Forward substitution, row by row (Lm lower triangular)."""
    k = Lm.shape[0]
    Z = np.array(X, dtype=np.float64, copy=True)
    for i in range(k):
        Z[i] = (Z[i] - Lm[i, :i] @ Z[:i]) / Lm[i, i]
    return Z


def _solve_upper(Um, X):
    """Back substitution, row by row (Um upper triangular)."""
    k = Um.shape[0]
    Z = np.array(X, dtype=np.float64, copy=True)
    for i in range(k - 1, -1, -1):
        Z[i] = (Z[i] - Um[i, i + 1:] @ Z[i + 1:]) / Um[i, i]
    return Z


def check_dims(m: int, n: int, k: int, l: int) -> None:
    """Algorithm 1 input: l >= k >= 1; the lemmas behind theorem trm:rand_lu_err need l <= min(m, n)."""
    if not (1 <= k <= l <= min(m, n)):
        raise ValueError(f"need 1 <= k <= l <= min(m, n); got m={m} n={n} k={k} l={l}")


def lu_normalize(X: np.ndarray) -> np.ndarray:
    """The normalisation between power-iteration rounds (the normalised scheme that the
    power-iteration subsection of Section 5 refers to for larger q), read here as: replace
    the block X (r x l) by the lower factor of its partial-pivot LU, with the rows put back
    in X's order, Lt = P^T L (so X = Lt U and range(Lt) = range(X) when U is invertible).
    Its entries are bounded by 1, so a following product with A or A^T starts from
    well-scaled columns instead of ones that all lean towards the top singular vector."""
    X_lu, perm, _, _ = lu_partial_pivot(X)
    r, l = X.shape
    L = np.tril(X_lu[:, :l], -1) + np.eye(r, l)
    Lt = np.empty_like(L)
    Lt[perm] = L
    return Lt


def project(A: np.ndarray, G: np.ndarray, q: int = 0, normalized: bool = False) -> np.ndarray:
    """Step 2, Y = A G, or with the power iterations of Section 5 ("Power Iterations"):
    Y = (A A^*)^q A G for a small integer q, applied as q rounds of Y <- A (A^T Y) (A real,
    so A^* = A^T). ``normalized``: every round first replaces Y by lu_normalize(Y) and
    A^T Y by lu_normalize(A^T Y). Each normalisation multiplies the block on the right by
    the inverse of an upper triangular U, so the result is (A A^T)^q A G T with T upper
    triangular: the same column space, and (exact arithmetic) the same pivots and L_y in
    step 3, since P (Y T) = L_y (U_y T)."""
    if q < 0:
        raise ValueError("q must be >= 0")
    Y = A @ G
    for _ in range(q):
        if normalized:
            Y = lu_normalize(Y)
            Y = A @ lu_normalize(A.T @ Y)
        else:
            Y = A @ (A.T @ Y)
    return Y


def rlu_factor(A: np.ndarray, k: int, l: int, seed: int, stream_id: int = 0,
               G: np.ndarray | None = None, q: int = 0, normalized: bool = False) -> dict:
    """Algorithm 1, steps 1-8, in FP64. A is upcast exactly. Returns P, Q (gather form),
    L (m x k, unit lower trapezoidal), U (k x n, upper trapezoidal) and the intermediates
    G, Y (A G, or (A A^T)^q A G with q power iterations, LU-normalised between products
    when ``normalized``), Y_lu (factored Y), L_y, B, plus zero-pivot steps and per-step
    pivot gaps."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    check_dims(m, n, k, l)
    if G is None:
        G = gaussian(seed, stream_id, n, l)                 # step 1
    Y = project(A, G, q, normalized)                        # step 2
    Y_lu, P, zero_y, gaps_y = lu_partial_pivot(Y)           # step 3
    Ly = np.tril(Y_lu[:, :k], -1) + np.eye(m, k)            # step 4: first k columns
    B = pinv_apply(Ly, A[P, :])                             # step 5
    Lb, Ub, Q, zero_b, gaps_b = lu_column_pivot(B)          # step 6
    L = Ly @ Lb                                             # step 7
    U = Ub                                                  # step 8
    return dict(P=P, Q=Q, L=L, U=U, G=G, Y=Y, Y_lu=Y_lu, Ly=Ly, B=B, Lb=Lb,
                first_zero_y=zero_y, first_zero_b=zero_b, gaps_y=gaps_y, gaps_b=gaps_b)


# ---------------------------------------------------------------------------------------
# Algorithm 3 (Section 5, "Rank Deficient Least Squares"): min ||A x - b|| from the factors
# of Algorithm 1. With A ~ P^T L U Q^T: c = P b, y = L^+ c (a full-rank least-squares
# problem, normal equations as in step 5), z_1 = U_1^{-1} y with U_1 the leading k x k block
# of U, z = (z_1, 0), x = Q z. In the gather convention (P A Q)[i][j] = A[P[i]][Q[j]]:
# c[i] = b[P[i]] and x[Q[j]] = z[j].
# ---------------------------------------------------------------------------------------

def rdls_apply(P, Q, L, U, b: np.ndarray) -> np.ndarray:
    """Steps 2-5 of Algorithm 3 on given factors; b is m or m x r (r right-hand sides)."""
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    B = b.reshape(b.shape[0], -1)
    L = np.asarray(L, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    k = L.shape[1]
    n = U.shape[1]
    c = B[np.asarray(P)]                        # step 2: c = P b
    y = pinv_apply(L, c)                        #         y = L^+ c
    z1 = _solve_upper(U[:, :k], y)              # step 3: z_1 = U_1^{-1} y
    X = np.zeros((n, B.shape[1]))
    X[np.asarray(Q)[:k]] = z1                   # steps 4-5: z = (z_1, 0), x = Q z
    return X[:, 0] if vec else X


def rdls_solve(A: np.ndarray, b: np.ndarray, k: int, l: int, seed: int, q: int = 0,
               normalized: bool = False) -> dict:
    """Algorithm 3: step 1 is Algorithm 1 on A; returns x and the factors."""
    res = rlu_factor(A, k, l, seed, q=q, normalized=normalized)
    res["x"] = rdls_apply(res["P"], res["Q"], res["L"], res["U"], b)
    return res


# ---------------------------------------------------------------------------------------
# Error of Eq. (1): ||L U - P A Q||, spectral (the paper's norm) and Frobenius.
# ---------------------------------------------------------------------------------------

def spectral_norm(R: np.ndarray, dense_limit: int = 2048, seed: int = 7) -> float:
    """Largest singular value: LAPACK SVD when min(shape) <= dense_limit, else power
    iteration on R^T R from a seeded start (relative change < 1e-12 or 500 steps)."""
    if min(R.shape) <= dense_limit:
        return float(np.linalg.norm(R, 2)) if R.size else 0.0
    x = np.random.default_rng(seed).standard_normal(R.shape[1])
    x /= np.linalg.norm(x)
    prev = 0.0
    for _ in range(500):
        y = R.T @ (R @ x)
        s = float(np.linalg.norm(y))
        if s == 0.0:
            return 0.0
        x = y / s
        if abs(s - prev) <= 1e-12 * s:
            break
        prev = s
    return math.sqrt(s)


def reconstruct_error(A, P, Q, L, U, spectral: bool = True):
    """(||P A Q - L U||_F, ||P A Q - L U||_2) with R materialised in FP64."""
    A = np.asarray(A, dtype=np.float64)
    R = A[np.asarray(P)][:, np.asarray(Q)] - np.asarray(L, np.float64) @ np.asarray(U, np.float64)
    fro = float(np.linalg.norm(R))
    spec = spectral_norm(R) if spectral else float("nan")
    return fro, spec


# ---------------------------------------------------------------------------------------
# Algorithm 2 (alg:randomized_orth, Section 4.3): the randomized range finder with an
# orthogonal basis, the comparator of the error experiment of Section 5.
# ---------------------------------------------------------------------------------------

def randomized_orth(A: np.ndarray, k: int, l: int, seed: int, stream_id: int = 0,
                    G: np.ndarray | None = None) -> dict:
    """Algorithm 2: G (n x l) Gaussian (step 1, the same generator as Algorithm 1), Y = A G
    (step 2), U = the left singular vectors of Y (step 3, LAPACK SVD as a library step),
    Q = its first k columns (step 4), so that Q^T Q = I and ||Q Q^T A - A|| is bounded.
    Also returns B = Q^T A (A ~ Q B, the rank-k approximation whose error Section 5
    compares with the randomized LU's) and the singular values of Y."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    check_dims(m, n, k, l)
    if G is None:
        G = gaussian(seed, stream_id, n, l)                 # step 1
    Y = A @ G                                               # step 2
    Uy, sy, _ = np.linalg.svd(Y, full_matrices=False)       # step 3
    Q = Uy[:, :k]                                           # step 4
    return dict(Q=Q, B=Q.T @ A, sigma_y=sy, G=G, Y=Y)


def orth_error(A: np.ndarray, Q: np.ndarray, B: np.ndarray | None = None, spectral=True):
    """(||Q B - A||_F, ||Q B - A||_2) with B = Q^T A unless given: ||Q Q^* A - A||."""
    A = np.asarray(A, dtype=np.float64)
    if B is None:
        B = Q.T @ A
    R = Q @ B - A
    fro = float(np.linalg.norm(R))
    return fro, (spectral_norm(R) if spectral else float("nan"))


def halko_bound(sigma: np.ndarray, k: int, l: int) -> float:
    """The bound of Corollary 10.9 of Halko, Martinsson and Tropp that Section 4.3 quotes
    for Algorithm 2 (p = l - k >= 4, failure probability at most 6 e^{-p}):
    (1 + 17 sqrt(1 + k/p)) sigma_{k+1} + 8 sqrt(k + p) / (p + 1) (sum_{j>k} sigma_j^2)^{1/2}."""
    p = l - k
    if p < 4:
        raise ValueError("the bound needs p = l - k >= 4")
    s = np.asarray(sigma, dtype=np.float64)
    return float((1.0 + 17.0 * math.sqrt(1.0 + k / p)) * s[k]
                 + 8.0 * math.sqrt(k + p) / (p + 1.0) * math.sqrt(float(np.sum(s[k:] ** 2))))


# ---------------------------------------------------------------------------------------
# the error theorem of Section 4 (trm:rand_lu_err): error constant and success probability xi.
# ---------------------------------------------------------------------------------------

def theorem1_constant(n: int, k: int, l: int, beta: float, gamma: float) -> float:
    """2 sqrt(2 n l beta^2 gamma^2 + 1) + 2 sqrt(2 n l) beta gamma (k (n-k) + 1)."""
    bg = beta * gamma
    return (2.0 * math.sqrt(2.0 * n * l * bg * bg + 1.0)
            + 2.0 * math.sqrt(2.0 * n * l) * bg * (k * (n - k) + 1))


def theorem1_failure_terms(n: int, k: int, l: int, beta: float, gamma: float):
    """The two subtracted terms of Eq. (rand_lu_err_prob), evaluated in log space."""
    p = l - k + 1
    t1 = math.exp(-0.5 * math.log(2.0 * math.pi * p) + p * (1.0 - math.log(p * beta)))
    g2 = gamma * gamma
    log_t2 = (-math.log(4.0 * (g2 - 1.0) * math.sqrt(math.pi * n * g2))
              + n * (math.log(2.0 * g2) - (g2 - 1.0)))
    t2 = math.exp(log_t2) if log_t2 > -745.0 else 0.0
    return t1, t2


def theorem1_success_probability(n: int, k: int, l: int, beta: float, gamma: float) -> float:
    t1, t2 = theorem1_failure_terms(n, k, l, beta, gamma)
    return 1.0 - t1 - t2
