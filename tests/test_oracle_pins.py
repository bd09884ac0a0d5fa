"""Pins for the FP64 oracle: each test ties an oracle function to something other than
itself (a library routine, a closed form, an invariant, a value printed in the paper, or
brute force on a tiny input). CPU only."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.stats as st

import oracle as O
from paper_1310_7202_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------------------
# Step 1: Philox4x32-10 against an independent library implementation (Triton's, run by
# its CPU interpreter in a child process), for several keys, counters and stream ids.
# ----------------------------------------------------------------------------------------

_TRITON_SCRIPT = r"""
import json, sys
import numpy as np
import torch, triton, triton.language as tl
from triton.language.random import philox_impl

@triton.jit
def kern(c_ptr, out_ptr, k0, k1, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + offs * 4 + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + offs * 4 + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + offs * 4 + 3).to(tl.uint32, bitcast=True)
    a, b, c, d = philox_impl(c0, c1, c2, c3, k0.to(tl.uint32), k1.to(tl.uint32))
    tl.store(out_ptr + offs * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + offs * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + offs * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + offs * 4 + 3, d.to(tl.int32, bitcast=True))

cases = json.loads(sys.stdin.read())
res = []
for case in cases:
    ctr = np.array(case["ctr"], dtype=np.uint32).view(np.int32)
    n = len(ctr) // 4
    out = torch.zeros(4 * n, dtype=torch.int32)
    kern[(1,)](torch.from_numpy(ctr.copy()), out, case["k0"], case["k1"], N=n)
    res.append((out.numpy().view(np.uint32)).tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    cases = []
    for k0, k1 in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x243F6A88, 0x85A308D3), (7, 1)]:
        ctr = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        cases.append(dict(ctr=ctr.reshape(-1).tolist(), k0=k0, k1=k1))
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                         capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for case, want in zip(cases, ref):
        ctr = np.array(case["ctr"], dtype=np.uint64).reshape(-1, 4)
        got = O.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3],
                              case["k0"], case["k1"])
        got = np.stack(got, axis=1).reshape(-1)
        assert got.tolist() == want


def test_philox_stream_layout():
    # counter = (index lo, index hi, stream, 0), key = (seed lo, seed hi)
    seed, stream = 0x0123456789ABCDEF, 3
    s = O.philox_stream(seed, stream, (1 << 32) - 2, 4).reshape(4, 4)
    for t, idx in enumerate(range((1 << 32) - 2, (1 << 32) + 2)):
        one = O.philox4x32_10(np.array([idx & 0xFFFFFFFF]), np.array([idx >> 32]),
                              np.array([stream]), np.array([0]),
                              seed & 0xFFFFFFFF, seed >> 32)
        assert [int(v[0]) for v in one] == s[t].tolist()


# ----------------------------------------------------------------------------------------
# Box-Muller series against libm (error bounds) and the Gaussian's distribution.
# ----------------------------------------------------------------------------------------

def test_series_ln_matches_libm():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 2**32, size=200000, dtype=np.uint64)
    edge = np.array([0, 1, 2**31 - 1, 2**31, 0xB504F333, 0xB504F334, 2**32 - 2, 2**32 - 1],
                    dtype=np.uint64)
    x = np.concatenate([x, edge])
    u = (x.astype(np.float64) + 1.0) * 2.0**-32
    got = O.series_ln(u)
    want = np.log(u)
    # within 4 ulp of |ln u| (ln u = 0 exactly at u = 1)
    tol = 4 * np.spacing(np.maximum(np.abs(want), 1e-300))
    assert np.all(np.abs(got - want) <= tol)
    assert O.series_ln(np.array([1.0]))[0] == 0.0


def test_series_sincos_matches_libm():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2**32, size=200000, dtype=np.uint64)
    x = np.concatenate([x, np.arange(0, 2**32, 2**29, dtype=np.uint64),
                        np.arange(0, 2**32, 2**29, dtype=np.uint64) + 1,
                        np.arange(2**29, 2**32 + 1, 2**29, dtype=np.uint64) - 1])
    s, c = O.series_sincos_2pi(x)
    th = 2.0 * np.pi * (x.astype(np.float64) * 2.0**-32)
    # libm's argument itself carries the rounding of 2*pi*x (<= 2 ulp of 2*pi)
    assert np.max(np.abs(s - np.sin(th))) < 4e-15
    assert np.max(np.abs(c - np.cos(th))) < 4e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) < 1e-15


def test_gaussian_distribution_and_layout():
    n, l = 1000, 1000
    G = O.gaussian(12345, 0, n, l)
    z = G.T.reshape(-1)                      # element order e = j*n + i
    N = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / N)
    assert st.kstest(z, "norm").pvalue > 1e-3
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05
    # layout: elements 4c..4c+3 come from counter c as (BM(x0,x1), BM(x2,x3))
    w = O.philox_stream(12345, 0, 0, 2).reshape(2, 4)
    a0, a1 = O.box_muller(w[:, 0], w[:, 1])
    b0, b1 = O.box_muller(w[:, 2], w[:, 3])
    first8 = np.stack([a0, a1, b0, b1], axis=1).reshape(-1)
    assert np.array_equal(first8, G[:8, 0])
    # ragged tail: n*l not a multiple of 4
    G2 = O.gaussian(9, 1, 7, 3)
    assert G2.shape == (7, 3)
    assert np.array_equal(G2, O.gaussian(9, 1, 21, 1).reshape(3, 7).T)


def test_gaussian_streams_differ():
    a = O.gaussian(1, 0, 64, 4)
    b = O.gaussian(1, 1, 64, 4)
    c = O.gaussian(2, 0, 64, 4)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


# ----------------------------------------------------------------------------------------
# Step 3: partial-pivot LU against LAPACK getrf (scipy.linalg.lu_factor).
# ----------------------------------------------------------------------------------------

def _ipiv_to_perm(ipiv, m):
    perm = np.arange(m)
    for j, p in enumerate(ipiv):
        perm[[j, p]] = perm[[p, j]]
    return perm


@pytest.mark.parametrize("m,l", [(7, 3), (40, 12), (97, 31), (16, 16)])
def test_lu_partial_pivot_matches_lapack(m, l):
    rng = np.random.default_rng(m * 100 + l)
    Y = rng.standard_normal((m, l))
    LU, perm, zero, gaps = O.lu_partial_pivot(Y)
    ref, ipiv = sl.lu_factor(Y)
    assert np.array_equal(perm, _ipiv_to_perm(ipiv, m)[:m])
    assert np.allclose(LU, ref, rtol=0, atol=1e-12)
    assert zero == -1
    Ly = np.tril(LU, -1) + np.eye(m, l)
    Uy = np.triu(LU[:l])
    assert np.max(np.abs(Ly)) <= 1.0
    assert np.allclose(Ly @ Uy, Y[perm], atol=1e-12)


def test_lu_partial_pivot_zero_column_and_ties():
    Y = np.array([[0.0, 1.0], [0.0, 2.0], [0.0, -2.0]])
    LU, perm, zero, _ = O.lu_partial_pivot(Y)
    assert zero == 0 and perm[0] == 0          # zero pivot: no swap, reported
    # tie in |value|: the first in current row order wins (getf2 / i?amax rule)
    Y = np.array([[1.0, 0.0], [-3.0, 1.0], [3.0, 5.0]])
    _, perm, _, _ = O.lu_partial_pivot(Y)
    assert perm[0] == 1


# ----------------------------------------------------------------------------------------
# Step 6: column-pivoted LU = getrf of B^T (same Schur complements, same pivots).
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("k,n", [(3, 9), (12, 50), (20, 20)])
def test_lu_column_pivot_matches_lapack_on_transpose(k, n):
    rng = np.random.default_rng(k * 1000 + n)
    B = rng.standard_normal((k, n))
    Lb, Ub, q, zero, _ = O.lu_column_pivot(B)
    _, ipiv = sl.lu_factor(B.T)
    assert np.array_equal(q, _ipiv_to_perm(ipiv, n))
    assert np.allclose(Lb @ Ub, B[:, q], atol=1e-12)
    d = np.abs(np.diag(Ub))
    for j in range(k):
        assert np.all(np.abs(Ub[j, j:]) <= d[j] * (1 + 1e-15))
    assert np.allclose(np.diag(Lb), 1.0) and np.allclose(np.triu(Lb, 1), 0.0)


# ----------------------------------------------------------------------------------------
# Step 5: B = L_y^+ P A against least squares (QR/SVD based, independent of the Gram).
# ----------------------------------------------------------------------------------------

def test_pinv_apply_matches_lstsq():
    rng = np.random.default_rng(3)
    m, k, n = 120, 9, 40
    Y = rng.standard_normal((m, k + 2))
    LU, _, _, _ = O.lu_partial_pivot(Y)
    Ly = np.tril(LU[:, :k], -1) + np.eye(m, k)
    PA = rng.standard_normal((m, n))
    B = O.pinv_apply(Ly, PA)
    ref = np.linalg.lstsq(Ly, PA, rcond=None)[0]
    assert np.allclose(B, ref, rtol=1e-11, atol=1e-11)
    # normal equations hold: L_y^T (L_y B - PA) = 0
    assert np.max(np.abs(Ly.T @ (Ly @ B - PA))) < 1e-10


# ----------------------------------------------------------------------------------------
# End to end: closed forms, the identity in the proof of theorem trm:rand_lu_err, brute force.
# ----------------------------------------------------------------------------------------

def _check_structure(res, m, n, k):
    P, Q, L, U = res["P"], res["Q"], res["L"], res["U"]
    assert sorted(P.tolist()) == list(range(m))
    assert sorted(Q.tolist()) == list(range(n))
    assert L.shape == (m, k) and U.shape == (k, n)
    assert np.allclose(np.triu(L[:k], 1), 0.0)
    assert np.allclose(np.diag(L[:k]), 1.0)
    assert np.allclose(np.tril(U[:, :k], -1), 0.0)


def test_exact_rank_k_reconstructs_to_rounding():
    m, n, k, l = 200, 150, 12, 17
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", min(m, n), k), 1, 2)
    res = O.rlu_factor(A, k, l, seed=5)
    _check_structure(res, m, n, k)
    fro, spec = O.reconstruct_error(A, res["P"], res["Q"], res["L"], res["U"])
    assert fro / np.linalg.norm(A) < 1e-12
    assert spec < 1e-12


# ----------------------------------------------------------------------------------------
# Section 5, power iterations: step 2 becomes Y = (A A^T)^q A G.
# ----------------------------------------------------------------------------------------

def test_project_power_closed_form():
    """(A A^T)^q A = U diag(sigma^(2q+1)) V^T for A = U diag(sigma) V^T: the oracle's q
    rounds of Y <- A (A^T Y) against that closed form. A transposed operand, a missing or
    extra round, or A^T A in place of A A^T changes the exponent or the singular vectors."""
    rng = np.random.default_rng(3)
    m, n, l = 40, 30, 6
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sigma = np.linspace(1.5, 0.2, n)
    A = (U * sigma) @ V.T
    G = rng.standard_normal((n, l))
    for q in (0, 1, 2, 3):
        want = (U * sigma ** (2 * q + 1)) @ (V.T @ G)
        got = O.project(A, G, q)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), q
    with pytest.raises(ValueError):
        O.project(A, G, -1)


@pytest.mark.parametrize("spec", ["paper_exp", "paper_slow"])
def test_power_iteration_lowers_the_error(spec):
    """The power-iteration subsection of Section 5: one power iteration lowers the error of
    Algorithm 1 for the exponentially decaying spectrum and for the slow decay
    sigma_k = 100 / (9 + k)^2 (normalised to sigma_1 = 1). Every rank-k error stays at or
    above sigma_{k+1}, the optimum."""
    m = n = 300
    k, l = 20, 25
    sigma = synth.spectrum(spec, n)
    e0, e1 = [], []
    for seed in range(3):
        A = synth.prescribed_matrix(m, n, sigma, 10 + seed, 20 + seed)
        for q, errs in ((0, e0), (1, e1)):
            r = O.rlu_factor(A, k, l, seed=seed, q=q)
            _, spec2 = O.reconstruct_error(A, r["P"], r["Q"], r["L"], r["U"])
            assert spec2 >= sigma[k] * (1 - 1e-9)
            errs.append(spec2)
    assert np.median(e1) < np.median(e0), (e0, e1)


def test_lu_normalize_is_scipys_permuted_lower_factor():
    """The normalisation between rounds: the lower factor of the partial-pivot LU with the
    rows put back (X = Lt U) is scipy's lu(X, permute_l=True) lower factor (LAPACK getrf)."""
    import scipy.linalg as sl
    rng = np.random.default_rng(8)
    for r, l in ((50, 8), (37, 37), (200, 31)):
        X = rng.standard_normal((r, l))
        Lt = O.rlu_oracle.lu_normalize(X)
        PL, Uf = sl.lu(X, permute_l=True)
        assert np.abs(Lt - PL).max() <= 1e-13
        assert np.abs(Lt @ Uf - X).max() <= 1e-12 * np.abs(X).max()
        assert np.abs(Lt).max() <= 1.0 + 1e-15


def test_normalized_power_is_an_upper_triangular_change_of_basis():
    """Normalised rounds give (A A^T)^q A G T with T upper triangular (each normalisation
    multiplies by the inverse of an upper triangular U factor): a least-squares fit of the
    normalised Y on the unnormalised one recovers an upper triangular T, exactly (to
    rounding) fitting. A normalisation that reordered or mixed columns would leave a lower
    part; one that lost a round would not fit."""
    rng = np.random.default_rng(4)
    m, n, l = 60, 45, 7
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.linspace(1.4, 0.3, n)) @ V.T
    G = rng.standard_normal((n, l))
    for q in (1, 2):
        Yu = O.project(A, G, q)
        Yn = O.project(A, G, q, normalized=True)
        T = np.linalg.lstsq(Yu, Yn, rcond=None)[0]
        assert np.abs(Yu @ T - Yn).max() <= 1e-11 * np.abs(Yn).max()
        assert np.abs(np.tril(T, -1)).max() <= 1e-9 * np.abs(T).max(), q


def test_normalized_power_gives_the_same_factors():
    """Y T with T upper triangular has the same partial-pivot pivots and lower factor as Y,
    so in exact arithmetic normalised and unnormalised rounds give the same P, Q, L, U;
    in FP64 on a well-resolved case they agree to rounding."""
    m, n, k, l = 300, 260, 20, 30
    A = synth.prescribed_matrix(m, n, synth.spectrum("paper_slow", n), 3, 4)
    for q in (1, 2):
        a = O.rlu_factor(A, k, l, seed=2, q=q)
        b = O.rlu_factor(A, k, l, seed=2, q=q, normalized=True)
        assert np.array_equal(a["P"], b["P"]) and np.array_equal(a["Q"], b["Q"])
        assert np.abs(a["L"] - b["L"]).max() <= 1e-8 * np.abs(a["L"]).max()
        assert np.abs(a["U"] - b["U"]).max() <= 1e-8 * np.abs(a["U"]).max()


def test_normalized_power_keeps_directions_that_unnormalized_rounds_lose():
    """Why the paper points to a normalised scheme for larger q: with sigma_i = i^-2 and
    q = 4, (sigma_{k+1} / sigma_1)^(2q+1) = 441^-9 ~ 1e-24 is far below FP64's unit, so
    the unnormalised product has lost the directions beyond the first few and the error
    grows past the q = 0 error, while the normalised rounds keep improving on it. Both stay
    at or above the optimum sigma_{k+1} (spectral norm)."""
    m = n = 300
    k, l = 20, 30
    sigma = synth.spectrum("inv_square", n)
    A = synth.prescribed_matrix(m, n, sigma, 3, 4)
    e = {}
    for q, norm in ((0, False), (4, False), (4, True)):
        r = O.rlu_factor(A, k, l, seed=2, q=q, normalized=norm)
        _, e[(q, norm)] = O.reconstruct_error(A, r["P"], r["Q"], r["L"], r["U"])
        assert e[(q, norm)] >= sigma[k] * (1 - 1e-9)
    assert e[(4, False)] > e[(0, False)]
    assert e[(4, True)] < 0.5 * e[(0, False)]
    assert e[(4, True)] < 0.25 * e[(4, False)]


def test_power_iteration_keeps_exact_rank():
    m, n, k, l = 120, 90, 10, 14
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", min(m, n), k), 3, 4)
    for q, norm in ((1, False), (2, False), (1, True), (3, True)):
        res = O.rlu_factor(A, k, l, seed=5, q=q, normalized=norm)
        _check_structure(res, m, n, k)
        fro, _ = O.reconstruct_error(A, res["P"], res["Q"], res["L"], res["U"], spectral=False)
        assert fro / np.linalg.norm(A) < 1e-12


# ----------------------------------------------------------------------------------------
# Algorithm 3 (rank-deficient least squares, Section 5).
# ----------------------------------------------------------------------------------------

def test_rdls_exact_rank_reaches_the_least_squares_minimum():
    """For rank(A) = k the randomized LU is exact, so x attains the least-squares minimum:
    the residual equals numpy.linalg.lstsq's, A^T (A x - b) = 0 (normal equations of the
    original problem), and x has at most k nonzero entries. A consistent b = A x0 is met to
    rounding."""
    m, n, k, l = 160, 120, 9, 14
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", n, k), 5, 6)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((m, 3))
    res = O.rdls_solve(A, b, k, l, seed=2)
    x = res["x"]
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    r_min = np.linalg.norm(A @ x_ls - b, axis=0)
    assert np.allclose(np.linalg.norm(A @ x - b, axis=0), r_min, rtol=1e-10, atol=1e-12)
    assert np.abs(A.T @ (A @ x - b)).max() < 1e-10 * np.abs(A.T @ b).max()
    assert all(np.count_nonzero(x[:, j]) <= k for j in range(3))
    x0 = rng.standard_normal(n)
    xv = O.rdls_apply(res["P"], res["Q"], res["L"], res["U"], A @ x0)
    assert np.linalg.norm(A @ xv - A @ x0) < 1e-11 * np.linalg.norm(A @ x0)


def test_rdls_permutation_conventions_by_brute_force():
    """Tiny case against a brute-force restatement with explicit permutation matrices: A
    approximated by P^T L U Q^T, y = argmin ||L y - P b||, z_1 = U_1^{-1} y, x = Q (z_1, 0)."""
    m, n, k, l = 12, 9, 3, 5
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", n, k), 7, 8)
    b = np.random.default_rng(2).standard_normal(m)
    res = O.rdls_solve(A, b, k, l, seed=3)
    Pm = np.eye(m)[res["P"]]          # (Pm A)[i] = A[P[i]]
    Qm = np.eye(n)[:, res["Q"]]       # (A Qm)[:, j] = A[:, Q[j]]
    assert np.allclose(Pm @ A @ Qm, res["L"] @ res["U"], atol=1e-12)
    y = np.linalg.lstsq(res["L"], Pm @ b, rcond=None)[0]
    z = np.zeros(n)
    z[:k] = np.linalg.solve(res["U"][:, :k], y)
    assert np.allclose(res["x"], Qm @ z, atol=1e-12)


def test_full_rank_k_equals_n_is_exact_lu():
    n = 24
    rng = np.random.default_rng(4)
    A = rng.standard_normal((n, n))
    res = O.rlu_factor(A, n, n, seed=3)
    fro, _ = O.reconstruct_error(A, res["P"], res["Q"], res["L"], res["U"])
    assert fro / np.linalg.norm(A) < 1e-12


def test_proof_identity_eq_main_bound():
    # LU - PAQ = (L_y L_y^+ - I) P A Q  (proof of theorem trm:rand_lu_err, Eq. main_bound_proof, Section 4.2)
    m, n, k, l = 90, 70, 8, 11
    A = synth.prescribed_matrix(m, n, synth.spectrum("inv_square", min(m, n)), 3, 4)
    res = O.rlu_factor(A, k, l, seed=8)
    P, Q, L, U, Ly = res["P"], res["Q"], res["L"], res["U"], res["Ly"]
    PAQ = A[P][:, Q]
    lhs = L @ U - PAQ
    rhs = (Ly @ np.linalg.pinv(Ly) - np.eye(m)) @ PAQ
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    # ||L_y L_y^+|| <= 1 and L_y^+ L_y = I (used in the proof of lemma lem:rand_lu_bound1)
    assert np.linalg.norm(Ly @ np.linalg.pinv(Ly), 2) <= 1 + 1e-12
    assert np.allclose(np.linalg.pinv(Ly) @ Ly, np.eye(k), atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_bounds_tiny(seed):
    # sigma_{k+1} <= ||LU - PAQ||_2 <= C(n,k,l,beta=5,gamma=5) sigma_{k+1} (theorem trm:rand_lu_err;
    # the lower bound is Eckart-Young). sigma by full SVD of A.
    m, n, k, l = 48, 40, 6, 9
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) @ np.diag(0.7 ** np.arange(n)) @ rng.standard_normal((n, n))
    s = np.linalg.svd(A, compute_uv=False)
    res = O.rlu_factor(A, k, l, seed=seed + 10)
    _, spec = O.reconstruct_error(A, res["P"], res["Q"], res["L"], res["U"])
    C = O.theorem1_constant(n, k, l, 5.0, 5.0)
    assert s[k] * (1 - 1e-10) <= spec <= C * s[k]


def test_reconstruct_error_known_residual():
    # R = PAQ - LU with L U = 0 and A = x y^T: ||R||_F = ||R||_2 = |x||y|
    m, n, k = 30, 20, 2
    x = np.arange(1.0, m + 1)
    y = np.linspace(-1, 1, n)
    A = np.outer(x, y)
    P = np.arange(m)[::-1]
    Q = np.roll(np.arange(n), 3)
    fro, spec = O.reconstruct_error(A, P, Q, np.zeros((m, k)), np.zeros((k, n)))
    want = np.linalg.norm(x) * np.linalg.norm(y)
    assert abs(fro - want) < 1e-12 * want and abs(spec - want) < 1e-12 * want


def test_power_iteration_matches_svd():
    rng = np.random.default_rng(6)
    R = rng.standard_normal((300, 200)) @ np.diag(np.linspace(3, 1, 200))
    want = np.linalg.norm(R, 2)
    got = O.spectral_norm(R, dense_limit=10)
    assert abs(got - want) < 1e-6 * want


# ----------------------------------------------------------------------------------------
# Theorem trm:rand_lu_err: the success probability against Table 1 of the paper.
# ----------------------------------------------------------------------------------------

def test_theorem1_xi_matches_table1():
    rows = []
    with open(os.path.join(HERE, "golden", "xi_table.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                a, b, c, d = line.split()
                rows.append((int(a), float(b), float(c), float(d)))
    assert len(rows) == 9
    for lk, beta, gamma, one_minus_xi in rows:
        k = 20
        t1, t2 = O.theorem1_failure_terms(10000, k, k + lk, beta, gamma)
        got = t1 + t2
        # the table prints two significant digits
        assert abs(got - one_minus_xi) <= 0.025 * one_minus_xi, (lk, beta, gamma, got)


def test_theorem1_constant_closed_form():
    # n=1, k=0, l=1, beta=gamma=1: 2*sqrt(3) + 2*sqrt(2)*(0+1)
    assert abs(O.theorem1_constant(1, 0, 1, 1.0, 1.0) - (2 * math.sqrt(3) + 2 * math.sqrt(2))) < 1e-14


def test_check_dims():
    O.check_dims(10, 8, 3, 8)
    for bad in [(10, 8, 0, 3), (10, 8, 4, 3), (10, 8, 3, 9), (5, 8, 3, 6)]:
        with pytest.raises(ValueError):
            O.check_dims(*bad)


# ----------------------------------------------------------------------------------------
# The FP32 transform of the FP32 / BF16 paths against libm and the distribution.
# ----------------------------------------------------------------------------------------

def test_box_muller_f32_matches_libm():
    rng = np.random.default_rng(11)
    xa = rng.integers(0, 2**32, size=200000, dtype=np.uint64)
    xb = rng.integers(0, 2**32, size=200000, dtype=np.uint64)
    xa[:4] = [0, 255, 2**32 - 1, 2**31]
    xb[:4] = [0, 2**29, 2**32 - 1, 3 * 2**29 + 31]
    z0, z1 = O.box_muller_f32(xa, xb)
    assert z0.dtype == np.float32 and z1.dtype == np.float32
    u = ((xa >> 8).astype(np.float64) + 1.0) * 2.0**-24
    r = np.sqrt(-2.0 * np.log(u))
    th = 2.0 * np.pi * ((xb >> 5).astype(np.float64) * 2.0**-27)
    # a few float32 ulps of r (r <= 5.8)
    assert np.max(np.abs(z0 - r * np.cos(th))) < 8 * np.spacing(np.float32(6.0))
    assert np.max(np.abs(z1 - r * np.sin(th))) < 8 * np.spacing(np.float32(6.0))


def test_gaussian_f32_distribution_and_layout():
    G = O.gaussian_f32(77, 0, 1000, 1000)
    assert G.dtype == np.float32
    z = G.T.reshape(-1).astype(np.float64)
    N = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / N)
    assert st.kstest(z, "norm").pvalue > 1e-3
    # close to the FP64 transform of the same words (both are N(0,1) samples of the
    # same uniforms, up to the FP32 uniform's 24-bit resolution)
    G64 = O.gaussian(77, 0, 1000, 1000)
    assert np.median(np.abs(G - G64)) < 1e-5


# ----------------------------------------------------------------------------------------
# Algorithm 2 (randomized range finder with an orthogonal basis), the comparator of the
# error experiment of Section 5.
# ----------------------------------------------------------------------------------------

def test_randomized_orth_closed_form():
    """A = U diag(sigma) V^T and G = V[:, :l] (a fixed test matrix in place of the Gaussian)
    give Y = U[:, :l] diag(sigma_1..l): the top-k left singular vectors of Y are U[:, :k], so
    Q Q^T = U_k U_k^T and the errors are the optimal rank-k ones, sqrt(sum_{i>k} sigma_i^2)
    (Frobenius) and sigma_{k+1} (spectral). Taking the last k columns, A^T for A, or a G
    of the wrong side breaks each equality."""
    rng = np.random.default_rng(11)
    m, n, k, l = 60, 45, 6, 10
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sigma = np.sort(rng.uniform(0.1, 2.0, n))[::-1]
    A = (U * sigma) @ V.T
    r = O.randomized_orth(A, k, l, seed=0, G=V[:, :l].copy())
    assert np.abs(r["Q"] @ r["Q"].T - U[:, :k] @ U[:, :k].T).max() <= 1e-12
    assert np.abs(r["sigma_y"] - sigma[:l]).max() <= 1e-12
    fro, spec = O.orth_error(A, r["Q"])
    assert abs(fro - np.sqrt(np.sum(sigma[k:] ** 2))) <= 1e-12
    assert abs(spec - sigma[k]) <= 1e-12


def test_randomized_orth_exact_rank_and_orthonormal_basis():
    m, n, k, l = 120, 90, 10, 16
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", min(m, n), k), 3, 4)
    r = O.randomized_orth(A, k, l, seed=5)
    assert np.abs(r["Q"].T @ r["Q"] - np.eye(k)).max() <= 1e-13
    assert np.abs(r["B"] - r["Q"].T @ A).max() <= 1e-13
    fro, _ = O.orth_error(A, r["Q"], spectral=False)
    assert fro / np.linalg.norm(A) < 1e-13


@pytest.mark.parametrize("spec", ["paper_exp", "paper_slow", "inv_square"])
def test_randomized_orth_bounds(spec):
    """Eckart-Young: no rank-k Q reaches below sigma_{k+1}; the bound of Corollary 10.9 of
    Halko et al. quoted in Section 4.3 holds (failure probability 6 e^{-10} < 3e-4 per
    draw at p = 10)."""
    m = n = 200
    sigma = synth.spectrum(spec, n)
    for seed in range(3):
        A = synth.prescribed_matrix(m, n, sigma, 30 + seed, 40 + seed)
        for k in (8, 25):
            r = O.randomized_orth(A, k, k + 10, seed=seed)
            _, spec2 = O.orth_error(A, r["Q"])
            assert sigma[k] * (1 - 1e-9) <= spec2 <= O.halko_bound(sigma, k, k + 10)


def test_randomized_lu_error_close_to_randomized_orth():
    """Section 5 reports the randomized LU and the randomized SVD errors as almost identical
    on an exponentially decaying spectrum; here their ratio stays within [1/3, 3]."""
    m = n = 300
    sigma = synth.spectrum("paper_exp", n)
    A = synth.prescribed_matrix(m, n, sigma, 7, 8)
    for k in (10, 20, 40):
        r = O.randomized_orth(A, k, k + 3, seed=2)
        _, e_svd = O.orth_error(A, r["Q"])
        lu = O.rlu_factor(A, k, k + 3, seed=2)
        _, e_lu = O.reconstruct_error(A, lu["P"], lu["Q"], lu["L"], lu["U"])
        assert 1 / 3 <= e_lu / e_svd <= 3, (k, e_lu, e_svd)
