"""Pins of the fast randomized LU oracle (Algorithm 4): each step is tied to something other
than the oracle itself: numpy's FFT and scipy's DFT matrix for the SRFT, LAPACK's zgetrf
(scipy.linalg.lu_factor) for both complex pivoted LUs, the exact identity Y = X Y(J,:) of
the ID, numpy's least squares for the pseudo-inverse, and exact reconstruction of a matrix
of rank k."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle.frlu_oracle as F
import oracle as O
from paper_1310_7202_gb300 import synth


def _perm_from_lapack(piv: np.ndarray, m: int) -> np.ndarray:
    """Gather-form row permutation from LAPACK's sequence of interchanges."""
    perm = np.arange(m)
    for i, p in enumerate(piv):
        perm[[i, p]] = perm[[p, i]]
    return perm


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n,l", [(8, 3), (12, 12), (30, 7), (64, 20)])
def test_srft_columns_are_orthonormal(n, l):
    """R = D F S with unitary D F and distinct selected columns: R^H R = I_l."""
    theta, s = synth.srft_params(n, l, seed=n + l)
    R = F.srft_matrix(n, theta, s)
    assert np.abs(R.conj().T @ R - np.eye(l)).max() < 1e-13
    assert np.allclose(np.abs(R), 1.0 / math.sqrt(n), atol=1e-15)


def test_srft_without_d_is_the_unitary_dft():
    """theta = 0, s = 0..n-1: R is scipy's unitary DFT matrix (forward sign convention)."""
    n = 30
    R = F.srft_matrix(n, np.zeros(n), np.arange(n))
    assert np.abs(R - scipy.linalg.dft(n, scale="sqrtn")).max() < 1e-13


@pytest.mark.parametrize("m,n,l", [(5, 16, 4), (9, 30, 11), (4, 128, 10)])
def test_srft_apply_matches_fft(m, n, l):
    """Y = A D F S is the FFT of each row of A D, scaled by n^-1/2, at the frequencies s."""
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    theta, s = synth.srft_params(n, l, seed=3)
    d = np.exp(2j * np.pi * theta.astype(np.float64))
    Y_fft = np.fft.fft(A * d, axis=1)[:, s] / math.sqrt(n)
    assert np.abs(F.srft_apply(A, theta, s) - Y_fft).max() < 1e-12 * math.sqrt(n)


def test_srft_rejects_repeated_columns():
    with pytest.raises(ValueError):
        F.srft_matrix(8, np.zeros(8), np.array([1, 2, 1]))


@pytest.mark.parametrize("m,l", [(6, 6), (40, 9), (17, 17), (90, 30)])
def test_complex_partial_pivot_lu_matches_zgetrf(m, l):
    """Same pivots and factors as LAPACK's zgetrf (pivot = first max of |Re| + |Im|)."""
    rng = np.random.default_rng(m + 100 * l)
    Y = _crandn(rng, m, l)
    LU, perm, first_zero = F.clu_partial_pivot(Y)
    lu, piv = scipy.linalg.lu_factor(Y)
    assert np.array_equal(perm, _perm_from_lapack(piv, m))
    assert np.abs(LU - lu).max() < 1e-12
    assert first_zero == -1
    L = np.tril(LU, -1) + np.eye(m, l)
    U = np.triu(LU)[:l]
    assert np.abs(Y[perm] - L @ U).max() < 1e-12


def test_complex_lu_of_real_data_is_the_real_lu():
    """On real data |Re| + |Im| = |x|: the complex LU reduces to Algorithm 1's real LU."""
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((50, 12))
    LU, perm, _ = F.clu_partial_pivot(Y)
    LUr, permr, _, _ = O.lu_partial_pivot(Y)
    assert np.array_equal(perm, permr)
    assert np.abs(LU.imag).max() == 0.0 and np.abs(LU.real - LUr).max() < 1e-14


def test_complex_lu_zero_column_is_reported():
    rng = np.random.default_rng(6)
    Y = _crandn(rng, 10, 4)
    Y[:, 2] = Y[:, 0] * (1 - 2j)           # column 2 depends on column 0: zero at step 2
    Y[:, 1] *= 0.0
    LU, perm, first_zero = F.clu_partial_pivot(Y)
    assert first_zero == 1
    L = np.tril(LU, -1) + np.eye(10, 4)
    assert np.abs(Y[perm] - L @ np.triu(LU)[:4]).max() < 1e-12


@pytest.mark.parametrize("k,n", [(5, 5), (6, 31), (12, 40)])
def test_complex_column_pivot_lu_matches_zgetrf_of_transpose(k, n):
    """B Q = L_b U_b has the pivots of zgetrf(B^T); its factors are those of B^T rescaled:
    U_b = diag(U') L'^T, L_b = U'^T diag(U')^-1."""
    rng = np.random.default_rng(k * n)
    B = _crandn(rng, k, n)
    Lb, Ub, q, first_zero = F.clu_column_pivot(B)
    lu, piv = scipy.linalg.lu_factor(B.T)
    assert np.array_equal(q, _perm_from_lapack(piv, n))
    Lp = np.tril(lu, -1)[:, :k] + np.eye(n, k)
    Up = np.triu(lu[:k])
    d = np.diag(Up)
    assert np.abs(Ub - d[:, None] * Lp.T).max() < 1e-11
    assert np.abs(Lb - Up.T / d[None, :]).max() < 1e-11
    assert np.abs(B[:, q] - Lb @ Ub).max() < 1e-12
    assert first_zero == -1


@pytest.mark.parametrize("m,l", [(20, 5), (64, 16), (33, 33)])
def test_id_reproduces_y_exactly(m, l):
    """Y = X Y(J,:) (to rounding) and the rows J of X are the rows of the identity."""
    rng = np.random.default_rng(m + l)
    Y = _crandn(rng, m, l)
    Y_lu, perm, _ = F.clu_partial_pivot(Y)
    J, X = F.id_from_lu(Y_lu, perm, l)
    assert np.abs(X @ Y[J] - Y).max() < 1e-12 * np.abs(Y).max()
    assert np.abs(X[J] - np.eye(l)).max() < 1e-14
    # X = Y Y(J,:)^-1 when Y(J,:) is invertible (scipy's solve, not the LU above)
    assert np.abs(X - scipy.linalg.solve(Y[J].T, Y.T).T).max() < 1e-10


def test_pinv_apply_is_least_squares():
    rng = np.random.default_rng(8)
    Ly = np.tril(_crandn(rng, 40, 7), -1) + np.eye(40, 7)
    T = _crandn(rng, 40, 11)
    B = F.cpinv_apply(Ly, T)
    assert np.abs(B - np.linalg.lstsq(Ly, T, rcond=None)[0]).max() < 1e-12
    assert np.abs(Ly.conj().T @ (Ly @ B - T)).max() < 1e-11


@pytest.mark.parametrize("m,n,r,k,l", [(60, 48, 6, 6, 12), (80, 64, 5, 8, 20),
                                       (45, 45, 10, 10, 30)])
def test_frlu_exact_for_rank_k(m, n, r, k, l):
    """A of rank r <= k is reproduced to rounding; factors have the stated shapes."""
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", r, r), 1 + m, 2 + n)
    theta, s = synth.srft_params(n, l, seed=m + n)
    o = F.frlu_factor(A, k, l, theta, s)
    fro, spec = F.creconstruct_error(A, o["P"], o["Q"], o["L"], o["U"])
    assert fro < 1e-12 * np.linalg.norm(A)
    assert sorted(o["P"].tolist()) == list(range(m)) and sorted(o["Q"].tolist()) == list(range(n))
    assert np.abs(np.triu(o["L"][:k], 1)).max() == 0 and np.allclose(np.diag(o["L"][:k]), 1)
    assert np.abs(np.tril(o["U"], -1)).max() == 0


def test_frlu_error_tracks_sigma_k1():
    """Decaying spectrum: the spectral error is a modest multiple of sigma_{k+1}, far below
    the first term of the bound of the fast randomized LU error theorem, and shrinks with k
    as the randomized LU's does (Section 6, Fast Randomized LU)."""
    m = n = 96
    sigma = synth.spectrum("paper_exp", n)
    A = synth.prescribed_matrix(m, n, sigma, 7, 8)
    errs = []
    for k in (8, 16, 24):
        l = 2 * k
        theta, s = synth.srft_params(n, l, seed=k)
        o = F.frlu_factor(A, k, l, theta, s)
        _, spec = F.creconstruct_error(A, o["P"], o["Q"], o["L"], o["U"])
        bound = (1 + math.sqrt(1 + 4 * k * (n - k))) * math.sqrt(1 + 7 * n / l) * sigma[k]
        assert spec <= 50 * sigma[k] and spec <= bound, (k, spec, sigma[k])
        errs.append(spec)
    assert errs[0] > errs[1] > errs[2]


def test_srft_params_are_seeded_distinct_and_in_range():
    """The SRFT's random numbers: theta in [0, 1) (FP32), s distinct in [0, n), both fixed
    by the seed and different for another seed."""
    theta, s = synth.srft_params(3000, 200, seed=4)
    assert theta.dtype == np.float32 and theta.shape == (3000,)
    assert np.all((theta >= 0) & (theta < 1))
    assert s.dtype == np.int32 and len(np.unique(s)) == 200 and s.min() >= 0 and s.max() < 3000
    t2, s2 = synth.srft_params(3000, 200, seed=4)
    assert np.array_equal(theta, t2) and np.array_equal(s, s2)
    t3, s3 = synth.srft_params(3000, 200, seed=5)
    assert not np.array_equal(s, s3)
    with pytest.raises(ValueError):
        synth.srft_params(10, 11, seed=1)
