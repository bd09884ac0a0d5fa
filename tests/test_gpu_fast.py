"""Fast randomized LU (Algorithm 4, include/rlu_fast.h) on the GPU against the complex128
oracle: the SRFT product element by element, the factorization through its pivots and its
error (the tolerance of the other parity tests: 1.1x the oracle's ||PAQ - LU||_F plus
1e-4 ||A||_2), structure and edge cases, and properties at the benchmark size
(4096 x 4096, k = 256, l = 432 = 3 log2(n)^2). GPU only."""
import math

import numpy as np
import pytest
import torch

import oracle.frlu_oracle as F
from paper_1310_7202_gb300 import rlu, synth
from tests.gpu_helpers import leading_agreement

pytestmark = pytest.mark.gpu


def _factor(A: np.ndarray, k: int, l: int, seed: int):
    theta, s = synth.srft_params(A.shape[1], l, seed)
    o = rlu.fast_factor(torch.from_numpy(A).cuda(), k, l, theta, s)
    torch.cuda.synchronize()
    return {key: v.cpu().numpy() for key, v in o.items()}, theta, s


@pytest.mark.parametrize("m,n,l", [(37, 64, 10), (50, 360, 40), (20, 3000, 23),
                                   (9, 16384, 50), (24, 8192, 507), (5, 8, 8)])
def test_srft_apply_matches_oracle(m, n, l):
    """Y = A D F S element by element: FP32 transform error ~ eps log2(n) ||row||."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    theta, s = synth.srft_params(n, l, seed=n)
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    Y = rlu.srft_apply(torch.from_numpy(A).cuda(), torch.from_numpy(theta).cuda(),
                       torch.from_numpy(s).cuda(), info).cpu().numpy()
    Yo = F.srft_apply(A.astype(np.float64), theta, s)
    tol = 2e-6 * math.log2(2 * n) * np.linalg.norm(A.astype(np.float64), axis=1)
    assert np.all(np.abs(Y - Yo).max(axis=1) <= tol), np.abs(Y - Yo).max()
    assert info[0].item() == 0


@pytest.mark.parametrize("m,n,k,l", [(300, 240, 20, 40), (513, 360, 30, 48), (200, 200, 12, 15),
                                     (1000, 1000, 50, 100), (64, 30, 30, 30)])
def test_fast_factor_against_oracle(m, n, k, l):
    sigma = synth.spectrum("exp_k", min(m, n), k)
    A = synth.prescribed_matrix(m, n, sigma, m, n, dtype=np.float32)
    g, theta, s = _factor(A, k, l, seed=k)
    o = F.frlu_factor(A.astype(np.float64), k, l, theta, s)
    fro_o, _ = F.creconstruct_error(A, o["P"], o["Q"], o["L"], o["U"])
    fro_g, _ = F.creconstruct_error(A, g["P"], g["Q"], g["L"], g["U"])
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert sorted(g["P"].tolist()) == list(range(m)) and sorted(g["Q"].tolist()) == list(range(n))
    assert leading_agreement(g["P"], o["P"], l) >= min(5, l)
    L, U = g["L"], g["U"]
    assert np.all(np.diag(L[:k]) == 1) and np.all(np.triu(L[:k], 1) == 0)
    assert np.all(np.tril(U, -1) == 0)
    assert g["info"].tolist()[:3] == [0, -1, -1]


def test_fast_factor_paper_error_shape():
    """The shape of the paper's error comparison of Algorithms 1 and 4 (Section 6): 3000 x 3000
    (n = 2^3 3 5^3, a mixed-radix row transform), exponentially decaying spectrum, l = k + 3."""
    m = n = 3000
    k, l = 20, 23
    sigma = synth.spectrum("paper_exp", n)
    A = synth.prescribed_matrix(m, n, sigma, 81, 82, dtype=np.float32)
    g, theta, s = _factor(A, k, l, seed=83)
    o = F.frlu_factor(A.astype(np.float64), k, l, theta, s)
    fro_o, _ = F.creconstruct_error(A, o["P"], o["Q"], o["L"], o["U"])
    fro_g, _ = F.creconstruct_error(A, g["P"], g["Q"], g["L"], g["U"])
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert g["info"].tolist()[:3] == [0, -1, -1]


def test_fast_factor_exact_for_rank_k():
    m, n, r, k, l = 400, 256, 8, 8, 24
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", r, r), 3, 4, dtype=np.float32)
    g, _, _ = _factor(A, k, l, seed=2)
    fro, _ = F.creconstruct_error(A, g["P"], g["Q"], g["L"], g["U"])
    assert fro <= 1e-5 * np.linalg.norm(A.astype(np.float64))


def test_fast_factor_zero_matrix_reports_zero_pivots():
    """A = 0: every pivot of both LUs is zero (skipped, reported at step 0); L U = 0."""
    A = np.zeros((64, 60), dtype=np.float32)
    g, _, _ = _factor(A, 4, 8, seed=1)
    assert g["info"].tolist()[:3] == [0, 0, 0]
    assert np.all(g["U"] == 0)
    assert np.all(np.diag(g["L"][:4]) == 1)
    assert sorted(g["P"].tolist()) == list(range(64))


def test_srft_out_of_range_index_sets_status():
    A = torch.ones(4, 16, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.tensor([1, 16, 3], dtype=torch.int32, device="cuda")
    Y = rlu.srft_apply(A, torch.zeros(16, device="cuda"), s, info)
    torch.cuda.synchronize()
    assert info[0].item() == 1                      # RLU_EINVAL
    assert torch.all(Y[:, 1] == 0)


def test_fast_factor_rejects_sizes_outside_the_limits():
    with pytest.raises(rlu.RluError):
        rlu.FastFactorizer(64, 14, 2, 4)             # 14 = 2 * 7: no row transform
    with pytest.raises(rlu.RluError):
        rlu.FastFactorizer(64, 64, 9, 8)             # k > l
    with pytest.raises(rlu.RluError):
        rlu.FastFactorizer(4096, 4096, 100, 600)     # l > 512
    with pytest.raises(rlu.RluError):
        rlu.FastFactorizer(4096, 4096, 422, 432)     # Gram's real form 844 x 844: too large


def test_fast_factor_benchmark_size_properties():
    """4096 x 4096, sigma_i = i^-2, k = 256, l = 432: valid permutations and structure, sampled
    rows of Y against numpy's FFT, the error within 10x the randomized LU's on the same A
    (both decay at the same rate, Section 6) and below the first term of the bound of the
    fast randomized LU error theorem."""
    m = n = 4096
    k, l = 256, 432
    sigma = synth.spectrum("inv_square", n)
    A = synth.prescribed_matrix_torch(m, n, sigma, 61, 62, torch.float32)
    theta, s = synth.srft_params(n, l, seed=63)
    f = rlu.FastFactorizer(m, n, k, l)
    o = f.run(A, torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda())
    Y = rlu.srft_apply(A, torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda())
    torch.cuda.synchronize()
    assert o["info"].tolist()[:3] == [0, -1, -1]
    assert torch.equal(torch.sort(o["P"].long())[0], torch.arange(m, device="cuda"))
    assert torch.equal(torch.sort(o["Q"].long())[0], torch.arange(n, device="cuda"))
    rows = np.random.default_rng(1).choice(m, 16, replace=False)
    Ar = A[rows].double().cpu().numpy()
    d = np.exp(2j * np.pi * theta.astype(np.float64))
    Yr = np.fft.fft(Ar * d, axis=1)[:, s] / math.sqrt(n)
    tol = 2e-6 * math.log2(2 * n) * np.linalg.norm(Ar, axis=1)
    assert np.all(np.abs(Y[rows].cpu().numpy() - Yr).max(axis=1) <= tol)
    Ad = A.double()
    R = Ad[o["P"].long()][:, o["Q"].long()] - o["L"].to(torch.complex128) @ o["U"].to(torch.complex128)
    fro_fast = torch.linalg.norm(R).item()
    spec_fast = torch.linalg.matrix_norm(R, ord=2).item()
    P, Q, L, U, _ = rlu.Factorizer(m, n, k, l, "f32")(A, 63)
    fro_rlu = torch.linalg.norm(Ad[P.long()][:, Q.long()] - L.double() @ U.double()).item()
    assert fro_fast <= 10 * fro_rlu + 1e-4 * sigma[0], (fro_fast, fro_rlu)
    bound = (1 + math.sqrt(1 + 4 * k * (n - k))) * math.sqrt(1 + 7 * n / l) * sigma[k]
    assert spec_fast <= bound
