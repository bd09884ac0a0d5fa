"""Algorithm 3 (Section 5, rank-deficient least squares) through rlu_lstsq: the GPU's solve
on the GPU's own factors against the oracle's steps 2-5 on the same factors, and end to end
on exactly rank-k inputs, where x must attain the least-squares minimum. GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


def _factors(A, k, l, prec, seed=3):
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    P, Q, L, U, info = rlu.Factorizer(A.shape[0], A.shape[1], k, l, prec)(At, seed)
    torch.cuda.synchronize()
    return At, P.clone(), Q.clone(), L.clone(), U.clone()


@pytest.mark.parametrize("prec,m,n,k,l,r", [
    ("f64", 500, 300, 20, 26, 1),
    ("f64", 700, 650, 37, 45, 5),       # ragged 32-row blocks of U_1
    ("f64", 3000, 800, 300, 310, 3),    # k > 256: FP64 LDL^T; ten blocks of U_1
    ("f32", 2000, 1500, 64, 74, 4),
    ("mixed", 4096, 2048, 200, 210, 16),
])
def test_lstsq_matches_oracle_on_the_same_factors(prec, m, n, k, l, r):
    dt = np.float64 if prec == "f64" else np.float32
    A = synth.prescribed_matrix(m, n, synth.spectrum("inv_square", min(m, n)), 1, 2, dtype=dt)
    At, P, Q, L, U = _factors(A, k, l, prec)
    b = np.random.default_rng(4).standard_normal((m, r)).astype(dt)
    bt = torch.from_numpy(b).cuda().t().contiguous().t()
    info = torch.empty(4, dtype=torch.int32, device="cuda")
    x = rlu.lstsq(P, Q, L, U, bt if r > 1 else bt[:, 0], info=info)
    torch.cuda.synchronize()
    x = x.cpu().numpy().reshape(n, r).astype(np.float64)
    xo = O.rdls_apply(P.cpu().numpy(), Q.cpu().numpy(), L.cpu().numpy(), U.cpu().numpy(),
                      b.astype(np.float64))
    tol = 1e-9 if prec == "f64" else 2e-3
    assert np.linalg.norm(x - xo) <= tol * np.linalg.norm(xo), np.linalg.norm(x - xo) / np.linalg.norm(xo)
    A64 = A.astype(np.float64)
    res_g = np.linalg.norm(A64 @ x - b, axis=0)
    res_o = np.linalg.norm(A64 @ xo - b, axis=0)
    assert np.all(res_g <= res_o * (1 + (1e-9 if prec == "f64" else 1e-2)))
    assert all(np.count_nonzero(x[:, j]) <= k for j in range(r))
    assert info.cpu().tolist()[:3] == [0, -1, -1]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lstsq_exact_rank_attains_the_minimum(prec):
    m, n, k, l = 1200, 900, 25, 32
    dt = np.float64 if prec == "f64" else np.float32
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", n, k), 5, 6, dtype=dt)
    At, P, Q, L, U = _factors(A, k, l, prec)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(m).astype(dt)
    x = rlu.lstsq(P, Q, L, U, torch.from_numpy(b).cuda()).cpu().numpy().astype(np.float64)
    A64 = A.astype(np.float64)
    # the minimum over rank-k solutions: A rounded to FP32 has singular values ~1e-7 past k,
    # which a full-rank solve would use (rcond cuts them)
    x_ls = np.linalg.lstsq(A64, b.astype(np.float64), rcond=1e-4)[0]
    r_min = np.linalg.norm(A64 @ x_ls - b)
    tol = 1e-10 if prec == "f64" else 1e-5
    assert abs(np.linalg.norm(A64 @ x - b) - r_min) <= tol * np.linalg.norm(b)
    # a consistent right-hand side is met to rounding
    x0 = rng.standard_normal(n)
    b0 = (A64 @ x0).astype(dt)
    x = rlu.lstsq(P, Q, L, U, torch.from_numpy(b0).cuda()).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(A64 @ x - b0) <= (1e-10 if prec == "f64" else 1e-4) * np.linalg.norm(b0)
