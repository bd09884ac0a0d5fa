"""Algorithm 2 (the orthogonal-basis range finder, the comparator of the error experiment of
Section 5) on the GPU through rlu_rsvd, against the FP64 oracle's restatement (LAPACK SVD of
Y): the same G bit for bit, the singular values of Y, the subspace of Q, and the rank-k
error ||Q Q^T A - A||. GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


def _run(A, k, l, seed):
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    r = rlu.rsvd(At, k, l, seed)
    torch.cuda.synchronize()
    return At, {x: r[x].cpu().numpy() for x in ("Q", "B", "sigma", "info")}, r


@pytest.mark.parametrize("m,n,k,l,spec", [
    (500, 400, 20, 30, "paper_exp"),
    (600, 700, 37, 47, "inv_square"),     # odd l: a padding index in the eigensolver
    (300, 300, 1, 1, "paper_slow"),       # one vector
    (2000, 1500, 100, 110, "paper_slow"),
    (1200, 900, 250, 260, "paper_slow"),  # many rounds and sweeps
])
def test_rsvd_matches_the_oracle(m, n, k, l, spec):
    sigma = synth.spectrum(spec, min(m, n))
    A = synth.prescribed_matrix(m, n, sigma, 13, 14)
    At, g, _ = _run(A, k, l, 9)
    o = O.randomized_orth(A, k, l, seed=9)
    sy = o["sigma_y"]
    assert np.abs(g["sigma"] - sy).max() <= 1e-9 * sy[0]
    Q = g["Q"]
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-10
    assert np.abs(g["B"] - Q.T @ A).max() <= 1e-11 * np.abs(A).max() * np.sqrt(m)
    fro_g, _ = O.orth_error(A, Q, g["B"], spectral=False)
    fro_o, _ = O.orth_error(A, o["Q"], spectral=False)
    assert abs(fro_g - fro_o) <= 1e-8 * fro_o, (fro_g, fro_o)
    # the subspaces agree where Y has a gap after its k-th singular value
    if k < l and sy[k] < 0.99 * sy[k - 1]:
        cosines = np.linalg.svd(o["Q"].T @ Q, compute_uv=False)
        assert cosines.min() >= 1 - 1e-8
    assert g["info"].tolist()[0] == 0


def test_rsvd_flags_singular_values_below_the_gram_resolution():
    """sigma_i = e^{-(i-1)/10} with k = 250: sigma_k(Y) / sigma_1(Y) ~ 1e-11, below what the
    eigenvalues of the FP64 Gram matrix resolve (about 1e-7): the unresolved singular values
    come back as 0, their columns of Q as zero, and the status says so; the resolved ones
    still match the oracle's SVD."""
    m, n, k, l = 1200, 900, 250, 260
    sigma = synth.spectrum("paper_exp", n)
    A = synth.prescribed_matrix(m, n, sigma, 13, 14)
    At, g, _ = _run(A, k, l, 9)
    sy = O.randomized_orth(A, k, l, seed=9)["sigma_y"]
    assert g["info"].tolist()[0] == rlu.RLU_EINVAL
    ok = sy > 1e-6 * sy[0]
    assert ok.sum() >= 100
    assert np.abs(g["sigma"][ok] - sy[ok]).max() <= 1e-9 * sy[0]
    assert np.all(g["sigma"][sy < 1e-9 * sy[0]] == 0)


def test_rsvd_exact_rank_and_device_error_measure():
    m, n, k, l = 400, 300, 12, 20
    A = synth.prescribed_matrix(m, n, synth.spectrum("rank_k", min(m, n), k), 3, 4)
    At, g, r = _run(A, k, l, 2)
    fro, _ = O.orth_error(A, g["Q"], g["B"], spectral=False)
    assert fro / np.linalg.norm(A) < 1e-12
    # ||Q B - A|| through the library's error measure with identity permutations
    ident_m = torch.arange(m, dtype=torch.int32, device="cuda")
    ident_n = torch.arange(n, dtype=torch.int32, device="cuda")
    fro_d, _ = rlu.reconstruct_error(At, ident_m, ident_n, r["Q"], r["B"])
    torch.cuda.synchronize()
    assert fro_d.item() / np.linalg.norm(A) < 1e-12


def test_rsvd_and_randomized_lu_on_the_papers_error_shape():
    """The error experiment of Section 5 (3000 x 3000, exponentially decaying singular
    values, l = k + 3): the randomized LU (FP64 path) and Algorithm 2 give errors of the
    same size (the paper: almost identical), both at or above sigma_{k+1}."""
    m = n = 3000
    sigma = synth.spectrum("paper_exp", n)
    A = synth.prescribed_matrix(m, n, sigma, 21, 22)
    At = torch.from_numpy(A).cuda()
    for k in (20, 60):
        r = rlu.rsvd(At, k, k + 3, 4)
        P, Q, L, U, _ = rlu.Factorizer(m, n, k, k + 3, "f64")(At, 4)
        ident_m = torch.arange(m, dtype=torch.int32, device="cuda")
        ident_n = torch.arange(n, dtype=torch.int32, device="cuda")
        _, e_svd = rlu.reconstruct_error(At, ident_m, ident_n, r["Q"], r["B"], power_iters=60)
        _, e_lu = rlu.reconstruct_error(At, P, Q, L, U, power_iters=60)
        torch.cuda.synchronize()
        assert e_svd.item() >= sigma[k] * (1 - 1e-3) and e_lu.item() >= sigma[k] * (1 - 1e-3)
        assert 1 / 3 <= e_lu.item() / e_svd.item() <= 3, (k, e_lu.item(), e_svd.item())


def test_rsvd_rejects_bad_arguments():
    lib = rlu.load_library()
    assert lib.rlu_rsvd_workspace_size(100, 80, 10, 90) == 0     # l > min(m, n)
    assert lib.rlu_rsvd_workspace_size(100, 80, 0, 5) == 0
    A = torch.zeros((64, 48), dtype=torch.float32, device="cuda")
    with pytest.raises(rlu.RluError):
        rlu.rsvd(A, 4, 6, 1)                                     # FP64 only
