"""Power iterations (Section 5): step 2 becomes Y = (A A^T)^q A G, through rlu_factor_power.
FP64: identical pivots and L, U within 1e-10 (max-norm relative) of the FP64 oracle run with
the same q. The single-precision forms: Y against an FP64 evaluation of (A A^T)^q A G on the
same stored A and G (the products of the rounds are FP32 accurate), and the error against
the oracle's (1.1x its ||PAQ - LU||_F plus 1e-4 ||A||_2). GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth
from tests.gpu_helpers import assert_pivots, oracle_for, rel_max, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,l,q", [
    (600, 500, 20, 30, 1),
    (700, 450, 25, 33, 2),
    (12000, 300, 30, 40, 1),   # several register panels of the LU of Y
])
def test_fp64_power_parity(m, n, k, l, q):
    A = synth.prescribed_matrix(m, n, synth.spectrum("paper_slow", min(m, n)), 5, 6)
    g = run_gpu(A, k, l, 3, "f64", q)
    o = oracle_for(A, k, l, 3, "f64", q)
    assert rel_max(g["Y"], o["Y"]) < 1e-12
    assert_pivots(g["P"], o["P"], o["gaps_y"], 1e-12)
    assert_pivots(g["Q"], o["Q"], o["gaps_b"], 1e-12)
    assert rel_max(g["L"], o["L"]) < 1e-10
    assert rel_max(g["U"], o["U"]) < 1e-10


def _projection_ref(A64, G64, q):
    Y = A64 @ G64
    for _ in range(q):
        Y = A64 @ (A64.T @ Y)
    return Y


@pytest.mark.parametrize("prec,m,n,k,l,q", [
    ("f32", 1000, 800, 20, 30, 1),
    ("mixed", 2048, 1536, 64, 74, 1),
    ("mixed", 1000, 776, 20, 37, 2),     # ragged tiles
    ("mixed", 1000, 777, 20, 37, 1),     # lda not a multiple of 4: SIMT products
    ("bf16", 2048, 1024, 64, 74, 1),
    ("bf16", 1500, 1000, 37, 45, 2),     # ragged tiles
])
def test_single_precision_power(prec, m, n, k, l, q):
    sigma = synth.spectrum("paper_slow", min(m, n))
    A32 = synth.prescribed_matrix(m, n, sigma, 7, 8, dtype=np.float32)
    if prec == "bf16":
        At = torch.from_numpy(A32).to(torch.bfloat16).cuda()
        A64 = At.double().cpu().numpy()
    else:
        At = torch.from_numpy(A32).cuda()
        A64 = A32.astype(np.float64)
    f = rlu.Factorizer(m, n, k, l, prec, q)
    st = f.stage_buffers()
    P, Q, L, U, info = f(At, 4, stages=st)
    torch.cuda.synchronize()
    G32 = st["G"].float().cpu().numpy()
    Y = st["Y"].cpu().numpy().astype(np.float64)
    # the rounds' products are FP32 accurate; the first product is the path's own: BF16 A
    # and G (exact inputs, FP32 accumulation) on the BF16 path, FP32 G read as TF32 by the
    # tensor cores on the mixed path (truncated or rounded to nearest: either reading)
    Gs = [G32]
    if prec == "mixed" and n % 4 == 0:
        bits = G32.view(np.uint32)
        Gs = [(bits & np.uint32(0xFFFFE000)).view(np.float32),
              ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)]
    rel = min(np.linalg.norm(Y - Yr) / np.linalg.norm(Yr)
              for Yr in (_projection_ref(A64, Gx.astype(np.float64), q) for Gx in Gs))
    assert rel < 2e-5, rel
    o = O.rlu_factor(A64, k, l, seed=4, q=q)
    fro_o, _ = O.reconstruct_error(A64, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A64, P.cpu().numpy(), Q.cpu().numpy(), L.cpu().numpy(),
                                   U.cpu().numpy(), spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert info.cpu().tolist()[0] == 0


def test_power_iteration_lowers_the_gpu_error():
    """The claim of the power-iteration subsection on the GPU: q = 1 lowers the error of the
    mixed path on the slow decay sigma_k = 100 / (9 + k)^2."""
    m, n, k, l = 2000, 1500, 40, 48
    sigma = synth.spectrum("paper_slow", min(m, n))
    A32 = synth.prescribed_matrix(m, n, sigma, 9, 10, dtype=np.float32)
    At = torch.from_numpy(A32).cuda()
    errs = []
    for q in (0, 1):
        P, Q, L, U, _ = rlu.Factorizer(m, n, k, l, "mixed", q)(At, 2)
        fro, _ = rlu.reconstruct_error(At, P, Q, L, U)
        errs.append(fro.item())
    assert errs[1] < errs[0], errs
    assert errs[1] >= np.sqrt(np.sum(sigma[k:] ** 2)) * (1 - 1e-6)


# ---- LU-normalised rounds (the normalised scheme the subsection refers to) ---------------

@pytest.mark.parametrize("m,n,k,l,q", [
    (600, 500, 20, 30, 1),
    (700, 450, 25, 33, 3),
    (12000, 300, 30, 40, 1),   # several register panels in the LUs of Y
    (300, 9000, 30, 40, 2),    # the normalisation LU of Z = A^T Y is the tall one
])
def test_fp64_normalized_power_parity(m, n, k, l, q):
    A = synth.prescribed_matrix(m, n, synth.spectrum("paper_slow", min(m, n)), 5, 6)
    g = run_gpu(A, k, l, 3, "f64", q, normalized=True)
    o = oracle_for(A, k, l, 3, "f64", q, normalized=True)
    assert rel_max(g["Y"], o["Y"]) < 1e-11
    assert_pivots(g["P"], o["P"], o["gaps_y"], 1e-12)
    assert_pivots(g["Q"], o["Q"], o["gaps_b"], 1e-12)
    assert rel_max(g["L"], o["L"]) < 1e-10
    assert rel_max(g["U"], o["U"]) < 1e-10
    assert g["info"].tolist()[:3] == [0, -1, -1]


@pytest.mark.parametrize("prec,m,n,k,l,q", [
    ("mixed", 2048, 2048, 64, 74, 1),
    ("mixed", 2048, 2048, 64, 74, 2),
    ("f32", 2048, 2048, 64, 74, 1),
    ("bf16", 2048, 2048, 64, 74, 1),
    ("bf16", 2048, 1536, 64, 74, 2),
    ("mixed", 4096, 4096, 200, 210, 1),   # the bench workload's k and l
])
def test_single_precision_normalized_power_on_inverse_square_spectrum(prec, m, n, k, l, q):
    """sigma_i = i^-2 (the bench workload's spectrum): (sigma_{k+1}/sigma_1)^(2q+1) is far
    below FP32's unit, so unnormalised single-precision rounds lose the trailing directions;
    the LU-normalised rounds must meet the tolerance against the FP64 oracle run with the
    same q (normalised, which in FP64 is as accurate as the exact power iteration) and
    improve on the q = 0 error."""
    sigma = synth.spectrum("inv_square", min(m, n))
    A32 = synth.prescribed_matrix(m, n, sigma, 11, 12, dtype=np.float32)
    if prec == "bf16":
        At = torch.from_numpy(A32).to(torch.bfloat16).cuda()
        A64 = At.double().cpu().numpy()
    else:
        At = torch.from_numpy(A32).cuda()
        A64 = A32.astype(np.float64)
    P, Q, L, U, info = rlu.Factorizer(m, n, k, l, prec, q, normalized=True)(At, 4)
    fro_d, _ = rlu.reconstruct_error(At, P, Q, L, U)
    P0, Q0, L0, U0, _ = rlu.Factorizer(m, n, k, l, prec)(At, 4)
    fro0_d, _ = rlu.reconstruct_error(At, P0, Q0, L0, U0)
    torch.cuda.synchronize()
    o = O.rlu_factor(A64, k, l, seed=4, q=q, normalized=True)
    fro_o, _ = O.reconstruct_error(A64, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    assert fro_d.item() <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_d.item(), fro_o)
    assert fro_d.item() < fro0_d.item(), (fro_d.item(), fro0_d.item())
    assert info.cpu().tolist()[0] == 0
    assert sorted(P.cpu().tolist()) == list(range(m))


def test_normalized_rounds_workspace_and_arguments():
    m, n, k, l = 512, 384, 16, 24
    A = torch.randn(m, n, device="cuda")
    lib = rlu.load_library()
    # the workspace query does not depend on the normalisation
    assert lib.rlu_workspace_size_power(m, n, k, l, rlu.RLU_PREC_MIXED, 2) > \
        lib.rlu_workspace_size(m, n, k, l, rlu.RLU_PREC_MIXED)
    f = rlu.Factorizer(m, n, k, l, "mixed", 2, normalized=True)
    f.normalized = 2  # not 0 or 1: rejected before anything is enqueued
    with pytest.raises(rlu.RluError, match="status 1"):
        f(A, 1)
