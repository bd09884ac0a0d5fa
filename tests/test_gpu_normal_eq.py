"""Step 5 of Algorithm 1 on its own: B = L_y^+ P A through the normal equations (Gram
matrix, LDL^T factorization, blocked triangular solves), checked against an FP64
least-squares solve with the GPU's own L_y and P, so that pivot choices of the earlier
steps do not enter. The FP32 LDL^T on one CTA serves k <= 256; larger k take the FP64
cluster factorization; the FP64 path at k = 400 takes the narrow-block triangular solve.
GPU only."""
import numpy as np
import pytest

from paper_1310_7202_gb300 import synth
from tests.gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def _case(m, n, k, l, prec, seed):
    sigma = synth.spectrum("inv_square", min(m, n))
    dt = np.float64 if prec == "f64" else np.float32
    A = synth.prescribed_matrix(m, n, sigma, seed, seed + 1, dtype=dt)
    g = run_gpu(A, k, l, seed, prec)
    Ly = g["Ly"].astype(np.float64)
    PA = A.astype(np.float64)[g["P"]]
    B_ref = np.linalg.lstsq(Ly, PA, rcond=None)[0]
    B = g["B"].astype(np.float64)
    return A, Ly, B, B_ref


@pytest.mark.parametrize("m,n,k,l,prec", [
    (2000, 1500, 200, 210, "f32"),    # FP32 LDL^T on one CTA, 7 diagonal blocks, ragged
    (2000, 1500, 200, 210, "mixed"),  # tensor-core Gram and C
    (1200, 1000, 256, 260, "f32"),    # the largest k of the one-CTA factorization
    (1200, 1000, 300, 310, "f32"),    # FP64 cluster LDL^T, FP32 triangular solves
    (700, 650, 33, 40, "f32"),        # one full block and a 1-wide tail
])
def test_normal_equations_single(m, n, k, l, prec):
    A, Ly, B, B_ref = _case(m, n, k, l, prec, 5)
    # the part of B - B_ref that reaches the factorization error ||P A Q - L U||
    proj = np.linalg.norm(Ly @ (B - B_ref)) / np.linalg.norm(A)
    assert proj < 2e-5, proj
    assert np.linalg.norm(B - B_ref) / np.linalg.norm(B_ref) < 5e-3


@pytest.mark.parametrize("m,n,k,l", [(900, 900, 400, 410), (500, 450, 97, 100)])
def test_normal_equations_fp64(m, n, k, l):
    A, Ly, B, B_ref = _case(m, n, k, l, "f64", 6)
    assert np.linalg.norm(B - B_ref) / np.linalg.norm(B_ref) < 1e-9
