"""Step 5 of Algorithm 1 on its own: B = L_y^+ P A through the normal equations (Gram
matrix, LDL^T factorization, blocked triangular solves), checked against an FP64
least-squares solve with the GPU's own L_y and P, so that pivot choices of the earlier
steps do not enter. The FP32 LDL^T runs on one CTA for k <= 256 and on a cluster of up to
8 CTAs for 256 < k <= 512; the FP64 path takes the FP64 cluster factorization (at k = 400
also the narrow-block triangular solve). GPU only."""
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
    (1200, 1000, 300, 310, "f32"),    # FP32 cluster LDL^T: 10 block rows on 8 CTAs
    (1000, 900, 257, 265, "mixed"),   # the smallest cluster case: a 1-wide last block
    (1500, 1200, 512, 520, "f32"),    # the largest: 16 block rows, two per CTA
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
