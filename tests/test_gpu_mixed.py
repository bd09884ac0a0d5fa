"""The mixed-precision path (RLU_PREC_MIXED): Y = A G on the tcgen05 tensor cores with TF32
inputs. Y is checked against an FP64 product of the same stored A and G; the whole
factorization against the FP64 oracle's error (1.1x the oracle's ||PAQ - LU||_F plus
1e-4 ||A||_2). GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth
from tests.gpu_helpers import oracle_for, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,l", [
    (1024, 1024, 32, 40),     # whole tiles
    (1000, 776, 20, 37),      # ragged M, N (l), K
    (1000, 777, 20, 37),      # lda not a multiple of 4: SIMT fallback for Y
    (300, 5000, 8, 16),       # long K: split-K partials
    (4096, 2048, 200, 210),   # the bench's l
    (2048, 1800, 256, 266),   # l > 256: two N tiles of the tensor-core products
    (3000, 2500, 300, 310),   # k > 256: N tiles in the Gram and C products, FP64 LDL^T
])
def test_mixed_projection_and_error(m, n, k, l):
    sigma = synth.spectrum("inv_square", min(m, n))
    A = synth.prescribed_matrix(m, n, sigma, 3, 4, dtype=np.float32)
    g = run_gpu(A, k, l, 9, "mixed")
    G = O.gaussian_f32(9, 0, n, l).astype(np.float64)
    assert np.array_equal(g["G"], G.astype(np.float32))
    Yref = A.astype(np.float64) @ G
    rel = np.linalg.norm(g["Y"] - Yref) / np.linalg.norm(Yref)
    assert rel < 2e-3, rel           # TF32 inputs: ~2^-11 relative rounding
    o = oracle_for(A, k, l, 9, "f32")
    fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert g["info"].tolist()[0] == 0
