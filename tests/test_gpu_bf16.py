"""Precision form (RLU_PREC_BF16): A stored in BF16, Y = A G on the BF16 tensor cores with
FP32 accumulation, C = L~^T A from L~ in three BF16 parts. The projection is checked against
an FP64 product of the same BF16 inputs; B against an FP64 least-squares solve with the
GPU's own L_y; the whole factorization against the FP64 oracle, which factors the same BF16
values with its own unrounded FP64 G (the rounding of G counts as error): tolerance
1.1 x the oracle's ||PAQ - LU||_F plus 1e-4 ||A||_2. GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


def _bf16_case(m, n, k, l, spec, seed):
    sigma = synth.spectrum(spec, min(m, n))
    A32 = synth.prescribed_matrix(m, n, sigma, seed, seed + 1, dtype=np.float32)
    At = torch.from_numpy(A32).to(torch.bfloat16).cuda()
    A64 = At.double().cpu().numpy()   # the stored values, exactly
    f = rlu.Factorizer(m, n, k, l, "bf16")
    st = f.stage_buffers()
    P, Q, L, U, info = f(At, seed, stages=st)
    torch.cuda.synchronize()
    g = {"P": P.cpu().numpy(), "Q": Q.cpu().numpy(), "L": L.cpu().numpy(), "U": U.cpu().numpy(),
         "info": info.cpu().numpy()}
    for key, t in st.items():
        g[key] = t.float().cpu().numpy() if t.dtype == torch.bfloat16 else t.cpu().numpy()
    return At, A64, sigma, g


@pytest.mark.parametrize("m,n,k,l", [
    (2048, 1024, 64, 74),     # whole tiles
    (1500, 1000, 37, 45),     # ragged M, N, K
    (3000, 2000, 300, 310),   # l > 256: two N tiles of Y; k = 300: three N tiles of C
    (200, 160, 20, 24),       # one CTA of Y whose second 128-row tile is empty
])
def test_bf16_factorization(m, n, k, l):
    At, A64, sigma, g = _bf16_case(m, n, k, l, "geometric_099", 7)
    # G: the FP32 transform rounded to BF16, bit for bit
    want_g = torch.from_numpy(O.gaussian_f32(7, 0, n, l)).to(torch.bfloat16).float().numpy()
    assert np.array_equal(g["G"], want_g)
    # Y = A G: exact BF16 inputs, FP32 accumulation
    Yref = A64 @ g["G"].astype(np.float64)
    assert np.linalg.norm(g["Y"] - Yref) / np.linalg.norm(Yref) < 1e-5
    # B = L_y^+ P A with the GPU's own L_y and P: FP32-accurate products and solve
    Ly = g["Ly"].astype(np.float64)
    B_ref = np.linalg.lstsq(Ly, A64[g["P"]], rcond=None)[0]
    proj = np.linalg.norm(Ly @ (g["B"] - B_ref)) / np.linalg.norm(A64)
    # the same stored values through the FP32-accurate TF32-split path: the three-part
    # BF16 product of C must be as accurate (both share the FP32 LDL^T solve, whose error
    # grows with cond(L_y)^2)
    f32 = rlu.Factorizer(m, n, k, l, "mixed")
    st32 = f32.stage_buffers()
    P2, *_ = f32(At.float(), 7, stages=st32)
    torch.cuda.synchronize()
    Ly2 = st32["Ly"].cpu().numpy().astype(np.float64)
    B2_ref = np.linalg.lstsq(Ly2, A64[P2.cpu().numpy()], rcond=None)[0]
    proj2 = np.linalg.norm(Ly2 @ (st32["B"].cpu().numpy() - B2_ref)) / np.linalg.norm(A64)
    assert proj <= 2.0 * proj2 + 1e-6, (proj, proj2)
    # the whole factorization against the FP64 oracle (its own FP64 G)
    o = O.rlu_factor(A64, k, l, seed=7)
    fro_o, _ = O.reconstruct_error(A64, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A64, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert sorted(g["P"].tolist()) == list(range(m))
    assert sorted(g["Q"].tolist()) == list(range(n))
    assert g["info"].tolist()[0] == 0


def test_bf16_device_error_measure_reads_bf16_a():
    At, A64, sigma, g = _bf16_case(1024, 768, 32, 40, "geometric_099", 3)
    fro_h, _ = O.reconstruct_error(A64, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    P, Q = (torch.from_numpy(g[x]).cuda() for x in ("P", "Q"))
    L = torch.from_numpy(g["L"]).cuda()
    U = torch.from_numpy(g["U"]).cuda()
    L = L.t().contiguous().t()  # column-major, as rlu_factor writes it
    fro_d, _ = rlu.reconstruct_error(At, P, Q, L, U)
    assert abs(fro_d.item() - fro_h) <= 1e-6 * fro_h


def test_bf16_rejects_unaligned_rows():
    A = torch.zeros(256, 260, dtype=torch.bfloat16, device="cuda")[:, :252]  # lda = 260
    f = rlu.Factorizer(256, 252, 8, 12, "bf16")
    with pytest.raises(rlu.RluError, match="status 1"):
        f(A, 1)
    with pytest.raises(rlu.RluError, match="status 3"):  # BF16 path needs BF16 storage
        rlu.Factorizer(256, 256, 8, 12, "bf16")(torch.zeros(256, 256, device="cuda"), 1)
