"""FP8 form (RLU_PREC_FP8): Y = A G in e4m3 with per-tile power-of-two scales (1 x 128
tiles of A, 128 x 128 tiles of G), FP32 accumulation on the block-scaled tensor cores; the
rest of the path as the BF16 form.

The quantisation rule is restated here in plain torch CPU operations: per tile, 2^e with the
smallest e such that the tile's max |x| <= 448 * 2^e (448 the largest e4m3 value), then
x / 2^e rounded to the nearest e4m3 (ties to even). The GPU's projection must equal the
FP64 product of the dequantised operands to FP32 accumulation accuracy; a single element
quantised differently would move its entries by ~1e-3 relative, far above that bound.
The factorization is then compared with the oracle's steps 3-8 run on that same FP8
projection (the form's own definition), within the reduced-precision tolerance. Its error
against the FP64 oracle with the exact A is measured and reported by the benchmark: e4m3
keeps 4 significant bits, so the quantised A carries ~3% relative noise. GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


def _scale_exp(amax32: np.ndarray) -> np.ndarray:
    """Smallest e with amax <= 448 * 2^e, from the FP32 bits of amax (0 for a zero tile)."""
    b = np.ascontiguousarray(amax32, dtype=np.float32).view(np.uint32).astype(np.int64)
    E = (b >> 23) - 127
    e = E - 8 + ((b & 0x7FFFFF) > 0x600000)
    e = np.where(b < 0x00800000, 0, e)
    return np.clip(e, -126, 126)


def quantize(X: np.ndarray, tile_rows: int, tile_cols: int = 128):
    """e4m3 tiles of X (rows x cols, the K index along the columns) dequantised to FP64,
    and the scale exponents per tile."""
    r, c = X.shape
    rp, cp = -(-r // tile_rows) * tile_rows, -(-c // tile_cols) * tile_cols
    Xp = np.zeros((rp, cp))
    Xp[:r, :c] = X
    T = Xp.reshape(rp // tile_rows, tile_rows, cp // tile_cols, tile_cols)
    amax = np.abs(T).max(axis=(1, 3)).astype(np.float32)
    e = _scale_exp(amax)
    sc = np.exp2(e.astype(np.float64))[:, None, :, None]
    q = np.clip(T / sc, -448.0, 448.0)
    q8 = torch.from_numpy(q).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    return (q8 * sc).reshape(rp, cp)[:r, :c], e


def _case(m, n, k, l, spec, seed):
    sigma = synth.spectrum(spec, min(m, n))
    A32 = synth.prescribed_matrix(m, n, sigma, seed, seed + 1, dtype=np.float32)
    buf = torch.zeros((m, (n + 7) // 8 * 8), dtype=torch.bfloat16)
    buf[:, :n] = torch.from_numpy(A32).to(torch.bfloat16)
    At = buf.cuda()[:, :n]
    A64 = At.double().cpu().numpy()
    f = rlu.Factorizer(m, n, k, l, "fp8")
    st = f.stage_buffers()
    P, Q, L, U, info = f(At, seed, stages=st)
    torch.cuda.synchronize()
    g = {"P": P.cpu().numpy(), "Q": Q.cpu().numpy(), "L": L.cpu().numpy(),
         "U": U.cpu().numpy(), "info": info.cpu().numpy(),
         "G": st["G"].cpu().numpy(), "Y": st["Y"].cpu().numpy().astype(np.float64)}
    return At, A64, sigma, g


@pytest.mark.parametrize("m,n,k,l", [
    (1024, 768, 48, 58),      # whole 128-column blocks, one N tile
    (1000, 700, 37, 45),      # ragged M, a partial last K block, narrow N tile
    (600, 1300, 230, 240),    # two N tiles of G8 (224 + 16), ragged everything
    (300, 256, 20, 24),       # one CTA whose second 128-row accumulator is partly empty
])
def test_fp8_projection_is_the_quantised_product(m, n, k, l):
    At, A64, sigma, g = _case(m, n, k, l, "geometric_099", 3)
    assert np.array_equal(g["G"], O.gaussian_f32(3, 0, n, l))   # FP32 G before quantisation
    A8, _ = quantize(A64, 1)
    G8t, _ = quantize(g["G"].astype(np.float64).T, 128)          # G^T: row j = column j of G
    Yref = A8 @ G8t.T
    err = np.abs(g["Y"] - Yref).max() / np.abs(Yref).max()
    assert err < 2e-6, err
    assert g["info"].tolist()[0] == 0


@pytest.mark.parametrize("m,n,k,l", [(1024, 768, 48, 58), (1500, 1000, 37, 45)])
def test_fp8_factorization_matches_the_oracle_on_its_projection(m, n, k, l):
    """Steps 3-8 of the oracle on the FP8 projection (the FP64 product of the quantised A
    and G): the GPU's factors must meet the reduced-precision tolerance against them."""
    At, A64, sigma, g = _case(m, n, k, l, "geometric_099", 5)
    A8, _ = quantize(A64, 1)
    G8t, _ = quantize(g["G"].astype(np.float64).T, 128)
    Y = A8 @ G8t.T
    Y_lu, P, _, _ = O.lu_partial_pivot(Y)
    Ly = np.tril(Y_lu[:, :k], -1) + np.eye(m, k)
    B = O.pinv_apply(Ly, A64[P, :])
    Lb, Ub, Qo, _, _ = O.lu_column_pivot(B)
    fro_o, _ = O.reconstruct_error(A64, P, Qo, Ly @ Lb, Ub, spectral=False)
    fro_g, _ = O.reconstruct_error(A64, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert sorted(g["P"].tolist()) == list(range(m))
    assert sorted(g["Q"].tolist()) == list(range(n))


def test_fp8_rejects_unaligned_or_non_bf16_input():
    A = torch.zeros(256, 260, dtype=torch.bfloat16, device="cuda")[:, :252]
    with pytest.raises(rlu.RluError, match="status 1"):
        rlu.Factorizer(256, 252, 8, 12, "fp8")(A, 1)
    with pytest.raises(rlu.RluError, match="status 3"):
        rlu.Factorizer(256, 256, 8, 12, "fp8")(torch.zeros(256, 256, device="cuda"), 1)
