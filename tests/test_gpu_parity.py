"""Parity of the CUDA path (through the C ABI) with the FP64 oracle. GPU only.

FP64 path: Philox words and G bit-exact; pivots identical up to the first step whose two
largest candidates differ by less than 1e-12 (relative); Y within 1e-13, L_y, B, L, U within
1e-10 (max-norm relative). FP32 path: G bit-exact against the oracle's FP32 transform;
||PAQ - LU||_F within 1.1x the oracle's plus 1e-4 ||A||_2."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth
from tests.gpu_helpers import assert_pivots, leading_agreement, oracle_for, rel_max, run_gpu

pytestmark = pytest.mark.gpu


# ---- step 1 -----------------------------------------------------------------------------

@pytest.mark.parametrize("seed,stream,first,count", [
    (0, 0, 0, 1), (1, 0, 0, 1000), (0x0123456789ABCDEF, 3, (1 << 32) - 5, 37),
    (2**64 - 1, 2**32 - 1, 2**63, 513)])
def test_philox_words_bit_exact(seed, stream, first, count):
    got = rlu.philox_u32(seed, stream, first, count).cpu().numpy().view(np.uint32)
    want = O.philox_stream(seed, stream, first, count)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,l", [(512, 25), (7, 3), (1001, 13), (8192, 210)])
def test_gaussian_fp64_bit_exact(n, l):
    got = rlu.gaussian(5, 0, n, l, torch.float64).cpu().numpy()
    want = O.gaussian(5, 0, n, l)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,l", [(513, 25), (8192, 210)])
def test_gaussian_fp32_bf16_bit_exact(n, l):
    want = O.gaussian_f32(9, 2, n, l)
    got = rlu.gaussian(9, 2, n, l, torch.float32).cpu().numpy()
    assert np.array_equal(got, want)
    gotb = rlu.gaussian(9, 2, n, l, torch.bfloat16).cpu()
    wantb = torch.from_numpy(want).to(torch.bfloat16)
    assert torch.equal(gotb, wantb)


# ---- FP64 path: the 512 x 512, k = 20, l = 25 two-level-spectrum workload ----------------

@pytest.fixture(scope="module")
def fp64_512():
    w = synth.WORKLOADS["fp64_512"]
    A = synth.prescribed_matrix(w["m"], w["n"], synth.spectrum("two_level", w["m"]),
                                w["seed_u"], w["seed_v"])
    g = run_gpu(A, w["k"], w["l"], w["seed_g"], "f64")
    o = oracle_for(A, w["k"], w["l"], w["seed_g"], "f64")
    return A, g, o


def test_fp64_stages_match_oracle(fp64_512):
    A, g, o = fp64_512
    assert np.array_equal(g["G"], o["G"])
    assert rel_max(g["Y"], o["Y"]) < 1e-13
    assert_pivots(g["P"], o["P"], o["gaps_y"], 1e-12)
    assert rel_max(g["Ly"], o["Ly"]) < 1e-10
    assert rel_max(g["B"], o["B"]) < 1e-10


def test_fp64_factors_match_oracle(fp64_512):
    A, g, o = fp64_512
    assert_pivots(g["P"], o["P"], o["gaps_y"], 1e-12)
    assert_pivots(g["Q"], o["Q"], o["gaps_b"], 1e-12)
    assert rel_max(g["L"], o["L"]) < 1e-10
    assert rel_max(g["U"], o["U"]) < 1e-10
    assert g["info"].tolist() == [0, -1, -1, 0]


def test_fp64_reconstruction_error(fp64_512):
    A, g, o = fp64_512
    fro_o, spec_o = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"])
    fro_g, spec_g = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"])
    assert abs(fro_g - fro_o) <= 1e-6 * fro_o
    # the C ABI's error entry point on the GPU's own factors
    At, P, Q, L, U = g["_dev"]
    fro_d, spec_d = rlu.reconstruct_error(At, P, Q, L, U, power_iters=200)
    assert abs(fro_d.item() - fro_g) <= 1e-10 * fro_g
    assert abs(spec_d.item() - spec_g) <= 1e-3 * spec_g
    # Eckart-Young lower bound: sigma_{k+1} = 1e-3 for this spectrum
    assert spec_g >= 1e-3 * (1 - 1e-9)


def test_fp64_deterministic(fp64_512):
    A, g, o = fp64_512
    g2 = run_gpu(A, 20, 25, 1, "f64")
    for key in ("P", "Q", "L", "U", "Y", "B"):
        assert np.array_equal(g[key], g2[key]), key


# ---- FP64 path: ragged sizes, multi-panel clusters and the degenerate cases -------------

@pytest.mark.parametrize("m,n,k,l", [
    (300, 257, 13, 19),        # ragged tiles, single-CTA LUs
    (20000, 300, 30, 40),      # Y needs several panels on a 16-CTA cluster
    (300, 20000, 30, 40),      # B^T needs several panels (Crout form)
    (200, 500, 10, 15),        # wide A
    (64, 40, 40, 40),          # l = min(m, n)
    (1500, 700, 20, 30),       # 3-CTA cluster for Y, 2-CTA for B^T
    (12000, 300, 30, 40),      # 2 rows per thread, panels starting at odd step pairs
    (40000, 64, 10, 16),       # more rows than the register kernel holds: the smem kernel
])
def test_fp64_shapes(m, n, k, l):
    A = synth.lowrank_plus_noise(m, n, min(60, min(m, n)), 1e-6, seed=m + n)
    _check_fp64(A, k, l)


@pytest.mark.parametrize("m,n,k,l", [
    (3000, 400, 90, 100),     # 1 row per thread: blocks of two 36-column panels (Y and B^T)
    (12000, 300, 60, 100),    # 2 rows per thread: blocks of four 18-column panels
    (20000, 300, 60, 130),    # 4 rows per thread: blocks of eleven 6-column panels
    (300, 20000, 90, 100),    # B^T with 4 rows per thread (Crout form), two blocks
])
def test_fp64_blocked_panels(m, n, k, l):
    """Panels grouped into column blocks: within a block each panel updates the rest of the
    block; the block's pivot rows are then solved and its update applied to the columns
    after it. A full-rank Gaussian A keeps every one of the l steps on signal."""
    A = np.random.default_rng(m + 7 * n).standard_normal((m, n))
    _check_fp64(A, k, l)


def _check_fp64(A, k, l):
    g = run_gpu(A, k, l, 3, "f64")
    o = oracle_for(A, k, l, 3, "f64")
    assert np.array_equal(g["G"], o["G"])
    assert_pivots(g["P"], o["P"], o["gaps_y"], 1e-12)
    assert_pivots(g["Q"], o["Q"], o["gaps_b"], 1e-12)
    assert rel_max(g["L"], o["L"]) < 1e-10
    assert rel_max(g["U"], o["U"]) < 1e-10
    fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= fro_o * (1 + 1e-6) + 1e-12 * np.linalg.norm(A)


def test_fp64_square_full_rank_is_exact():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((64, 64))
    g = run_gpu(A, 64, 64, 2, "f64")
    fro, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro / np.linalg.norm(A) < 1e-12


def test_fp64_exact_rank_k():
    A = synth.prescribed_matrix(400, 300, synth.spectrum("rank_k", 300, 10), 5, 6)
    g = run_gpu(A, 10, 14, 7, "f64")
    o = oracle_for(A, 10, 14, 7, "f64")
    # steps beyond rank k pivot on rounding noise: compare the first k pivots only
    assert np.array_equal(g["P"][:10], o["P"][:10])
    fro, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro / np.linalg.norm(A) < 1e-12


def test_fp64_zero_matrix_reports_zero_pivots():
    A = np.zeros((64, 48))
    g = run_gpu(A, 4, 6, 1, "f64")
    assert g["info"].tolist() == [0, 0, 0, 0]
    assert np.array_equal(g["P"], np.arange(64)) and np.array_equal(g["Q"], np.arange(48))
    assert np.all(g["U"] == 0) and np.all(np.isfinite(g["L"]))


def test_nonfinite_input_is_flagged():
    A = synth.lowrank_plus_noise(128, 96, 20, 1e-6, seed=1)
    A[5, 7] = np.nan
    g = run_gpu(A, 4, 8, 1, "f64")
    assert g["info"][3] == 1


def test_invalid_arguments_raise():
    A = torch.zeros((32, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(rlu.RluError):
        rlu.factor(A, 0, 4, 1)
    with pytest.raises(rlu.RluError):
        rlu.factor(A, 5, 17, 1)
    with pytest.raises(rlu.RluError):
        rlu.factor(A.float(), 4, 6, 1, prec="f64")


# ---- FP32 path --------------------------------------------------------------------------

def _fp32_case(m, n, k, l, spec, seed_g, gpu_input=False):
    sigma = synth.spectrum(spec, min(m, n))
    if gpu_input:
        At = synth.prescribed_matrix_torch(m, n, sigma, 21, 22, torch.float32)
        A = At.cpu().numpy()
    else:
        A = synth.prescribed_matrix(m, n, sigma, 21, 22, dtype=np.float32)
    g = run_gpu(A, k, l, seed_g, "f32")
    o = oracle_for(A, k, l, seed_g, "f32")
    return A, g, o, sigma


@pytest.mark.parametrize("m,n,k,l", [(2048, 2048, 64, 74), (1500, 999, 37, 45)])
def test_fp32_error_within_tolerance(m, n, k, l):
    A, g, o, sigma = _fp32_case(m, n, k, l, "inv_square", 2)
    assert np.array_equal(g["G"], O.gaussian_f32(2, 0, n, l))
    fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    # the FP32 rounding moves pivots only at close calls: most leading steps agree
    assert leading_agreement(g["P"], o["P"], l) >= min(10, l)
    At, P, Q, L, U = g["_dev"]
    fro_d, _ = rlu.reconstruct_error(At, P, Q, L, U)
    assert abs(fro_d.item() - fro_g) <= 1e-9 * fro_g


@pytest.mark.parametrize("m,n,k,l", [(12000, 300, 30, 40), (20000, 300, 30, 40),
                                     (20000, 400, 80, 150), (400, 16000, 100, 110)])
def test_fp32_tall_register_configs(m, n, k, l):
    """Y (or B^T) taller than one row per thread of a 16-CTA cluster: 2 and 4 rows per
    thread, with l = 150 (Y) and k = 100 (B^T) spanning several column blocks."""
    A, g, o, sigma = _fp32_case(m, n, k, l, "inv_square", 2)
    fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert leading_agreement(g["P"], o["P"], l) >= min(10, l)
    assert sorted(g["P"].tolist()) == list(range(m))


@pytest.mark.slow
def test_fp32_8192_workload():
    """The full-size FP32 workload (m = n = 8192, k = 200, l = 210, sigma_i = i^-2), in the
    same launch configuration as the benchmark."""
    w = synth.WORKLOADS["fp32_8192"]
    A, g, o, sigma = _fp32_case(w["m"], w["n"], w["k"], w["l"], "inv_square", w["seed_g"],
                                gpu_input=True)
    fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
    fro_g, _ = O.reconstruct_error(A, g["P"], g["Q"], g["L"], g["U"], spectral=False)
    assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (fro_g, fro_o)
    assert np.array_equal(g["G"], O.gaussian_f32(w["seed_g"], 0, w["n"], w["l"]))
    assert sorted(g["P"].tolist()) == list(range(w["m"]))
    assert sorted(g["Q"].tolist()) == list(range(w["n"]))
    assert g["info"].tolist()[:3] == [0, -1, -1]
