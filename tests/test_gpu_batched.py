"""Batched form (include/rlu_batch.h): many uneven FP32 problems per launch sequence, plain
FP32 and mixed (tensor-core products). Each problem is checked against the FP64 oracle (same
FP32 Gaussian, tolerance 1.1x the oracle's ||PAQ - LU||_F plus 1e-4 ||A||_2) and against the
single-problem path; a CUDA-graph replay of the batch reproduces the direct launch bit for
bit. GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth
from tests.gpu_helpers import leading_agreement

pytestmark = pytest.mark.gpu


def _padded(A: np.ndarray) -> torch.Tensor:
    """A on the device with rows padded to a multiple of 4 floats (16-byte aligned rows, as
    the tensor-core products of the mixed precision read them)."""
    m, n = A.shape
    buf = torch.zeros(m, (n + 3) // 4 * 4, device="cuda")
    buf[:, :n] = torch.from_numpy(A).cuda()
    return buf[:, :n]


@pytest.fixture(scope="module", params=["f32", "mixed"])
def batch(request):
    shapes = synth.batch_shapes(40, seed=3, max_m=768, max_n=512)
    probs, mats = [], []
    for i, (m, n, k, l) in enumerate(shapes):
        sigma = np.exp(-np.arange(1, min(m, n) + 1) / k)
        A = synth.prescribed_matrix(m, n, sigma, 100 + i, 200 + i, dtype=np.float32)
        mats.append((A, sigma))
        probs.append({"A": _padded(A), "k": k, "l": l, "seed": 1000 + i})
    b = rlu.Batch(probs, request.param)
    b.run()
    torch.cuda.synchronize()
    res = [{key: v.clone() for key, v in o.items()} for o in b.outs]
    return shapes, mats, probs, b, res


def test_batched_against_oracle(batch):
    shapes, mats, probs, b, res = batch
    for (m, n, k, l), (A, sigma), p, r in zip(shapes, mats, probs, res):
        G = O.gaussian_f32(p["seed"], 0, n, l).astype(np.float64)
        o = O.rlu_factor(A.astype(np.float64), k, l, seed=p["seed"], G=G)
        fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
        P, Q, L, U = (r[x].cpu().numpy() for x in ("P", "Q", "L", "U"))
        fro_g, _ = O.reconstruct_error(A, P, Q, L, U, spectral=False)
        assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (m, n, k, fro_g, fro_o)
        assert sorted(P.tolist()) == list(range(m)) and sorted(Q.tolist()) == list(range(n))
        assert leading_agreement(P, o["P"], l) >= min(5, l), (m, n, k)
        assert r["info"].tolist()[:3] == [0, -1, -1]


def test_batched_matches_single_problem_path(batch):
    shapes, mats, probs, b, res = batch
    for (m, n, k, l), (A, sigma), p, r in zip(shapes, mats, probs, res):
        s = rlu.factor(p["A"], k, l, p["seed"], b.prec)
        fro_s, _ = rlu.reconstruct_error(p["A"], s["P"], s["Q"], s["L"], s["U"])
        fro_b, _ = rlu.reconstruct_error(p["A"], r["P"], r["Q"], r["L"], r["U"])
        assert abs(fro_b.item() - fro_s.item()) <= 0.05 * fro_s.item() + 1e-6, (m, n, k)


def test_graph_replay_reproduces_batch(batch):
    shapes, mats, probs, b, res = batch
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run()  # warm-up outside the capture (kernel attributes are set here)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        b.run()
    for o in b.outs:
        for t in o.values():
            t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(b.outs, res):
        for key in ("P", "Q", "L", "U", "info"):
            assert torch.equal(o[key], r[key]), key
    assert b.launches() <= 10 + 2 * 16


def test_batched_rejects_problems_outside_the_form():
    A = torch.zeros(300, 200, device="cuda")
    with pytest.raises(rlu.RluError):
        rlu.Batch([{"A": A, "k": 80, "l": 90, "seed": 1}])   # l > 76: two LU panels
    with pytest.raises(rlu.RluError):                          # rows not 16-byte aligned
        rlu.Batch([{"A": torch.zeros(300, 203, device="cuda")[:, :201], "k": 8, "l": 18,
                    "seed": 1}], "mixed")


@pytest.mark.parametrize("prec,options", [("f32", {"lu_rows_per_cta": 256}),
                                          ("f32", {"gemm_tile_y": 1, "gemm_tile_c": 1,
                                                   "gemm_tile_l": 1}),
                                          ("mixed", {"umma_ctas_y": 2, "umma_ctas_c": 2})])
def test_batched_kernel_choices_keep_results(prec, options):
    """The autotuner's alternatives (256-row LU CTAs, 64 x 64 SIMT tiles, tensor-core
    products at two CTAs per SM) factor the same problems within the same tolerance."""
    shapes = synth.batch_shapes(12, seed=9, max_m=1100, max_n=600)
    probs, mats = [], []
    for i, (m, n, k, l) in enumerate(shapes):
        sigma = np.exp(-np.arange(1, min(m, n) + 1) / k)
        A = synth.prescribed_matrix(m, n, sigma, 300 + i, 400 + i, dtype=np.float32)
        mats.append((A, sigma))
        probs.append({"A": _padded(A), "k": k, "l": l, "seed": 70 + i})
    b = rlu.Batch(probs, prec, options)
    b.run()
    torch.cuda.synchronize()
    if prec == "mixed":  # a shallower ring keeps the order of every accumulation
        d = rlu.Batch(probs, prec)
        d.run()
        torch.cuda.synchronize()
        for o, od in zip(b.outs, d.outs):
            for key in ("P", "Q", "L", "U"):
                assert torch.equal(o[key], od[key]), key
    for (m, n, k, l), (A, sigma), p, o in zip(shapes, mats, probs, b.outs):
        G = O.gaussian_f32(p["seed"], 0, n, l).astype(np.float64)
        orc = O.rlu_factor(A.astype(np.float64), k, l, seed=p["seed"], G=G)
        fro_o, _ = O.reconstruct_error(A, orc["P"], orc["Q"], orc["L"], orc["U"],
                                       spectral=False)
        fro_g, _ = O.reconstruct_error(A, *(o[x].cpu().numpy() for x in ("P", "Q", "L", "U")),
                                       spectral=False)
        assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (m, n, k, options)


@pytest.mark.parametrize("prec", ["f32", "mixed"])
def test_batched_rank_above_64_takes_the_blocked_kernels(prec):
    """A batch with one problem of k = 66 (l = 76, the register panel's width) runs the
    blocked substitution and the SIMT product for L instead of the k <= 64 register kernels;
    every problem still holds the oracle tolerance."""
    shapes = [(300, 200, 66, 76), (150, 120, 20, 30), (700, 500, 40, 50)]
    probs, mats = [], []
    for i, (m, n, k, l) in enumerate(shapes):
        sigma = np.exp(-np.arange(1, min(m, n) + 1) / k)
        A = synth.prescribed_matrix(m, n, sigma, 500 + i, 600 + i, dtype=np.float32)
        mats.append((A, sigma))
        probs.append({"A": _padded(A), "k": k, "l": l, "seed": 90 + i})
    b = rlu.Batch(probs, prec)
    b.run()
    torch.cuda.synchronize()
    for (m, n, k, l), (A, sigma), p, o in zip(shapes, mats, probs, b.outs):
        G = O.gaussian_f32(p["seed"], 0, n, l).astype(np.float64)
        orc = O.rlu_factor(A.astype(np.float64), k, l, seed=p["seed"], G=G)
        fro_o, _ = O.reconstruct_error(A, orc["P"], orc["Q"], orc["L"], orc["U"],
                                       spectral=False)
        fro_g, _ = O.reconstruct_error(A, *(o[x].cpu().numpy() for x in ("P", "Q", "L", "U")),
                                       spectral=False)
        assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (m, n, k, prec)
        assert o["info"].tolist()[:3] == [0, -1, -1]


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    from paper_1310_7202_gb300 import autotune
    monkeypatch.setenv("RLU_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    shapes = synth.batch_shapes(16, seed=11, max_m=600, max_n=400)
    probs = [{"A": torch.randn(m, (n + 3) // 4 * 4, device="cuda")[:, :n], "k": k, "l": l,
              "seed": i} for i, (m, n, k, l) in enumerate(shapes)]
    r = autotune.tune(probs, "f32", reps=2)
    assert not r["cached"] and r["ms"] <= r["default_ms"]
    for knob, v in r["options"].items():
        assert v in autotune.KNOBS[knob]
    assert len(r["trials"]) >= 4
    again = autotune.tune(probs, "f32", reps=2)
    assert again["cached"] and again["options"] == r["options"]
