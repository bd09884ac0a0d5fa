"""Serving form (include/rlu_server.h): requests of mixed sizes and precisions admitted by
slot and workspace budget, running concurrently on their own streams. Each result must be
the same in the mix as alone, and within the form's error tolerance of the FP64 oracle.
GPU only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


def _mix(seed=5, count=12):
    """Request shapes drawn like the serving workload (log-uniform m, n; k uniform;
    l = k + 10, k resampled while l > min(m, n)), at sizes the oracle handles quickly. The
    classes cycle through the FP32-accuracy path (mixed), plain FP32, FP64 and the
    BF16-accuracy class (BF16-stored A, the precision form)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(256), np.log(2048))))
        n = int(np.exp(rng.uniform(np.log(256), np.log(2048))))
        while True:
            k = int(rng.integers(16, 65))
            if k + 10 <= min(m, n):
                break
        prec = ["mixed", "f32", "f64", "bf16"][i % 4]
        out.append((m, n, k, k + 10, prec, 100 + i))
    return out


def _matrix(m, n, prec, seed):
    """(the stored values in FP64, the device tensor, sigma); BF16 requests store A in
    BF16 (the FP32 values rounded to nearest even, rows 16-byte aligned) and the oracle
    factors those values."""
    sigma = synth.spectrum("inv_1p5", min(m, n))
    dt = np.float64 if prec == "f64" else np.float32
    A = synth.prescribed_matrix(m, n, sigma, seed, seed + 1, dtype=dt)
    At = torch.from_numpy(A)
    if prec != "bf16":
        return A.astype(np.float64), At.cuda(), sigma
    # the BF16 products read A with TMA: rows padded to a multiple of 8 elements
    buf = torch.zeros((m, (n + 7) // 8 * 8), dtype=torch.bfloat16, device="cuda")
    buf[:, :n] = At.to(torch.bfloat16).cuda()
    Ad = buf[:, :n]
    return Ad.double().cpu().numpy(), Ad, sigma


@pytest.fixture(scope="module")
def served():
    cases = _mix()
    mats = [_matrix(m, n, p, s) for (m, n, k, l, p, s) in cases]
    dev = [At for _, At, _ in mats]
    alone = []
    for (m, n, k, l, p, s), A in zip(cases, dev):
        r = rlu.factor(A, k, l, s, p)
        torch.cuda.synchronize()
        alone.append({key: v.clone() for key, v in r.items()})
    srv = rlu.Server(budget_bytes=512 << 20, max_inflight=4)
    ids = [srv.submit(A, k, l, s, p) for (m, n, k, l, p, s), A in zip(cases, dev)]
    srv.wait_all()
    states = [srv.poll(i) for i in ids]
    mixed = [srv.result(i) for i in ids]
    stats = srv.stats()
    srv.close()
    return cases, mats, alone, mixed, states, stats


def test_every_request_completes(served):
    cases, mats, alone, mixed, states, stats = served
    assert all(s["state"] == rlu.RLU_REQ_DONE for s in states), states
    assert all(s["t_submit"] <= s["t_start"] <= s["t_done"] for s in states)
    assert stats["done"] == len(cases) and stats["failed"] == 0
    assert stats["peak_running"] > 1          # the requests' work overlapped
    assert stats["peak_arena_bytes"] <= 512 << 20


def test_results_same_alone_and_in_mix(served):
    cases, mats, alone, mixed, states, stats = served
    for c, a, b in zip(cases, alone, mixed):
        assert torch.equal(a["P"], b["P"]), c
        assert torch.equal(a["Q"], b["Q"]), c
        assert torch.equal(a["L"], b["L"]), c
        assert torch.equal(a["U"], b["U"]), c
        assert torch.equal(a["info"], b["info"]), c


def test_every_class_is_served(served):
    cases, mats, alone, mixed, states, stats = served
    assert {c[4] for c in cases} == {"mixed", "f32", "f64", "bf16"}


def test_mixed_results_within_tolerance_of_oracle(served):
    cases, mats, alone, mixed, states, stats = served
    for (m, n, k, l, p, s), (A, _, sigma), b in zip(cases, mats, mixed):
        # the oracle draws its own G: FP64 for the FP64 and BF16 classes (the BF16 path's
        # rounding of G counts as error), the FP32 transform for the FP32 classes
        G = None if p in ("f64", "bf16") else O.gaussian_f32(s, 0, n, l).astype(np.float64)
        o = O.rlu_factor(A.astype(np.float64), k, l, seed=s, G=G)
        fro_o, _ = O.reconstruct_error(A, o["P"], o["Q"], o["L"], o["U"], spectral=False)
        fro_g, _ = O.reconstruct_error(A, b["P"].cpu().numpy(), b["Q"].cpu().numpy(),
                                       b["L"].cpu().numpy(), b["U"].cpu().numpy(),
                                       spectral=False)
        if p == "f64":
            assert fro_g <= fro_o * (1 + 1e-6) + 1e-12 * sigma[0], (m, n, k, fro_g, fro_o)
        else:
            assert fro_g <= 1.1 * fro_o + 1e-4 * sigma[0], (m, n, k, p, fro_g, fro_o)


def test_budget_admission_lets_small_requests_pass():
    """A budget that holds one large request: smaller ones queued behind a waiting large
    one are admitted ahead of it, the arena never exceeds the budget, all complete."""
    big = (4096, 4096, 200, 210)
    small = (512, 512, 16, 26)
    ws_big = rlu.workspace_size(*big, rlu.RLU_PREC_MIXED)
    ws_small = rlu.workspace_size(*small, rlu.RLU_PREC_MIXED)
    budget = ws_big + 2 * ws_small + (1 << 20)
    Ab = torch.randn(big[0], big[1], device="cuda")
    As = torch.randn(small[0], small[1], device="cuda")
    srv = rlu.Server(budget_bytes=budget, max_inflight=4)
    ids = [srv.submit(Ab, *big[2:], 1, "mixed"), srv.submit(Ab, *big[2:], 2, "mixed")]
    ids += [srv.submit(As, *small[2:], 10 + i, "mixed") for i in range(6)]
    srv.wait_all()
    st = srv.stats()
    states = [srv.poll(i) for i in ids]
    srv.close()
    assert all(s["state"] == rlu.RLU_REQ_DONE for s in states)
    assert st["peak_arena_bytes"] <= budget
    assert st["bypassed_admissions"] > 0
    # the second large request waited for the first one's memory
    assert states[1]["t_start"] >= states[0]["t_done"]


def test_submit_rejects_oversize_and_bad_requests():
    srv = rlu.Server(budget_bytes=1 << 20, max_inflight=2)
    A = torch.randn(4096, 4096, device="cuda")
    with pytest.raises(rlu.RluError, match="status 2"):
        srv.submit(A, 200, 210, 1, "mixed")      # workspace larger than the whole budget
    with pytest.raises(rlu.RluError):
        srv.submit(A, 0, 10, 1, "mixed", m=64, n=64)   # k < 1
    srv.close()
