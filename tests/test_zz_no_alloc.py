"""The allocation-free error entry point (rlu_reconstruct_error_static) against the
workspace one (rlu_reconstruct_error), through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory (a framework owning the whole device
pool, or paths where cudaMalloc/cudaFree would synchronise the device): its scratch is a
fixed 8 MiB array inside the library. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1310_7202_gb300 import rlu, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,m,n,k,l", [("f32", 1024, 768, 32, 40), ("f64", 300, 257, 13, 19)])
def test_static_scratch_matches_workspace_entry_point(prec, m, n, k, l):
    dt = np.float32 if prec == "f32" else np.float64
    A = synth.prescribed_matrix(m, n, synth.spectrum("inv_square", min(m, n)), 7, 8, dtype=dt)
    At = torch.from_numpy(A).cuda()
    out = rlu.factor(At, k, l, seed=5, prec=prec)
    P, Q, L, U = out["P"], out["Q"], out["L"], out["U"]
    fro_ws, spec_ws = rlu.reconstruct_error(At, P, Q, L, U, power_iters=40)
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        fro_st, spec_st = rlu.reconstruct_error_static(At, P, Q, L, U, power_iters=40)
        torch.cuda.synchronize()
        assert abs(fro_st.item() - fro_ws.item()) <= 1e-12 * fro_ws.item()
        assert abs(spec_st.item() - spec_ws.item()) <= 1e-12 * spec_ws.item()
    # Frobenius only (no power iteration)
    fro2, none = rlu.reconstruct_error_static(At, P, Q, L, U)
    torch.cuda.synchronize()
    assert none is None and abs(fro2.item() - fro_ws.item()) <= 1e-12 * fro_ws.item()


def test_static_scratch_rejects_oversized_problem():
    lib = rlu.load_library()
    A = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    big = 16384  # needs about 9.6 MiB of scratch > 8 MiB: rejected before any launch
    st = lib.rlu_reconstruct_error_static(A.data_ptr(), rlu.RLU_F32, big, big, big, 8,
                                          idx.data_ptr(), idx.data_ptr(), A.data_ptr(), big,
                                          A.data_ptr(), big, rlu.RLU_F32, res.data_ptr(),
                                          None, 0, None)
    assert st == rlu.RLU_ENOMEM
    assert lib.rlu_reconstruct_workspace_size(big, big, 8) > (8 << 20)
