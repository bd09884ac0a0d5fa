"""The allocation-free error entry point (rlu_reconstruct_error_static) against the
workspace one (rlu_reconstruct_error), through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory (a framework owning the whole device
pool, or paths where cudaMalloc/cudaFree would synchronise the device): its scratch is a
fixed 8 MiB array inside the library. This file is collected last on purpose: if it fails,
a run that stops at the first failure has already run every other test."""
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


def test_static_entry_point_allocates_nothing():
    """The property the entry point exists for: after one call (which may load the module
    and look up the array's address), further calls leave the device's free memory as it
    was. Every buffer, including the two result doubles, is allocated before the count."""
    lib = rlu.load_library()
    m, n, k, l = 640, 512, 24, 30
    A = synth.prescribed_matrix(m, n, synth.spectrum("inv_square", n), 17, 18, dtype=np.float32)
    At = torch.from_numpy(A).cuda()
    out = rlu.factor(At, k, l, seed=9, prec="f32")
    P, Q, L, U = out["P"], out["Q"], out["L"], out["U"]
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        return lib.rlu_reconstruct_error_static(
            At.data_ptr(), rlu.RLU_F32, m, n, At.stride(0), k, P.data_ptr(), Q.data_ptr(),
            L.data_ptr(), L.stride(1), U.data_ptr(), U.stride(0), rlu.RLU_F32, res.data_ptr(),
            res.data_ptr() + 8, 20, ctypes.c_void_p(stream.cuda_stream))

    assert call() == rlu.RLU_OK  # warm-up: module load and address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert call() == rlu.RLU_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    fro_ws, _ = rlu.reconstruct_error(At, P, Q, L, U)
    torch.cuda.synchronize()
    assert abs(res[0].item() - fro_ws.item()) <= 1e-12 * fro_ws.item()
