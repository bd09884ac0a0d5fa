"""Shared helpers of the GPU parity tests (run the CUDA path through the C ABI, compare with
the oracle)."""
import numpy as np
import torch

import oracle as O
from paper_1310_7202_gb300 import rlu


def run_gpu(A: np.ndarray, k: int, l: int, seed: int, prec: str, q: int = 0,
            normalized: bool = False):
    """Factor A on the GPU through rlu_factor_power (q power iterations, LU-normalised when
    ``normalized``) with the stage outputs; returns numpy copies."""
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    f = rlu.Factorizer(A.shape[0], A.shape[1], k, l, prec, q, normalized)
    st = f.stage_buffers()
    P, Q, L, U, info = f(At, seed, stages=st)
    torch.cuda.synchronize()
    out = {"P": P.cpu().numpy(), "Q": Q.cpu().numpy(), "L": L.cpu().numpy(),
           "U": U.cpu().numpy(), "info": info.cpu().numpy()}
    for name, t in st.items():
        out[name] = t.cpu().numpy()
    out["_dev"] = (At, P, Q, L, U)
    return out


def oracle_for(A: np.ndarray, k: int, l: int, seed: int, prec: str, q: int = 0,
               normalized: bool = False):
    """The oracle on the same stored A; the FP32 path's G definition for prec 'f32'."""
    G = None
    if prec == "f32":
        G = O.gaussian_f32(seed, 0, A.shape[1], l).astype(np.float64)
    return O.rlu_factor(np.asarray(A, dtype=np.float64), k, l, seed=seed, G=G, q=q,
                        normalized=normalized)


def rel_max(a, b) -> float:
    """max |a - b| / max |b|: the normwise (max-norm) relative difference. Entries of L and
    U that are small because of cancellation carry absolute rounding errors of the size of
    the terms that cancelled, so two correct implementations with different summation
    orders agree entrywise only to that absolute level; the bound that backward-error
    analysis gives, and the one tested, is relative to the largest entry."""
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / (scale if scale > 0 else 1.0))


def leading_agreement(p_gpu, p_or, steps: int) -> int:
    """Number of leading pivot steps on which the two pivot sequences agree."""
    neq = np.nonzero(np.asarray(p_gpu[:steps]) != np.asarray(p_or[:steps]))[0]
    return int(neq[0]) if neq.size else steps


def assert_pivots(p_gpu, p_or, gaps, tol):
    """Identical pivots up to the first near-tie step (relative top-two gap < tol); the
    whole permutation when there is none."""
    near = np.nonzero(np.asarray(gaps) < tol)[0]
    steps = len(gaps)
    upto = int(near[0]) if near.size else steps
    if upto == steps:
        assert np.array_equal(p_gpu, p_or), f"pivots differ at {leading_agreement(p_gpu, p_or, len(p_or))}"
    else:
        assert np.array_equal(p_gpu[:upto], p_or[:upto])
    return upto
