"""Seeded synthetic inputs: matrices with a prescribed singular spectrum,
A = U diag(sigma) V^T, U and V the orthonormal factors of the QR of seeded N(0,1)
matrices (sign-fixed so that diag(R) > 0).

This module is shared by the tests, the benchmark and the oracle side. It holds none of
the randomized LU's own arithmetic (its Gaussians come from numpy / torch generators,
not from the factorization's Philox stream).

Spectra used by the paper's experiments (Section 5) and by the workloads built on them:
  * exponential decay (Section 5.1, 3000 x 3000, l = k + 3),
  * sigma_k = 100 / (9 + k)^2 normalised to sigma_1 = 1 (Section 5.2),
and the workload spectra: a two-level spectrum (1 for i <= 20, then 1e-3 * 0.9^(i-21)),
i^-2, 0.99^i, exp(-i/k) and i^-1.5.
"""
from __future__ import annotations

import numpy as np


def spectrum(kind: str, r: int, k: int | None = None) -> np.ndarray:
    """Singular values sigma_1..sigma_r (1-based index i) of a named spectrum."""
    i = np.arange(1, r + 1, dtype=np.float64)
    if kind == "two_level":          # 1 for i <= 20, 1e-3 * 0.9^(i-21) after
        return np.where(i <= 20, 1.0, 1e-3 * 0.9 ** (i - 21))
    if kind == "inv_square":         # i^-2
        return i ** -2.0
    if kind == "geometric_099":      # 0.99^i
        return 0.99 ** i
    if kind == "exp_k":              # exp(-i/k)
        return np.exp(-i / float(k))
    if kind == "inv_1p5":            # i^-1.5
        return i ** -1.5
    if kind == "rank_k":             # exactly rank k: 1 for i <= k, 0 after
        return np.where(i <= k, 1.0, 0.0)
    if kind == "paper_slow":         # 100/(9+i)^2, normalised so that sigma_1 = 1
        s = 100.0 / (9.0 + i) ** 2
        return s / s[0]
    if kind == "paper_exp":          # exponential decay, e^(-i/10) scaled to sigma_1 = 1
        return np.exp(-(i - 1.0) / 10.0)
    raise ValueError(f"unknown spectrum {kind!r}")


def _haar_like_q(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def prescribed_matrix(m: int, n: int, sigma: np.ndarray, seed_u: int, seed_v: int,
                      dtype=np.float64) -> np.ndarray:
    """A = U diag(sigma) V^T (m x n) on the CPU in FP64, then rounded to ``dtype``.
    U is m x r and V is n x r with r = len(sigma) <= min(m, n)."""
    r = len(sigma)
    assert r <= min(m, n)
    U = _haar_like_q(np.random.default_rng(seed_u), m, r)
    V = _haar_like_q(np.random.default_rng(seed_v), n, r)
    A = (U * sigma) @ V.T
    return np.ascontiguousarray(A.astype(dtype))


def round_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) of the FP64 values x, rounded to nearest, ties to even, in
    one step (no intermediate FP32 rounding). Finite values in BF16's normal range."""
    u = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    drop = np.uint64(45)                      # 52 - 7 mantissa bits
    lsb = (u >> drop) & np.uint64(1)
    u = (u + (np.uint64((1 << 44) - 1) + lsb)) >> drop << drop
    return (u.view(np.float64).astype(np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """FP64 values (exact) of BF16 bit patterns."""
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def prescribed_matrix_bf16(m: int, n: int, sigma: np.ndarray, seed_u: int, seed_v: int,
                           rank: int) -> np.ndarray:
    """BF16 bit patterns (uint16, m x n row-major) of A = U diag(sigma) V^T with the first
    ``rank`` singular triplets, built on the CPU in FP64 (U: m x rank and V: n x rank from
    the QR of seeded N(0,1) matrices, as in prescribed_matrix) and rounded to BF16 in one
    step. Dropping sigma_i for i > rank changes A by at most sqrt(sum_{i>rank} sigma_i^2)
    in Frobenius norm; the precision workload takes rank = 2048 for sigma_i = 0.99^i
    (sigma_2049 = 1.1e-9), far below BF16's rounding of A."""
    r = min(rank, len(sigma), m, n)
    U = _haar_like_q(np.random.default_rng(seed_u), m, r)
    V = _haar_like_q(np.random.default_rng(seed_v), n, r)
    U *= sigma[:r]
    out = np.empty((m, n), dtype=np.uint16)
    for i0 in range(0, m, 4096):            # in row blocks: the FP64 product of the whole
        i1 = min(m, i0 + 4096)               # matrix would hold 4 GB at the workload size
        out[i0:i1] = round_to_bf16_bits(U[i0:i1] @ V.T)
    return out


def prescribed_matrix_torch(m: int, n: int, sigma: np.ndarray, seed_u: int, seed_v: int,
                            dtype, device: str = "cuda"):
    """Same construction with torch on ``device`` (for sizes where CPU QR is slow). The
    Gaussians come from torch's generator for that device; the QR and the product run in
    FP32 (or FP64 when ``dtype`` is float64) and the result is rounded to ``dtype``."""
    import torch

    r = len(sigma)
    work = torch.float64 if dtype == torch.float64 else torch.float32

    def q_of(seed, rows):
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        x = torch.randn(rows, r, generator=g, device=device, dtype=work)
        q, rr = torch.linalg.qr(x)
        d = torch.sign(torch.diagonal(rr))
        d[d == 0] = 1.0
        return q * d

    U = q_of(seed_u, m)
    V = q_of(seed_v, n)
    s = torch.as_tensor(sigma, dtype=work, device=device)
    A = (U * s) @ V.T
    return A.to(dtype).contiguous()


def lowrank_plus_noise(m: int, n: int, r: int, noise: float, seed: int,
                       dtype=np.float64) -> np.ndarray:
    """A = X diag(0.8^i) W^T + noise * E with Gaussian X (m x r), W (n x r), E (m x n):
    a fast (QR-free) decaying-spectrum matrix for large parity cases."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, r))
    W = rng.standard_normal((n, r))
    A = (X * 0.8 ** np.arange(r)) @ W.T / np.sqrt(n) + noise * rng.standard_normal((m, n))
    return np.ascontiguousarray(A.astype(dtype))


# The benchmark workloads: size, spectrum, storage and seeds.
WORKLOADS = {
    "fp64_512": dict(m=512, n=512, k=20, l=25, spectrum="two_level", dtype="f64",
                     seed_u=11, seed_v=12, seed_g=1),
    "fp32_8192": dict(m=8192, n=8192, k=200, l=210, spectrum="inv_square", dtype="f32",
                      seed_u=21, seed_v=22, seed_g=2),
    # A built on the CPU from its 2048 leading singular triplets, rounded to BF16 in one step
    # (prescribed_matrix_bf16), so that the stored FP64 oracle result of this matrix applies
    "bf16_32768x16384": dict(m=32768, n=16384, k=512, l=532, spectrum="geometric_099",
                             dtype="bf16", seed_u=31, seed_v=32, seed_g=3, rank=2048),
    # batched form: 4096 problems, sizes from batch_shapes, sigma_i = exp(-i/k), FP32
    "batch4096": dict(kind="batch", count=4096, spectrum="exp_k", dtype="f32", seed_shapes=4,
                      seed_u=41, seed_g=5000),
    # fast randomized LU (Algorithm 4): n x n with l = 3 log2(n)^2 (the timing shape of the
    # paper's comparison of Algorithms 1 and 4), k = 256, sigma_i = i^-2, FP32
    "frlu_4096": dict(kind="fast", m=4096, n=4096, k=256, l=432, spectrum="inv_square",
                      dtype="f32", seed_u=71, seed_v=72, seed_g=73),
    # served form: Poisson arrivals (rates and window from the bench's --serve-* flags)
    "serve": dict(kind="serve", spectrum="inv_1p5", dtype="mixed+bf16"),
}


def srft_params(n: int, l: int, seed: int):
    """Random numbers of the SRFT R = D F S of the fast randomized LU: theta (n FP32 values,
    uniform on [0, 1)) for the diagonal of D, and s (l distinct int32 indices in [0, n), a
    uniformly random ordered selection without replacement) for the columns of S."""
    if not 1 <= l <= n:
        raise ValueError("need 1 <= l <= n")
    rng = np.random.default_rng(seed)
    theta = rng.random(n, dtype=np.float32)
    s = rng.permutation(n)[:l].astype(np.int32)
    return theta, s


def batch_shapes(count: int, seed: int, max_m: int = 2048, max_n: int = 1024):
    """Problem sizes of the batched workload: m log-uniform in [64, max_m], n log-uniform in
    [64, max_n] and at most m, k uniform in {8..64}, l = k + 10; k is drawn again while
    l > n (the sizes must satisfy k <= l <= min(m, n))."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(64), np.log(max_m))))
        n = min(int(np.exp(rng.uniform(np.log(64), np.log(max_n)))), m)
        while True:
            k = int(rng.integers(8, 65))
            if k + 10 <= n:
                break
        out.append((m, n, k, k + 10))
    return out
