"""Writes rlu_bf16_32768x16384.json beside this script: the FP64 oracle of Algorithm 1 run
once on the precision workload's matrix (m = 32768, n = 16384, k = 512, l = 532,
sigma_i = 0.99^i, A stored in BF16), with the oracle's own FP64 Gaussian G (seed 3), and
its reconstruction error ||P A Q - L U|| in the Frobenius and spectral norms.

The stored numbers come from oracle/ alone (synth only builds the input); the GPU tests
and the benchmark compare the precision form's error with them:
    ||PAQ - LU||_F (GPU) <= 1.1 * oracle_fro + 1e-4 * sigma_1.

Run from the repository root (about 2 minutes and 25 GB of host memory on 8 x86 cores):
    python tests/golden/make_precision_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1310_7202_gb300 import synth  # noqa: E402

NAME = "bf16_32768x16384"


def main() -> None:
    w = synth.WORKLOADS[NAME]
    m, n, k, l = w["m"], w["n"], w["k"], w["l"]
    sigma = synth.spectrum(w["spectrum"], min(m, n))
    t0 = time.time()
    bits = synth.prescribed_matrix_bf16(m, n, sigma, w["seed_u"], w["seed_v"], w["rank"])
    sha = hashlib.sha256(bits.tobytes()).hexdigest()
    A = synth.bf16_bits_to_f64(bits)
    del bits
    t1 = time.time()
    res = O.rlu_factor(A, k, l, seed=w["seed_g"])
    t2 = time.time()
    fro, spec = O.reconstruct_error(A, res["P"], res["Q"], res["L"], res["U"], spectral=True)
    t3 = time.time()
    out = {
        "workload": NAME, "m": m, "n": n, "k": k, "l": l, "seed_g": w["seed_g"],
        "spectrum": w["spectrum"], "rank": w["rank"], "seed_u": w["seed_u"],
        "seed_v": w["seed_v"],
        "a_bf16_sha256": sha,
        "oracle": "oracle.rlu_factor (FP64, its own FP64 G) and oracle.reconstruct_error",
        "oracle_fro": fro, "oracle_spec": spec,
        "oracle_P_first_k": [int(x) for x in res["P"][:k]],
        "oracle_Q_first_k": [int(x) for x in res["Q"][:k]],
        "oracle_first_zero_y": int(res["first_zero_y"]),
        "oracle_first_zero_b": int(res["first_zero_b"]),
        "sigma_1": float(sigma[0]), "sigma_k1": float(sigma[k]),
        "a_fro": float(np.linalg.norm(A)),
        "host": f"{platform.machine()} {os.cpu_count()} cores, numpy {np.__version__}",
        "seconds": {"input": round(t1 - t0, 1), "factor": round(t2 - t1, 1),
                    "error": round(t3 - t2, 1)},
    }
    path = os.path.join(HERE, f"rlu_{NAME}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({k_: v for k_, v in out.items() if not k_.startswith("oracle_P")
                      and not k_.startswith("oracle_Q")}))


if __name__ == "__main__":
    main()
