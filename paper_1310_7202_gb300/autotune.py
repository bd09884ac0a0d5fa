"""Autotuner of the batched form (include/rlu_batch.h).

It times the kernel choices of a batch on the batch itself and keeps the fastest:
- the SIMT output tile of the three batched products (128 x 128 or 64 x 64);
- the rows each CTA of a problem's LU cluster holds (512 or 256, which sets the cluster
  sizes);
- under mixed precision, one or two CTAs per SM for each tensor-core product (a deep
  staging ring, or a shallower one shared by two CTAs).

Each trial is a CUDA-graph replay of the whole batch, timed with CUDA events (median of
several replays after warm-up). The search is one pass of coordinate descent from the
defaults: each knob is tried in turn with the others fixed at their best so far.

Results are cached in a JSON file keyed by the device name, the precision and a digest of
the problem sizes. The file is $RLU_AUTOTUNE_CACHE, else ~/.cache/rlu_autotune.json. A later
batch with the same sizes takes the cached choice without timing.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import torch

from . import rlu

KNOBS = {
    "lu_rows_per_cta": (512, 256),
    "gemm_tile_y": (0, 1),
    "gemm_tile_c": (0, 1),
    "gemm_tile_l": (0, 1),
    "umma_ctas_y": (1, 2),
    "umma_ctas_c": (1, 2),
}
DEFAULTS = {"lu_rows_per_cta": 512, "gemm_tile_y": 0, "gemm_tile_c": 0, "gemm_tile_l": 0,
            "umma_ctas_y": 1, "umma_ctas_c": 1}


def _cache_path() -> str:
    return os.environ.get("RLU_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rlu_autotune.json"))


def signature(problems: list[dict], prec: str | int) -> str:
    """Device, precision and a digest of the sorted (m, n, k, l) of the batch."""
    sizes = sorted((p["A"].shape[0], p["A"].shape[1], p["k"], p["l"]) for p in problems)
    h = hashlib.sha1(repr(sizes).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name()}|{prec}|{len(problems)}|{h}"


def time_config(problems: list[dict], prec, options: dict, reps: int = 5,
                warmup: int = 2) -> float:
    """Median milliseconds of a graph replay of the batch with these options."""
    b = rlu.Batch(problems, prec, options)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.run()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run()
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del g, b
    torch.cuda.empty_cache()
    return statistics.median(times)


def _applicable(knob: str, prec, problems: list[dict], value) -> bool:
    mixed = prec in ("mixed", rlu.RLU_PREC_MIXED)
    if mixed and knob in ("gemm_tile_y", "gemm_tile_c"):
        return value == DEFAULTS[knob]  # tensor-core products: the SIMT tile is unused
    if not mixed and knob in ("umma_ctas_y", "umma_ctas_c"):
        return value == DEFAULTS[knob]  # SIMT products: no tensor-core ring
    if knob == "gemm_tile_l" and max(p["k"] for p in problems) <= 64:
        return value == DEFAULTS[knob]  # L = L_y L_b runs one thread per row
    if knob == "lu_rows_per_cta":
        tallest = max(max(p["A"].shape) for p in problems)
        return tallest <= 16 * value
    return True


def tune(problems: list[dict], prec="f32", reps: int = 5, use_cache: bool = True) -> dict:
    """Best options for this batch: {"options", "ms", "default_ms", "trials", "cached"}."""
    key = signature(problems, prec)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        hit = dict(cache[key])
        hit["cached"] = True
        return hit
    best = dict(DEFAULTS)
    best_ms = time_config(problems, prec, best, reps)
    default_ms = best_ms
    trials = [{"options": dict(best), "ms": best_ms}]
    for knob, values in KNOBS.items():
        for v in values:
            if v == best[knob] or not _applicable(knob, prec, problems, v):
                continue
            cand = dict(best, **{knob: v})
            ms = time_config(problems, prec, cand, reps)
            trials.append({"options": cand, "ms": ms})
            if ms < best_ms:
                best, best_ms = cand, ms
    result = {"options": best, "ms": best_ms, "default_ms": default_ms, "trials": trials,
              "cached": False}
    if use_cache:
        cache[key] = {k: v for k, v in result.items() if k != "cached"}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return result
