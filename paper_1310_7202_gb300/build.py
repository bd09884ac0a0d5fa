"""Builds the sm_103a shared library ``librlu.so`` in-tree with nvcc (no CMake, no torch
extension machinery): every ``csrc/*.cu`` is compiled in parallel to an object under
``_build/`` and linked with the CUDA runtime into ``paper_1310_7202_gb300/librlu.so``.

Usage: ``python -m paper_1310_7202_gb300.build`` (or ``__graft_entry__.build()``)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build", "rlu")
LIB = os.path.join(PKG, "librlu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librlu.so")


def _flags() -> list[str]:
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _compile(src: str, obj: str) -> None:
    cmd = [nvcc_path(), "-c", src, "-o", obj] + _flags()
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr[-6000:]}")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link librlu.so; returns its path. Skips work when up to date."""
    os.makedirs(BUILD, exist_ok=True)
    # objects built on another host architecture (x86 container vs Arm GPU host) are never
    # reused: the stamp names the machine that built what is under _build/
    stamp = os.path.join(BUILD, "HOST_ARCH")
    host = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != host:
        force = True
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    inc = os.path.join(ROOT, "include")
    headers += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    newest_hdr = max(os.path.getmtime(h) for h in headers)
    jobs = []
    objs = []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if (force or not os.path.exists(obj) or os.path.getmtime(obj) < os.path.getmtime(src)
                or os.path.getmtime(obj) < newest_hdr):
            jobs.append((src, obj))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        futs = [ex.submit(_compile, s, o) for s, o in jobs]
        for f in futs:
            f.result()
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc_path(), "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link of librlu.so failed:\n" + res.stderr[-6000:])
    with open(stamp, "w") as f:
        f.write(host + "\n")
    if verbose:
        print(f"built {LIB} ({len(jobs)} of {len(srcs)} sources compiled)")
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
