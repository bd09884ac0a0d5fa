"""C ABI checks that need no GPU: librlu.so builds, loads, exports every entry point that
include/*.h declares, and rejects bad arguments on the host before any device work."""
import ctypes
import os
import re

import pytest

from paper_1310_7202_gb300 import build as B
from paper_1310_7202_gb300 import rlu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rlu.load_library(require_cuda=False)


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names.update(re.findall(r"\b(rlu_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_binding_exports():
    assert _declared_functions() == sorted(rlu.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert lib.rlu_version() >= 100
    assert lib.rlu_status_string(0) == b"ok"
    assert lib.rlu_status_string(1) == b"invalid argument"


def test_workspace_size_rejects_bad_dims(lib):
    assert lib.rlu_workspace_size(100, 80, 0, 5, 1) == 0        # k < 1
    assert lib.rlu_workspace_size(100, 80, 6, 5, 1) == 0        # k > l
    assert lib.rlu_workspace_size(100, 80, 5, 81, 1) == 0       # l > min(m, n)
    assert lib.rlu_workspace_size(100, 80, 5, 7, 9) == 0        # unknown precision
    assert lib.rlu_workspace_size(100, 80, 5, 7, 1) > 0


def test_factor_rejects_bad_arguments_on_host(lib):
    fake = ctypes.c_void_p(256)  # never dereferenced: validation happens first
    base = dict(A=fake, dtype=1, m=64, n=48, lda=48, k=4, l=6, seed=1, prec=1, P=fake, Q=fake,
                L=fake, ldl=64, U=fake, ldu=48, info=None, ws=fake, wsb=1 << 30, stream=None)

    def call(**over):
        a = dict(base, **over)
        return lib.rlu_factor(a["A"], a["dtype"], a["m"], a["n"], a["lda"], a["k"], a["l"],
                              a["seed"], a["prec"], a["P"], a["Q"], a["L"], a["ldl"], a["U"],
                              a["ldu"], a["info"], a["ws"], a["wsb"], a["stream"])
    assert call(k=0) == rlu.RLU_EINVAL
    assert call(k=7) == rlu.RLU_EINVAL
    assert call(l=49) == rlu.RLU_EINVAL
    assert call(lda=47) == rlu.RLU_EINVAL
    assert call(ldl=63) == rlu.RLU_EINVAL
    assert call(ldu=40) == rlu.RLU_EINVAL
    assert call(A=None) == rlu.RLU_EINVAL
    assert call(dtype=0) == rlu.RLU_EUNSUPPORTED          # FP64 A on the FP32 path
    assert call(prec=5) == rlu.RLU_EUNSUPPORTED
    assert call(wsb=16) == rlu.RLU_ENOMEM
    assert call(ws=ctypes.c_void_p(256 + 8)) == rlu.RLU_EINVAL   # workspace alignment


def test_philox_and_gaussian_reject_bad_arguments(lib):
    assert lib.rlu_philox_u32(1, 0, 0, 4, None, None) == rlu.RLU_EINVAL
    assert lib.rlu_philox_u32(1, 0, 0, -1, ctypes.c_void_p(256), None) == rlu.RLU_EINVAL
    assert lib.rlu_gaussian(1, 0, 10, 3, 0, None, 10, None) == rlu.RLU_EINVAL
    assert lib.rlu_gaussian(1, 0, 10, 3, 0, ctypes.c_void_p(256), 9, None) == rlu.RLU_EINVAL


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(rlu, "_lib", None)
    monkeypatch.setattr(rlu, "LIB_PATH", "/nonexistent/librlu.so")
    with pytest.raises(rlu.RluError):
        rlu.load_library(require_cuda=False)


def test_server_rejects_bad_arguments_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.rlu_server_create(0, 4, ctypes.byref(h)) == rlu.RLU_EINVAL        # no budget
    assert lib.rlu_server_create(1 << 20, 0, ctypes.byref(h)) == rlu.RLU_EINVAL  # no slots
    assert lib.rlu_server_create(1 << 20, 65, ctypes.byref(h)) == rlu.RLU_EINVAL
    assert lib.rlu_server_create(1 << 20, 4, None) == rlu.RLU_EINVAL
    rid = ctypes.c_int64()
    assert lib.rlu_server_submit(None, None, ctypes.byref(rid)) == rlu.RLU_EINVAL
    assert lib.rlu_server_poll(None, 0, None, None, None, None, None) == rlu.RLU_EINVAL
    assert lib.rlu_server_wait_all(None) == rlu.RLU_EINVAL
    assert lib.rlu_server_stats(None, None) == rlu.RLU_EINVAL
    assert lib.rlu_server_destroy(None) == rlu.RLU_EINVAL
