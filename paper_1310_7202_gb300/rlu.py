"""Python binding of the C ABI in include/rlu.h, include/rlu_server.h and include/rlu_batch.h
(ctypes; argument marshalling only).

Every computation runs in librlu.so's CUDA kernels. PyTorch only provides device memory
(the tensors passed in and the outputs allocated here) and the current CUDA stream.
Loading fails loudly if librlu.so has not been built or no CUDA device is present: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librlu.so")

RLU_OK, RLU_EINVAL, RLU_ENOMEM, RLU_EUNSUPPORTED, RLU_ECUDA = 0, 1, 2, 3, 4
RLU_F64, RLU_F32, RLU_BF16 = 0, 1, 2
RLU_PREC_F64, RLU_PREC_F32, RLU_PREC_MIXED, RLU_PREC_BF16, RLU_PREC_FP8 = 0, 1, 2, 3, 4

PREC_BY_NAME = {"f64": RLU_PREC_F64, "f32": RLU_PREC_F32, "mixed": RLU_PREC_MIXED,
                "bf16": RLU_PREC_BF16, "fp8": RLU_PREC_FP8}
_DT_OF_TORCH = {torch.float64: RLU_F64, torch.float32: RLU_F32, torch.bfloat16: RLU_BF16}
_TORCH_OF_PREC = {RLU_PREC_F64: torch.float64, RLU_PREC_F32: torch.float32,
                  RLU_PREC_MIXED: torch.float32, RLU_PREC_BF16: torch.float32,
                  RLU_PREC_FP8: torch.float32}

# Every symbol include/*.h declares.
EXPORTED = ("rlu_version", "rlu_status_string", "rlu_philox_u32", "rlu_gaussian",
            "rlu_workspace_size", "rlu_factor", "rlu_factor_stages", "rlu_timed_step_name",
            "rlu_launch_count", "rlu_reconstruct_workspace_size", "rlu_reconstruct_error",
            "rlu_reconstruct_error_static", "rlu_rsvd_workspace_size", "rlu_rsvd",
            "rlu_server_create", "rlu_server_submit",
            "rlu_server_poll", "rlu_server_wait_all", "rlu_server_stats", "rlu_server_destroy",
            "rlu_batch_workspace_size", "rlu_batch_create", "rlu_factor_batched",
            "rlu_batch_launches", "rlu_batch_destroy", "rlu_workspace_size_power",
            "rlu_factor_power", "rlu_lstsq_workspace_size", "rlu_lstsq",
            "rlu_fast_workspace_size", "rlu_fast_factor", "rlu_srft_workspace_size",
            "rlu_srft_apply")

RLU_REQ_QUEUED, RLU_REQ_RUNNING, RLU_REQ_DONE, RLU_REQ_FAILED = 0, 1, 2, 3


class RluError(RuntimeError):
    pass


class _Request(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("k", ctypes.c_int32),
                ("l", ctypes.c_int32), ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32),
                ("P", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("ldl", ctypes.c_int64), ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64),
                ("info", ctypes.c_void_p)]


class _Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("P", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("L", ctypes.c_void_p), ("ldl", ctypes.c_int64), ("U", ctypes.c_void_p),
                ("ldu", ctypes.c_int64), ("info", ctypes.c_void_p)]


class _BatchOptions(ctypes.Structure):
    _fields_ = [("gemm_tile_y", ctypes.c_int32), ("gemm_tile_c", ctypes.c_int32),
                ("gemm_tile_l", ctypes.c_int32), ("lu_rows_per_cta", ctypes.c_int32),
                ("umma_ctas_y", ctypes.c_int32), ("umma_ctas_c", ctypes.c_int32)]


class _StageOutputs(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("Ly", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("events", ctypes.POINTER(ctypes.c_void_p)),
                ("n_events", ctypes.c_int32)]


NUM_TIMED_STEPS = 11


_lib = None


def load_library(require_cuda: bool = True) -> ctypes.CDLL:
    """Load librlu.so and declare the prototypes of include/rlu.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RluError(f"{LIB_PATH} is missing: build it with "
                       "`python -m paper_1310_7202_gb300.build` (no CPU fallback exists)")
    if require_cuda and not torch.cuda.is_available():
        raise RluError("librlu needs a CUDA device (sm_103a); none is available")
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, u32, u64, vp, sz = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t)
    lib.rlu_version.restype = i32
    lib.rlu_version.argtypes = []
    lib.rlu_status_string.restype = ctypes.c_char_p
    lib.rlu_status_string.argtypes = [i32]
    lib.rlu_philox_u32.restype = i32
    lib.rlu_philox_u32.argtypes = [u64, u32, u64, i64, vp, vp]
    lib.rlu_gaussian.restype = i32
    lib.rlu_gaussian.argtypes = [u64, u32, i64, i64, i32, vp, i64, vp]
    lib.rlu_workspace_size.restype = sz
    lib.rlu_workspace_size.argtypes = [i64, i64, i32, i32, i32]
    fac = [vp, i32, i64, i64, i64, i32, i32, u64, i32, vp, vp, vp, i64, vp, i64, vp, vp, sz]
    lib.rlu_factor.restype = i32
    lib.rlu_factor.argtypes = fac + [vp]
    lib.rlu_factor_stages.restype = i32
    lib.rlu_factor_stages.argtypes = fac + [ctypes.POINTER(_StageOutputs), vp]
    lib.rlu_lstsq_workspace_size.restype = sz
    lib.rlu_lstsq_workspace_size.argtypes = [i64, i64, i32, i32, i32]
    lib.rlu_lstsq.restype = i32
    lib.rlu_lstsq.argtypes = [i32, i64, i64, i32, vp, vp, vp, i64, vp, i64, vp, i64, i32, vp,
                              i64, vp, vp, sz, vp]
    lib.rlu_workspace_size_power.restype = sz
    lib.rlu_workspace_size_power.argtypes = [i64, i64, i32, i32, i32, i32]
    lib.rlu_factor_power.restype = i32
    lib.rlu_factor_power.argtypes = fac[:9] + [i32, i32] + fac[9:] + [ctypes.POINTER(_StageOutputs),
                                                                vp]
    lib.rlu_timed_step_name.restype = ctypes.c_char_p
    lib.rlu_timed_step_name.argtypes = [i32]
    lib.rlu_launch_count.restype = ctypes.c_uint64
    lib.rlu_launch_count.argtypes = []
    lib.rlu_reconstruct_workspace_size.restype = sz
    lib.rlu_reconstruct_workspace_size.argtypes = [i64, i64, i32]
    lib.rlu_reconstruct_error.restype = i32
    lib.rlu_reconstruct_error.argtypes = [vp, i32, i64, i64, i64, i32, vp, vp, vp, i64, vp, i64,
                                          i32, vp, vp, i32, vp, sz, vp]
    lib.rlu_reconstruct_error_static.restype = i32
    lib.rlu_reconstruct_error_static.argtypes = [vp, i32, i64, i64, i64, i32, vp, vp, vp, i64,
                                                 vp, i64, i32, vp, vp, i32, vp]
    lib.rlu_rsvd_workspace_size.restype = sz
    lib.rlu_rsvd_workspace_size.argtypes = [i64, i64, i32, i32]
    lib.rlu_rsvd.restype = i32
    lib.rlu_rsvd.argtypes = [vp, i32, i64, i64, i64, i32, i32, u64, vp, i64, vp, i64, vp, vp,
                             vp, sz, vp]
    lib.rlu_server_create.restype = i32
    lib.rlu_server_create.argtypes = [sz, i32, ctypes.POINTER(vp)]
    lib.rlu_server_submit.restype = i32
    lib.rlu_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(i64)]
    lib.rlu_server_poll.restype = i32
    lib.rlu_server_poll.argtypes = [vp, i64] + [ctypes.POINTER(i32)] * 2 + [ctypes.POINTER(i64)] * 3
    lib.rlu_server_wait_all.restype = i32
    lib.rlu_server_wait_all.argtypes = [vp]
    lib.rlu_server_stats.restype = i32
    lib.rlu_server_stats.argtypes = [vp, ctypes.POINTER(i64)]
    lib.rlu_server_destroy.restype = i32
    lib.rlu_server_destroy.argtypes = [vp]
    lib.rlu_batch_workspace_size.restype = sz
    lib.rlu_batch_workspace_size.argtypes = [ctypes.POINTER(_Problem), i32, i32]
    lib.rlu_batch_create.restype = i32
    lib.rlu_batch_create.argtypes = [ctypes.POINTER(_Problem), i32, i32,
                                     ctypes.POINTER(_BatchOptions), vp, sz, ctypes.POINTER(vp)]
    lib.rlu_factor_batched.restype = i32
    lib.rlu_factor_batched.argtypes = [vp, vp]
    lib.rlu_batch_launches.restype = i32
    lib.rlu_batch_launches.argtypes = [vp]
    lib.rlu_batch_destroy.restype = i32
    lib.rlu_batch_destroy.argtypes = [vp]
    lib.rlu_fast_workspace_size.restype = sz
    lib.rlu_fast_workspace_size.argtypes = [i64, i64, i32, i32]
    lib.rlu_srft_workspace_size.restype = sz
    lib.rlu_srft_workspace_size.argtypes = [i64]
    lib.rlu_srft_apply.restype = i32
    lib.rlu_srft_apply.argtypes = [vp, i64, i64, i64, vp, vp, i32, vp, i64, vp, vp, sz, vp]
    lib.rlu_fast_factor.restype = i32
    lib.rlu_fast_factor.argtypes = [vp, i64, i64, i64, i32, i32, vp, vp, vp, vp, vp, i64, vp,
                                    i64, vp, vp, sz, vp]
    _lib = lib
    return lib


def _check(status: int, what: str) -> None:
    if status != RLU_OK:
        msg = _lib.rlu_status_string(status).decode() if _lib else str(status)
        raise RluError(f"{what} failed: {msg} (status {status})")


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else int(t.data_ptr())


def philox_u32(seed: int, stream_id: int, first_counter: int, n_counters: int,
               stream=None) -> torch.Tensor:
    """Raw Philox4x32-10 words (int32 tensor holding the uint32 bit patterns)."""
    lib = load_library()
    out = torch.empty(4 * max(n_counters, 1), dtype=torch.int32, device="cuda")
    _check(lib.rlu_philox_u32(seed, stream_id, first_counter, n_counters, _dev_ptr(out),
                              _stream_ptr(stream)), "rlu_philox_u32")
    return out[: 4 * n_counters]


def gaussian(seed: int, stream_id: int, n: int, l: int, dtype=torch.float64,
             stream=None) -> torch.Tensor:
    """Step 1: G (n x l) as an (n, l) tensor with column-major storage."""
    lib = load_library()
    store = torch.empty((l, n), dtype=dtype, device="cuda")
    _check(lib.rlu_gaussian(seed, stream_id, n, l, _DT_OF_TORCH[dtype], _dev_ptr(store), n,
                            _stream_ptr(stream)), "rlu_gaussian")
    return store.t()


def workspace_size(m: int, n: int, k: int, l: int, prec: int) -> int:
    return int(load_library().rlu_workspace_size(m, n, k, l, prec))


def _colmajor(rows: int, cols: int, dtype) -> torch.Tensor:
    return torch.empty((cols, rows), dtype=dtype, device="cuda").t()


class Factorizer:
    """Reusable buffers (outputs, workspace, info) for repeated rlu_factor calls of one
    size and precision."""

    def __init__(self, m: int, n: int, k: int, l: int, prec: int | str = RLU_PREC_F32,
                 q: int = 0, normalized: bool = False):
        self.lib = load_library()
        self.prec = PREC_BY_NAME[prec] if isinstance(prec, str) else int(prec)
        self.m, self.n, self.k, self.l, self.q = m, n, k, l, q
        self.normalized = 1 if normalized else 0  # LU-normalised power-iteration rounds
        dt = _TORCH_OF_PREC[self.prec]
        self.dtype = dt
        ws = self.lib.rlu_workspace_size_power(m, n, k, l, self.prec, q)
        if ws == 0:
            raise RluError(f"invalid sizes m={m} n={n} k={k} l={l} prec={self.prec}")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device="cuda")
        self.P = torch.empty(m, dtype=torch.int32, device="cuda")
        self.Q = torch.empty(n, dtype=torch.int32, device="cuda")
        self.L = _colmajor(m, k, dt)
        self.U = torch.empty((k, n), dtype=dt, device="cuda")
        self.info = torch.empty(4, dtype=torch.int32, device="cuda")

    def __call__(self, A: torch.Tensor, seed: int, stages: dict | None = None, stream=None):
        """Enqueue rlu_factor(A) on the current stream; returns (P, Q, L, U, info)."""
        m, n, k, l = self.m, self.n, self.k, self.l
        if A.shape != (m, n) or A.stride(1) != 1 or A.device.type != "cuda":
            raise RluError("A must be a row-major (m, n) CUDA tensor")
        dt = _DT_OF_TORCH[A.dtype]
        args = [_dev_ptr(A), dt, m, n, A.stride(0), k, l, seed, self.prec,
                _dev_ptr(self.P), _dev_ptr(self.Q), _dev_ptr(self.L), self.L.stride(1),
                _dev_ptr(self.U), self.U.stride(0), _dev_ptr(self.info),
                _dev_ptr(self.workspace), self.workspace.numel()]
        if stages is None and self.q == 0:
            st = self.lib.rlu_factor(*args, _stream_ptr(stream))
        elif stages is None:
            st = self.lib.rlu_factor_power(*args[:9], self.q, self.normalized, *args[9:], None,
                                           _stream_ptr(stream))
        else:
            ev = stages.get("events")
            ev_arr, n_ev = None, 0
            if ev is not None:
                for e in ev:  # torch creates the CUDA event on its first record
                    if int(e.cuda_event) == 0:
                        e.record()
                ev_arr = (ctypes.c_void_p * len(ev))(*[int(e.cuda_event) for e in ev])
                n_ev = len(ev)
            so = _StageOutputs(_dev_ptr(stages.get("G")), _dev_ptr(stages.get("Y")),
                               _dev_ptr(stages.get("Ly")), _dev_ptr(stages.get("B")),
                               ctypes.cast(ev_arr, ctypes.POINTER(ctypes.c_void_p))
                               if ev_arr is not None else None, n_ev)
            st = self.lib.rlu_factor_power(*args[:9], self.q, self.normalized, *args[9:],
                                           ctypes.byref(so), _stream_ptr(stream))
        _check(st, "rlu_factor")
        return self.P, self.Q, self.L, self.U, self.info

    def stage_buffers(self) -> dict:
        """Column-/row-major tensors laid out as rlu_stage_outputs expects."""
        m, n, k, l, dt = self.m, self.n, self.k, self.l, self.dtype
        gdt = torch.bfloat16 if self.prec == RLU_PREC_BF16 else dt  # G in the BF16 form
        return {"G": _colmajor(n, l, gdt), "Y": _colmajor(m, l, dt), "Ly": _colmajor(m, k, dt),
                "B": torch.empty((k, n), dtype=dt, device="cuda")}


def factor(A: torch.Tensor, k: int, l: int, seed: int, prec: int | str | None = None,
           stages: bool = False, q: int = 0, normalized: bool = False) -> dict:
    """One randomized LU of A (CUDA tensor, row-major). Returns P, Q, L, U, info (device
    tensors) and, with ``stages=True``, the intermediates G, Y, Ly, B."""
    if prec is None:
        prec = {torch.float64: RLU_PREC_F64, torch.bfloat16: RLU_PREC_BF16}.get(A.dtype,
                                                                               RLU_PREC_F32)
    f = Factorizer(A.shape[0], A.shape[1], k, l, prec, q, normalized)
    st = f.stage_buffers() if stages else None
    P, Q, L, U, info = f(A, seed, stages=st)
    out = {"P": P, "Q": Q, "L": L, "U": U, "info": info}
    if st:
        out.update(st)
    return out


def lstsq(P: torch.Tensor, Q: torch.Tensor, L: torch.Tensor, U: torch.Tensor,
          b: torch.Tensor, info: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Algorithm 3: x (n, or n x r) minimising ||A x - b|| from the factors of rlu_factor
    (L column-major, U row-major, b of L's dtype: (m,) or (m, r) column-major)."""
    lib = load_library()
    m, k = L.shape
    n = U.shape[1]
    if L.stride(0) != 1 or U.stride(1) != 1:
        raise RluError("L must be column-major and U row-major")
    vec = b.dim() == 1
    B = b.reshape(m, 1) if vec else b
    if B.stride(0) != 1:
        B = B.t().contiguous().t()
    r = B.shape[1]
    X = torch.empty((r, n), dtype=L.dtype, device="cuda").t()
    dt = _DT_OF_TORCH[L.dtype]
    ws_n = lib.rlu_lstsq_workspace_size(m, n, k, r, dt)
    if ws_n == 0:
        raise RluError(f"invalid sizes m={m} n={n} k={k} nrhs={r}")
    ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
    _check(lib.rlu_lstsq(dt, m, n, k, _dev_ptr(P), _dev_ptr(Q), _dev_ptr(L), L.stride(1),
                         _dev_ptr(U), U.stride(0), _dev_ptr(B), B.stride(1) if r > 1 else m,
                         r, _dev_ptr(X), X.stride(1) if r > 1 else n, _dev_ptr(info),
                         _dev_ptr(ws), ws_n, _stream_ptr(stream)),
           "rlu_lstsq")
    return X[:, 0] if vec else X


class FastFactorizer:
    """Algorithm 4 (include/rlu_fast.h) for one problem size, with its workspace allocated
    once: run(A, theta, s) factors a row-major FP32 CUDA matrix with the SRFT random numbers
    theta (n FP32 in [0, 1)) and s (l distinct int32 indices) and returns P, Q, L (m x k
    complex64, column-major), U (k x n complex64, row-major) and info."""

    def __init__(self, m: int, n: int, k: int, l: int):
        self.lib = load_library()
        self.m, self.n, self.k, self.l = m, n, k, l
        ws = self.lib.rlu_fast_workspace_size(m, n, k, l)
        if ws == 0:
            raise RluError(f"sizes outside the fast randomized LU: m={m} n={n} k={k} l={l}")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device="cuda")

    def run(self, A: torch.Tensor, theta: torch.Tensor, s: torch.Tensor, out: dict | None = None,
            stream=None) -> dict:
        m, n, k, l = self.m, self.n, self.k, self.l
        if A.shape != (m, n) or A.dtype != torch.float32 or A.stride(1) != 1:
            raise RluError("A must be a row-major FP32 CUDA matrix of the planned size")
        if theta.dtype != torch.float32 or theta.numel() != n or s.dtype != torch.int32 or s.numel() != l:
            raise RluError("theta must hold n FP32 values and s l int32 indices")
        o = out if out is not None else {
            "P": torch.empty(m, dtype=torch.int32, device="cuda"),
            "Q": torch.empty(n, dtype=torch.int32, device="cuda"),
            "L": torch.empty((k, m), dtype=torch.complex64, device="cuda").t(),
            "U": torch.empty((k, n), dtype=torch.complex64, device="cuda"),
            "info": torch.empty(4, dtype=torch.int32, device="cuda")}
        _check(self.lib.rlu_fast_factor(
            _dev_ptr(A), m, n, A.stride(0), k, l, _dev_ptr(theta.contiguous()),
            _dev_ptr(s.contiguous()), _dev_ptr(o["P"]), _dev_ptr(o["Q"]), _dev_ptr(o["L"]),
            o["L"].stride(1), _dev_ptr(o["U"]), o["U"].stride(0), _dev_ptr(o["info"]),
            _dev_ptr(self.workspace), self.workspace.numel(), _stream_ptr(stream)),
            "rlu_fast_factor")
        return o


def srft_apply(A: torch.Tensor, theta: torch.Tensor, s: torch.Tensor,
               info: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Steps 1-2 of Algorithm 4: Y = A D F S (m x l complex64, row-major)."""
    lib = load_library()
    m, n = A.shape
    l = s.numel()
    if A.dtype != torch.float32 or A.stride(1) != 1:
        raise RluError("A must be a row-major FP32 CUDA matrix")
    ws_n = lib.rlu_srft_workspace_size(n)
    if ws_n == 0:
        raise RluError(f"n={n} is outside the row transform's sizes")
    ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
    Y = torch.empty((m, l), dtype=torch.complex64, device="cuda")
    _check(lib.rlu_srft_apply(_dev_ptr(A), m, n, A.stride(0), _dev_ptr(theta.contiguous()),
                              _dev_ptr(s.contiguous()), l, _dev_ptr(Y), l, _dev_ptr(info),
                              _dev_ptr(ws), ws_n, _stream_ptr(stream)), "rlu_srft_apply")
    return Y


def fast_factor(A: torch.Tensor, k: int, l: int, theta, s, stream=None) -> dict:
    """One call of Algorithm 4 (allocates its workspace); theta and s may be numpy arrays."""
    m, n = A.shape
    th = torch.as_tensor(theta, dtype=torch.float32).cuda()
    ss = torch.as_tensor(s, dtype=torch.int32).cuda()
    return FastFactorizer(m, n, k, l).run(A, th, ss, stream=stream)


def timed_step_names() -> list[str]:
    lib = load_library(require_cuda=False)
    return [lib.rlu_timed_step_name(i).decode() for i in range(NUM_TIMED_STEPS)]


def launch_count() -> int:
    return int(load_library(require_cuda=False).rlu_launch_count())


def reconstruct_error(A: torch.Tensor, P: torch.Tensor, Q: torch.Tensor, L: torch.Tensor,
                      U: torch.Tensor, power_iters: int = 0, stream=None):
    """(||PAQ - LU||_F, ||PAQ - LU||_2 estimate or None) as device FP64 scalars."""
    lib = load_library()
    m, n = A.shape
    k = L.shape[1]
    if L.stride(0) != 1 or U.stride(1) != 1 or A.stride(1) != 1:
        raise RluError("L must be column-major, U and A row-major")
    ws = torch.empty(lib.rlu_reconstruct_workspace_size(m, n, k), dtype=torch.uint8,
                     device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    spec_ptr = _dev_ptr(out) + 8 if power_iters > 0 else None
    _check(lib.rlu_reconstruct_error(_dev_ptr(A), _DT_OF_TORCH[A.dtype], m, n, A.stride(0), k,
                                     _dev_ptr(P), _dev_ptr(Q), _dev_ptr(L), L.stride(1),
                                     _dev_ptr(U), U.stride(0), _DT_OF_TORCH[L.dtype],
                                     _dev_ptr(out), spec_ptr, power_iters, _dev_ptr(ws),
                                     ws.numel(), _stream_ptr(stream)),
           "rlu_reconstruct_error")
    return out[0], (out[1] if power_iters > 0 else None)


def rsvd(A: torch.Tensor, k: int, l: int, seed: int, stream=None) -> dict:
    """Algorithm 2 (the comparator of Section 5) on an FP64 row-major CUDA tensor A: Q
    (m x k, column-major, orthonormal), B = Q^T A (k x n), sigma (the l singular values of
    Y = A G, decreasing) and info (device tensors)."""
    lib = load_library()
    m, n = A.shape
    if A.dtype != torch.float64 or A.stride(1) != 1 or A.device.type != "cuda":
        raise RluError("A must be a row-major FP64 CUDA tensor")
    ws_n = lib.rlu_rsvd_workspace_size(m, n, k, l)
    if ws_n == 0:
        raise RluError(f"invalid sizes m={m} n={n} k={k} l={l}")
    ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
    Q = _colmajor(m, k, torch.float64)
    B = torch.empty((k, n), dtype=torch.float64, device="cuda")
    sigma = torch.empty(l, dtype=torch.float64, device="cuda")
    info = torch.empty(4, dtype=torch.int32, device="cuda")
    _check(lib.rlu_rsvd(_dev_ptr(A), RLU_F64, m, n, A.stride(0), k, l, seed, _dev_ptr(Q),
                        Q.stride(1), _dev_ptr(B), B.stride(0), _dev_ptr(sigma), _dev_ptr(info),
                        _dev_ptr(ws), ws_n, _stream_ptr(stream)), "rlu_rsvd")
    return {"Q": Q, "B": B, "sigma": sigma, "info": info, "_ws": ws}


def reconstruct_error_static(A: torch.Tensor, P: torch.Tensor, Q: torch.Tensor,
                             L: torch.Tensor, U: torch.Tensor, power_iters: int = 0,
                             stream=None):
    """reconstruct_error without a workspace: the library's fixed 8 MiB device scratch is
    used instead, for callers that must not allocate device memory (only the two-double
    result tensor is allocated here, by this Python convenience wrapper)."""
    lib = load_library()
    m, n = A.shape
    k = L.shape[1]
    if L.stride(0) != 1 or U.stride(1) != 1 or A.stride(1) != 1:
        raise RluError("L must be column-major, U and A row-major")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    spec_ptr = _dev_ptr(out) + 8 if power_iters > 0 else None
    _check(lib.rlu_reconstruct_error_static(
        _dev_ptr(A), _DT_OF_TORCH[A.dtype], m, n, A.stride(0), k, _dev_ptr(P), _dev_ptr(Q),
        _dev_ptr(L), L.stride(1), _dev_ptr(U), U.stride(0), _DT_OF_TORCH[L.dtype],
        _dev_ptr(out), spec_ptr, power_iters, _stream_ptr(stream)),
        "rlu_reconstruct_error_static")
    return out[0], (out[1] if power_iters > 0 else None)


class Server:
    """The serving loop of include/rlu_server.h: requests of mixed sizes and precisions are
    admitted as slots and workspace memory (a fixed device budget) free up, and run
    concurrently on their own streams. A and the outputs stay resident on the device; this
    wrapper allocates the outputs of each request (P, Q, L, U, info) with torch at submission
    and keeps references until the request is done."""

    def __init__(self, budget_bytes: int, max_inflight: int = 8):
        self.lib = load_library()
        h = ctypes.c_void_p()
        _check(self.lib.rlu_server_create(budget_bytes, max_inflight, ctypes.byref(h)),
               "rlu_server_create")
        self.h = h
        self.live: dict[int, dict] = {}

    def submit(self, A: torch.Tensor, k: int, l: int, seed: int, prec: int | str,
               m: int | None = None, n: int | None = None) -> int:
        """Queue a factorization of the top-left m x n block of the row-major CUDA tensor A
        (all of A by default); returns the request id."""
        prec = PREC_BY_NAME[prec] if isinstance(prec, str) else int(prec)
        m = A.shape[0] if m is None else m
        n = A.shape[1] if n is None else n
        if A.stride(1) != 1 or A.device.type != "cuda" or m > A.shape[0] or n > A.shape[1]:
            raise RluError("A must be a row-major CUDA tensor holding the m x n block")
        dt = _TORCH_OF_PREC[prec]
        out = {"P": torch.empty(m, dtype=torch.int32, device="cuda"),
               "Q": torch.empty(n, dtype=torch.int32, device="cuda"),
               "L": _colmajor(m, k, dt), "U": torch.empty((k, n), dtype=dt, device="cuda"),
               "info": torch.empty(4, dtype=torch.int32, device="cuda"), "A": A}
        # the outputs were allocated on torch's current stream; the request runs on a slot
        # stream of the server, so make the allocations visible before it can start
        torch.cuda.current_stream().synchronize()
        r = _Request(_dev_ptr(A), _DT_OF_TORCH[A.dtype], m, n, A.stride(0), k, l, seed, prec,
                     _dev_ptr(out["P"]), _dev_ptr(out["Q"]), _dev_ptr(out["L"]),
                     out["L"].stride(1), _dev_ptr(out["U"]), out["U"].stride(0),
                     _dev_ptr(out["info"]))
        rid = ctypes.c_int64()
        _check(self.lib.rlu_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)),
               "rlu_server_submit")
        self.live[rid.value] = out
        return rid.value

    def poll(self, rid: int) -> dict:
        st, status = ctypes.c_int32(), ctypes.c_int32()
        t = [ctypes.c_int64() for _ in range(3)]
        _check(self.lib.rlu_server_poll(self.h, rid, ctypes.byref(st), ctypes.byref(status),
                                        *[ctypes.byref(x) for x in t]), "rlu_server_poll")
        return {"state": st.value, "status": status.value, "t_submit": t[0].value,
                "t_start": t[1].value, "t_done": t[2].value}

    def result(self, rid: int) -> dict:
        """The output tensors of a request (valid once poll() reports it done)."""
        return self.live[rid]

    def release(self, rid: int) -> None:
        """Drop this wrapper's references to a finished request's outputs."""
        self.live.pop(rid, None)

    def wait_all(self) -> None:
        _check(self.lib.rlu_server_wait_all(self.h), "rlu_server_wait_all")

    def stats(self) -> dict:
        a = (ctypes.c_int64 * 6)()
        _check(self.lib.rlu_server_stats(self.h, a), "rlu_server_stats")
        return {"submitted": a[0], "done": a[1], "failed": a[2], "peak_arena_bytes": a[3],
                "peak_running": a[4], "bypassed_admissions": a[5]}

    def close(self) -> None:
        if self.h:
            _check(self.lib.rlu_server_destroy(self.h), "rlu_server_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """The batched form of include/rlu_batch.h: one plan for many problems of uneven sizes
    (dicts with A, a row-major FP32 CUDA tensor, and k, l, seed); run() enqueues the whole
    batch (a fixed number of launches), which can be captured in a CUDA graph."""

    def __init__(self, problems: list[dict], prec: int | str = RLU_PREC_F32,
                 options: dict | None = None):
        """options: the kernel choices of include/rlu_batch.h (gemm_tile_y, gemm_tile_c,
        gemm_tile_l, lu_rows_per_cta, umma_ctas_y, umma_ctas_c); missing keys take the
        defaults."""
        self.lib = load_library()
        self.prec = PREC_BY_NAME[prec] if isinstance(prec, str) else int(prec)
        self.options = dict(options or {})
        self.outs = []
        arr = (_Problem * len(problems))()
        for i, p in enumerate(problems):
            A = p["A"]
            m, n = A.shape
            k, l = p["k"], p["l"]
            if A.dtype != torch.float32 or A.stride(1) != 1 or A.device.type != "cuda":
                raise RluError("batched problems take row-major FP32 CUDA tensors")
            o = {"P": torch.empty(m, dtype=torch.int32, device="cuda"),
                 "Q": torch.empty(n, dtype=torch.int32, device="cuda"),
                 "L": _colmajor(m, k, torch.float32),
                 "U": torch.empty((k, n), dtype=torch.float32, device="cuda"),
                 "info": torch.empty(4, dtype=torch.int32, device="cuda")}
            self.outs.append(o)
            arr[i] = _Problem(_dev_ptr(A), m, n, A.stride(0), k, l, p["seed"], _dev_ptr(o["P"]),
                              _dev_ptr(o["Q"]), _dev_ptr(o["L"]), o["L"].stride(1),
                              _dev_ptr(o["U"]), o["U"].stride(0), _dev_ptr(o["info"]))
        self._problems = problems  # keep the inputs alive
        ws = self.lib.rlu_batch_workspace_size(arr, len(problems), self.prec)
        if ws == 0:
            raise RluError("a problem does not fit the batched form (see rlu_batch.h)")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        h = ctypes.c_void_p()
        opt = _BatchOptions(**{k: int(v) for k, v in self.options.items()})
        _check(self.lib.rlu_batch_create(arr, len(problems), self.prec, ctypes.byref(opt),
                                         _dev_ptr(self.workspace), ws, ctypes.byref(h)),
               "rlu_batch_create")
        self.h = h

    def run(self, stream=None) -> None:
        _check(self.lib.rlu_factor_batched(self.h, _stream_ptr(stream)), "rlu_factor_batched")

    def launches(self) -> int:
        return int(self.lib.rlu_batch_launches(self.h))

    def close(self) -> None:
        if self.h:
            _check(self.lib.rlu_batch_destroy(self.h), "rlu_batch_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
