"""GB300-native direct TSQR (Benson, Gleich, Demmel, arXiv:1301.1071).

Thin Python binding over the C-ABI of ``include/tsqr.h`` (libtsqr_gb300.so).
It only marshals arguments: torch provides device memory and the current
stream; every step of the factorisation runs in the library's CUDA kernels.
There is no CPU fallback -- the functions raise if the library or a CUDA
device is unavailable.

    Q, R = direct(A)                 # Sec. III-B direct TSQR (Alg. 2 tree)
    Qh, Rh = direct_host(Ah)         # same, host buffers, copies overlapped
    U, S, V = svd(A)                 # SVD variant, U = Q U_R
    R = r(A)                         # R only (Sec. II-B), A read once
    S, V = svd_values(A)             # singular values / V only (Sec. III-B)
    Q, R = cholqr(A, refine=0)       # Cholesky QR (+ refinement)
    Q, R = indirect_refine(A, 1)     # indirect TSQR + refinement
    dA = backward(Q, R, dQ, dR)      # QR adjoint
    QRFunction.apply(A)              # autograd wrapper
"""
from __future__ import annotations

import ctypes
import functools
import os
import threading

import torch

__all__ = ["direct", "direct_host", "direct_static", "svd", "r", "svd_values", "cholqr", "indirect_refine", "backward", "QRFunction", "TSQRError",
           "workspace_size", "launch_count", "plan_info", "accuracy", "library_path", "load", "STATUS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtsqr_gb300.so")
_lock = threading.Lock()
_lib = None

F64, F32 = 0, 1
PREC = {"native": 0, "df64": 1, "tf32x3": 2, "auto": 3, "ozaki": 4}
OP_DIRECT, OP_SVD, OP_CHOLQR, OP_INDIRECT, OP_BACKWARD, OP_DIRECT_HOST, OP_R, OP_SVD_VALUES, OP_ACCURACY = range(9)
NMAX = 100
STATUS = {0: "TSQR_OK", 1: "TSQR_ERR_ARG", 2: "TSQR_ERR_SHAPE", 3: "TSQR_ERR_ALIGN",
          4: "TSQR_ERR_WORKSPACE", 5: "TSQR_ERR_CUDA", 6: "TSQR_ERR_NOT_SPD", 7: "TSQR_ERR_SINGULAR",
          8: "TSQR_ERR_NONFINITE", 9: "TSQR_ERR_TIMEOUT", 10: "TSQR_ERR_NOCONV"}


class TSQRError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("block_rows", ctypes.c_int64), ("tree_fanout", ctypes.c_int32),
                ("sync", ctypes.c_int32), ("stage_events", ctypes.POINTER(ctypes.c_void_p)),
                ("prec", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("block_rows", ctypes.c_int64), ("blocks", ctypes.c_int64), ("tiles_per_block", ctypes.c_int32),
                ("tree_levels", ctypes.c_int32), ("tree_fanout", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("step3_tensor", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Loads libtsqr_gb300.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(_LIB_PATH)
        P, I64, I32, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
        OP = ctypes.POINTER(Opts)
        sigs = {
            "tsqr_workspace_size": [I32, I64, I64, I32, OP, ctypes.POINTER(SZ)],
            "tsqr_direct": [P, I64, I64, I64, I32, P, I64, P, I64, P, SZ, OP, P],
            "tsqr_direct_static": [P, I64, I64, I64, I32, P, I64, P, I64, OP, P],
            "tsqr_direct_host": [P, I64, I64, I32, P, P, P, P, SZ, OP, P, P],
            "tsqr_svd": [P, I64, I64, I64, I32, P, I64, P, P, I64, P, SZ, OP, P],
            "tsqr_r": [P, I64, I64, I64, I32, P, I64, P, SZ, OP, P],
            "tsqr_svd_values": [P, I64, I64, I64, I32, P, P, I64, P, SZ, OP, P],
            "cholqr": [P, I64, I64, I64, I32, P, I64, P, I64, I32, P, SZ, OP, P],
            "tsqr_indirect_refine": [P, I64, I64, I64, I32, P, I64, P, I64, I32, P, SZ, OP, P],
            "tsqr_backward": [P, P, P, P, I64, I64, I32, P, P, SZ, OP, P],
            "tsqr_read_status": [P, P],
            "tsqr_launch_count": [I32, I64, I64, I32, OP, I32, ctypes.POINTER(I32)],
            "tsqr_plan_query": [I32, I64, I64, I32, OP, ctypes.POINTER(PlanInfo)],
            "tsqr_accuracy": [P, P, P, I64, I64, I32, P, P, SZ, P],
        }
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.tsqr_status_string.argtypes = [I32]
        lib.tsqr_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype} (float64 or float32)")


def _on_device(fn):
    """Runs `fn` with the device of its first (tensor) argument current: the
    library resolves the workspace, the static scratch and its launches
    against the current device, and the stream passed is that device's."""
    @functools.wraps(fn)
    def wrapped(A, *args, **kw):
        if isinstance(A, torch.Tensor) and A.is_cuda:
            with torch.cuda.device(A.device):
                return fn(A, *args, **kw)
        return fn(A, *args, **kw)
    return wrapped


def _check_tall(A: torch.Tensor):
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor (there is no CPU path)")
    if A.dim() != 2:
        raise ValueError("A must be 2-D")
    m, n = A.shape
    if n < 1 or n > NMAX or m < n:
        raise ValueError(f"unsupported shape {tuple(A.shape)}: need 1 <= n <= {NMAX} and m >= n")
    return m, n


def _check_buf(t, shape, dtype, device, name):
    """Raises unless ``t`` is a contiguous tensor of exactly ``shape`` and
    ``dtype`` on ``device``: the library reads or writes the whole shape
    through its pointer and can check neither its size nor its device."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
        raise ValueError(f"{name} must be {tuple(shape)} {dtype}, got {tuple(t.shape)} {t.dtype}")
    if t.device != torch.device(device):
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def _opts(block_rows=0, fanout=0, sync=False, events=None, prec="native") -> Opts:
    o = Opts()
    o.block_rows = int(block_rows)
    o.tree_fanout = int(fanout)
    o.sync = 1 if sync else 0
    o.prec = PREC[prec]
    if events is not None:
        if any(not e.cuda_event for e in events):
            raise ValueError("stage events must have been recorded once (torch creates them lazily)")
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in events])
        o._events_keepalive = arr
        o.stage_events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
    return o


def launch_count(op: int, m: int, n: int, dtype: torch.dtype, block_rows=0, fanout=0, refine=0,
                 prec="native") -> int:
    """Kernel launches of one call (host-only query)."""
    lib = load()
    code = F64 if dtype == torch.float64 else F32
    out = ctypes.c_int32(0)
    o = _opts(block_rows, fanout, prec=prec)
    _raise(lib.tsqr_launch_count(op, m, n, code, ctypes.byref(o), int(refine), ctypes.byref(out)),
           "tsqr_launch_count")
    return int(out.value)


def plan_info(op: int, m: int, n: int, dtype: torch.dtype, block_rows=0, fanout=0, prec="native") -> dict:
    """The row-block partition and Step-2 tree a call would use (host-only
    query): block_rows, blocks, tiles_per_block, tree_levels, tree_fanout,
    the resolved precision and whether Step 3 runs on the tensor cores."""
    lib = load()
    code = F64 if dtype == torch.float64 else F32
    info = PlanInfo()
    o = _opts(block_rows, fanout, prec=prec)
    _raise(lib.tsqr_plan_query(op, m, n, code, ctypes.byref(o), ctypes.byref(info)), "tsqr_plan_query")
    names = {v: k for k, v in PREC.items()}
    return {"block_rows": int(info.block_rows), "blocks": int(info.blocks),
            "tiles_per_block": int(info.tiles_per_block), "tree_levels": int(info.tree_levels),
            "tree_fanout": int(info.tree_fanout), "prec": names.get(int(info.prec), int(info.prec)),
            "step3_tensor": bool(info.step3_tensor)}


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _raise(st: int, what: str):
    if st != 0:
        raise TSQRError(st, what)


def workspace_size(op: int, m: int, n: int, dtype: torch.dtype, block_rows=0, fanout=0, prec="native") -> int:
    lib = load()
    code = F64 if dtype == torch.float64 else F32
    out = ctypes.c_size_t(0)
    o = _opts(block_rows, fanout, prec=prec)
    _raise(lib.tsqr_workspace_size(op, m, n, code, ctypes.byref(o), ctypes.byref(out)), "tsqr_workspace_size")
    return int(out.value)


def _workspace(op, m, n, dtype, device, block_rows, fanout, work, prec="native"):
    """The caller's workspace when it is a contiguous buffer on ``device`` of
    at least the bytes the call needs, else a new one."""
    need = workspace_size(op, m, n, dtype, block_rows, fanout, prec)
    if work is not None and (work.device != torch.device(device) or not work.is_contiguous()):
        raise ValueError(f"work must be a contiguous buffer on {device}, got {work.device}")
    if work is None or _nbytes(work) < need:
        work = torch.empty(need, dtype=torch.uint8, device=device)
    return work


def _status(work: torch.Tensor, what: str, check: bool):
    if check:
        st = load().tsqr_read_status(_ptr(work), _stream(work.device))
        _raise(st, what)


@_on_device
def direct(A: torch.Tensor, block_rows: int = 0, fanout: int = 0, work: torch.Tensor | None = None,
           out: tuple | None = None, check: bool = True, stage_events=None, prec: str = "native"):
    """Direct TSQR: returns (Q, R), Q m x n in A's dtype, R n x n float64,
    diag(R) >= 0.  ``check`` synchronises and raises on a device error.
    ``stage_events``: 4 torch.cuda.Event recorded at the start and after
    Steps 1, 2 and 3.  ``prec``: "native" or "df64" (FP64 data only)."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    if out is not None:
        Q = _check_buf(out[0], (m, n), A.dtype, A.device, "out[0] (Q)")
        R = _check_buf(out[1], (n, n), torch.float64, A.device, "out[1] (R)")
    else:
        Q, R = torch.empty_like(A), torch.empty(n, n, dtype=torch.float64, device=A.device)
    work = _workspace(OP_DIRECT, m, n, A.dtype, A.device, block_rows, fanout, work, prec)
    o = _opts(block_rows, fanout, events=stage_events, prec=prec)
    st = lib.tsqr_direct(_ptr(A), m, n, n, _dtype_code(A), _ptr(Q), n, _ptr(R), n, _ptr(work), _nbytes(work),
                         ctypes.byref(o), _stream(A.device))
    _raise(st, "tsqr_direct")
    _status(work, "tsqr_direct", check)
    return Q, R


def direct_host(A: torch.Tensor, block_rows: int = 0, fanout: int = 0, out: tuple | None = None,
                dbuf: torch.Tensor | None = None, work: torch.Tensor | None = None,
                copy_stream: torch.cuda.Stream | None = None, device=None, check: bool = True,
                prec: str = "native"):
    """Direct TSQR of a HOST matrix A (CPU tensor, m x n, float64/float32;
    page-locked for the copies to overlap the kernels): returns (Q, R) on the
    host.  The rows go to the device in chunks on ``copy_stream`` while Step 1
    runs on the current stream, and Q comes back chunk by chunk behind Step 3
    (tsqr_direct_host).  ``dbuf`` (device, m x n) and ``work`` may be given
    to avoid allocations; ``out`` = (Q, R) host tensors (pinned for overlap).
    The current stream holds the whole call when it returns."""
    if A.is_cuda or A.dim() != 2:
        raise ValueError("A must be a 2-D host (CPU) tensor")
    m, n = A.shape
    if n < 1 or n > NMAX or m < n:
        raise ValueError(f"unsupported shape {tuple(A.shape)}: need 1 <= n <= {NMAX} and m >= n")
    A = A.contiguous()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if dev.type != "cuda":
        raise ValueError(f"device must be a CUDA device, got {dev}")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        return _direct_host(A, m, n, dev, block_rows, fanout, out, dbuf, work, copy_stream, check, prec)


def _direct_host(A, m, n, dev, block_rows, fanout, out, dbuf, work, copy_stream, check, prec):
    lib = load()
    if out is not None:
        Q = _check_buf(out[0], (m, n), A.dtype, "cpu", "out[0] (Q)")
        R = _check_buf(out[1], (n, n), torch.float64, "cpu", "out[1] (R)")
    else:
        Q = torch.empty(m, n, dtype=A.dtype, pin_memory=True)
        R = torch.empty(n, n, dtype=torch.float64, pin_memory=True)
    if dbuf is None:
        dbuf = torch.empty(m, n, dtype=A.dtype, device=dev)
    else:
        _check_buf(dbuf, (m, n), A.dtype, dev, "dbuf")
    work = _workspace(OP_DIRECT_HOST, m, n, A.dtype, dev, block_rows, fanout, work, prec)
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=dev)
    o = _opts(block_rows, fanout, prec=prec)
    st = lib.tsqr_direct_host(_ptr(A), m, n, _dtype_code(A), _ptr(Q), _ptr(R), _ptr(dbuf), _ptr(work),
                              _nbytes(work), ctypes.byref(o), _stream(dev), ctypes.c_void_p(cs.cuda_stream))
    _raise(st, "tsqr_direct_host")
    _status(work, "tsqr_direct_host", check)
    return Q, R


@_on_device
def direct_static(A: torch.Tensor, block_rows: int = 0, fanout: int = 0, prec: str = "native"):
    """Direct TSQR on the library's fixed device scratch (no workspace is
    allocated for the call; problems needing more than 16 MiB of workspace
    are rejected).  Returns (Q, R); synchronises to report device errors."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    Q = torch.empty_like(A)
    R = torch.empty(n, n, dtype=torch.float64, device=A.device)
    o = _opts(block_rows, fanout, sync=True, prec=prec)
    st = lib.tsqr_direct_static(_ptr(A), m, n, n, _dtype_code(A), _ptr(Q), n, _ptr(R), n, ctypes.byref(o),
                                _stream(A.device))
    _raise(st, "tsqr_direct_static")
    return Q, R


@_on_device
def svd(A: torch.Tensor, block_rows: int = 0, fanout: int = 0, work: torch.Tensor | None = None,
        check: bool = True, prec: str = "native"):
    """SVD via direct TSQR: A = U diag(S) V^T (U m x n in A's dtype; S, V float64)."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    U = torch.empty_like(A)
    S = torch.empty(n, dtype=torch.float64, device=A.device)
    V = torch.empty(n, n, dtype=torch.float64, device=A.device)
    work = _workspace(OP_SVD, m, n, A.dtype, A.device, block_rows, fanout, work, prec)
    o = _opts(block_rows, fanout, prec=prec)
    st = lib.tsqr_svd(_ptr(A), m, n, n, _dtype_code(A), _ptr(U), n, _ptr(S), _ptr(V), n, _ptr(work),
                      _nbytes(work), ctypes.byref(o), _stream(A.device))
    _raise(st, "tsqr_svd")
    _status(work, "tsqr_svd", check)
    return U, S, V


@_on_device
def r(A: torch.Tensor, block_rows: int = 0, fanout: int = 0, work: torch.Tensor | None = None,
      check: bool = True, prec: str = "native"):
    """R factor only (Steps 1-2, no Q): returns R, n x n float64, diag(R) >= 0."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    R = torch.empty(n, n, dtype=torch.float64, device=A.device)
    work = _workspace(OP_R, m, n, A.dtype, A.device, block_rows, fanout, work, prec)
    o = _opts(block_rows, fanout, prec=prec)
    st = lib.tsqr_r(_ptr(A), m, n, n, _dtype_code(A), _ptr(R), n, _ptr(work), _nbytes(work), ctypes.byref(o),
                    _stream(A.device))
    _raise(st, "tsqr_r")
    _status(work, "tsqr_r", check)
    return R


@_on_device
def svd_values(A: torch.Tensor, want_v: bool = True, block_rows: int = 0, fanout: int = 0,
               work: torch.Tensor | None = None, check: bool = True, prec: str = "native"):
    """Singular values (descending, float64) and, if ``want_v``, V (n x n
    float64) without forming U: returns (S, V) (V is None when not wanted)."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    S = torch.empty(n, dtype=torch.float64, device=A.device)
    V = torch.empty(n, n, dtype=torch.float64, device=A.device) if want_v else None
    work = _workspace(OP_SVD_VALUES, m, n, A.dtype, A.device, block_rows, fanout, work, prec)
    o = _opts(block_rows, fanout, prec=prec)
    st = lib.tsqr_svd_values(_ptr(A), m, n, n, _dtype_code(A), _ptr(S), _ptr(V), n, _ptr(work), _nbytes(work),
                             ctypes.byref(o), _stream(A.device))
    _raise(st, "tsqr_svd_values")
    _status(work, "tsqr_svd_values", check)
    return S, V


@_on_device
def cholqr(A: torch.Tensor, refine: int = 0, work: torch.Tensor | None = None, check: bool = True):
    """Cholesky QR (+ `refine` refinement passes): returns (Q, R)."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    Q = torch.empty_like(A)
    R = torch.empty(n, n, dtype=torch.float64, device=A.device)
    work = _workspace(OP_CHOLQR, m, n, A.dtype, A.device, 0, 0, work)
    o = _opts()
    st = lib.cholqr(_ptr(A), m, n, n, _dtype_code(A), _ptr(Q), n, _ptr(R), n, int(refine), _ptr(work),
                    _nbytes(work), ctypes.byref(o), _stream(A.device))
    _raise(st, "cholqr")
    _status(work, "cholqr", check)
    return Q, R


@_on_device
def indirect_refine(A: torch.Tensor, refine: int = 1, block_rows: int = 0, fanout: int = 0,
                    work: torch.Tensor | None = None, check: bool = True):
    """Indirect TSQR + `refine` refinement passes: returns (Q, R)."""
    m, n = _check_tall(A)
    A = A.contiguous()
    lib = load()
    Q = torch.empty_like(A)
    R = torch.empty(n, n, dtype=torch.float64, device=A.device)
    work = _workspace(OP_INDIRECT, m, n, A.dtype, A.device, block_rows, fanout, work)
    o = _opts(block_rows, fanout)
    st = lib.tsqr_indirect_refine(_ptr(A), m, n, n, _dtype_code(A), _ptr(Q), n, _ptr(R), n, int(refine),
                                  _ptr(work), _nbytes(work), ctypes.byref(o), _stream(A.device))
    _raise(st, "tsqr_indirect_refine")
    _status(work, "tsqr_indirect_refine", check)
    return Q, R


@_on_device
def backward(Q: torch.Tensor, R: torch.Tensor, dQ: torch.Tensor | None, dR: torch.Tensor | None,
             work: torch.Tensor | None = None, check: bool = True):
    """QR adjoint: dA = (dQ + Q copyltu(M)) R^{-T}, M = R dR^T - dQ^T Q."""
    m, n = _check_tall(Q)
    Q = Q.contiguous()
    R = _check_buf(R.to(torch.float64).contiguous(), (n, n), torch.float64, Q.device, "R")
    dQ = None if dQ is None else _check_buf(dQ.to(Q.dtype).contiguous(), (m, n), Q.dtype, Q.device, "dQ")
    dR = None if dR is None else _check_buf(dR.to(torch.float64).contiguous(), (n, n), torch.float64, Q.device, "dR")
    lib = load()
    dA = torch.empty_like(Q)
    work = _workspace(OP_BACKWARD, m, n, Q.dtype, Q.device, 0, 0, work)
    o = _opts()
    st = lib.tsqr_backward(_ptr(Q), _ptr(R), _ptr(dQ), _ptr(dR), m, n, _dtype_code(Q), _ptr(dA), _ptr(work),
                           _nbytes(work), ctypes.byref(o), _stream(Q.device))
    _raise(st, "tsqr_backward")
    _status(work, "tsqr_backward", check)
    return dA


@_on_device
def accuracy(Q: torch.Tensor, R: torch.Tensor | None = None, A: torch.Tensor | None = None,
             work: torch.Tensor | None = None) -> dict:
    """Accuracy metrics of a factorisation (Sec. I-B) from tsqr_accuracy's
    compensated device sums: ``orth_2`` = ||Q^T Q - I||_2, ``orth_F``, and with
    A and R ``res_F`` = ||A - QR||_F/||A||_F and ``res_2`` = ||A - QR||_2/||R||_2.
    The 2-norms of the symmetric n x n results are taken on the host."""
    import numpy as np
    if not Q.is_cuda or Q.dim() != 2:
        raise ValueError("Q must be a 2-D CUDA tensor (there is no CPU path)")
    m, n = Q.shape
    if (A is None) != (R is None):
        raise ValueError("give both A and R, or neither")
    Q = Q.contiguous()
    _dtype_code(Q)
    if A is not None:
        A = _check_buf(A.to(Q.dtype).contiguous(), (m, n), Q.dtype, Q.device, "A")
        R = _check_buf(R.to(torch.float64).contiguous(), (n, n), torch.float64, Q.device, "R")
    lib = load()
    out = torch.empty(3 * n * n + 2, dtype=torch.float64, device=Q.device)
    need = workspace_size(OP_ACCURACY, m, n, Q.dtype)
    if work is not None and (work.device != Q.device or not work.is_contiguous()):
        raise ValueError(f"work must be a contiguous buffer on {Q.device}, got {work.device}")
    if work is None or _nbytes(work) < need:
        work = torch.empty(need, dtype=torch.uint8, device=Q.device)
    st = lib.tsqr_accuracy(_ptr(A), _ptr(Q), _ptr(R), m, n, _dtype_code(Q), _ptr(out), _ptr(work), _nbytes(work),
                           _stream(Q.device))
    _raise(st, "tsqr_accuracy")
    _status(work, "tsqr_accuracy", True)
    o = out.cpu().numpy()
    nn = n * n
    E = o[:nn].reshape(n, n) + o[nn:2 * nn].reshape(n, n)
    res = {"orth_2": float(np.max(np.abs(np.linalg.eigvalsh(E)))), "orth_F": float(np.linalg.norm(E))}
    if A is not None:
        F = o[2 * nn:3 * nn].reshape(n, n)
        r2 = float(np.linalg.norm(R.cpu().numpy(), 2))
        res["res_F"] = float(np.sqrt(o[3 * nn] / o[3 * nn + 1])) if o[3 * nn + 1] > 0 else float(np.sqrt(o[3 * nn]))
        res["res_2"] = float(np.sqrt(max(np.max(np.linalg.eigvalsh(F)), 0.0)) / r2) if r2 > 0 else float("nan")
    return res


class QRFunction(torch.autograd.Function):
    """Thin QR with the hand-written adjoint: forward = direct TSQR, backward =
    tsqr_backward on the saved Q and R.  R is returned in A's dtype."""

    @staticmethod
    def forward(ctx, A):
        Q, R = direct(A)
        ctx.save_for_backward(Q, R)
        return Q, R.to(A.dtype)

    @staticmethod
    def backward(ctx, gQ, gR):
        Q, R = ctx.saved_tensors
        dR = None if gR is None else torch.triu(gR.to(torch.float64))
        return backward(Q, R, gQ, dR)
