"""Python binding of libcsk (include/csk.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks tensor placement, allocates outputs and
the workspace with PyTorch on the tensors' device, passes raw pointers and the
current CUDA stream, and raises :class:`CskError` on a non-zero return code.
There is no fallback: if ``libcsk.so`` is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcsk.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "csk.h")

CSK_OK, CSK_MAXITER, CSK_INPROGRESS = 0, 1, 2
CSK_EINVAL, CSK_ENOMEM, CSK_ETIMEOUT, CSK_ENUMERIC, CSK_ECUDA, CSK_EUNSUPPORTED = -1, -2, -3, -4, -5, -6
CSK_F32, CSK_F64 = 0, 1
GEMV, GRAM, AUTO, UPDATE = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class CskError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lib().csk_strerror(code).decode()} ({code})")


class csk_params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("seed", ctypes.c_uint64), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int64), ("refresh_every", ctypes.c_int32),
                ("path", ctypes.c_int32), ("spin_limit", ctypes.c_int64),
                ("ik_log", ctypes.c_void_p), ("ik_log_len", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("fault_inject", ctypes.c_int32),
                ("x_log", ctypes.c_void_p), ("x_log_len", ctypes.c_int64),
                ("threads", ctypes.c_int32), ("gemv_variant", ctypes.c_int32),
                ("stage_events", ctypes.c_void_p * 5), ("log_system", ctypes.c_int32),
                ("log_rhs", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class csk_system(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("nrhs", ctypes.c_int32), ("reserved_", ctypes.c_int32), ("d", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("X0", ctypes.c_void_p), ("Xstar", ctypes.c_void_p),
                ("Xout", ctypes.c_void_p), ("info", ctypes.c_void_p), ("area", ctypes.c_void_p)]


INFO_DTYPE = np.dtype([("status", "<i4"), ("path", "<i4"), ("iters", "<i8"), ("rse", "<f8"),
                       ("resid", "<f8"), ("rows", "<i4"), ("empty_rows", "<i4"), ("grid", "<i4"),
                       ("reserved0", "<i4"), ("reserved1", "<f8"), ("reserved2", "<f8")])
assert INFO_DTYPE.itemsize == 64


class csk_host_problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("b", ctypes.c_void_p), ("x0", ctypes.c_void_p),
                ("x_star", ctypes.c_void_p), ("x_out", ctypes.c_void_p), ("info", ctypes.c_void_p)]


class csk_synth_system(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nrhs", ctypes.c_int32),
                ("reserved_", ctypes.c_int32), ("seed", ctypes.c_uint64), ("A", ctypes.c_void_p),
                ("X", ctypes.c_void_p), ("B", ctypes.c_void_p)]


def lib():
    """Load libcsk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcsk.so not found at {LIB_PATH}: build it with "
                               "paper_2004_02480_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u64, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                ctypes.c_size_t)
        L.csk_params_default.argtypes = [ctypes.POINTER(csk_params)]
        L.csk_strerror.argtypes = [ctypes.c_int]
        L.csk_strerror.restype = ctypes.c_char_p
        L.csk_version.restype = ctypes.c_int
        L.csk_sketch_workspace_size.argtypes = [i64, i64]
        L.csk_sketch_workspace_size.restype = sz
        L.csk_sketch.argtypes = [P, i64, i64, i64, P, i64, i32, i32, i64, u64, P, P, P, P, P, P,
                                 sz, P]
        L.csk_sketch.restype = ctypes.c_int
        L.csk_solve_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(csk_params)]
        L.csk_solve_workspace_size.restype = sz
        L.csk_solve.argtypes = [P, i64, i64, i64, P, i32, ctypes.POINTER(csk_params), P, P, P, P,
                                P, sz, P]
        L.csk_solve.restype = ctypes.c_int
        L.csk_kernel_launches.restype = ctypes.c_int64
        L.csk_solve_batched_workspace_size.argtypes = [ctypes.POINTER(csk_system), i32]
        L.csk_solve_batched_workspace_size.restype = sz
        L.csk_solve_batched.argtypes = [ctypes.POINTER(csk_system), i32,
                                        ctypes.POINTER(csk_params), P, sz, P]
        L.csk_solve_batched.restype = ctypes.c_int
        L.csk_gram_workspace_size.argtypes = [i64, i64]
        L.csk_gram_workspace_size.restype = sz
        L.csk_gram.argtypes = [P, i64, i64, P, P, i64, P, P, sz, P]
        L.csk_gram.restype = ctypes.c_int
        L.csk_sketch_noalloc.argtypes = [P, i64, i64, i64, P, i64, i32, i32, i64, u64, P, P, P,
                                         P, P, P]
        L.csk_sketch_noalloc.restype = ctypes.c_int
        L.csk_solve_host_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(csk_params)]
        L.csk_solve_host_workspace_size.restype = sz
        L.csk_solve_host.argtypes = [P, i64, i64, i64, P, i32, ctypes.POINTER(csk_params), P, P,
                                     P, P, P, sz, P]
        L.csk_solve_host.restype = ctypes.c_int
        L.csk_solve_host_many_workspace_size.argtypes = [ctypes.POINTER(csk_host_problem), i32, i32,
                                                         ctypes.POINTER(csk_params)]
        L.csk_solve_host_many_workspace_size.restype = sz
        L.csk_solve_host_many.argtypes = [ctypes.POINTER(csk_host_problem), i32, i32,
                                          ctypes.POINTER(csk_params), P, sz, P]
        L.csk_solve_host_many.restype = ctypes.c_int
        L.csk_synth_systems.argtypes = [ctypes.POINTER(csk_synth_system), i32, P]
        L.csk_synth_systems.restype = ctypes.c_int
        L.csk_batched_area_size.argtypes = [i64, i64, i32]
        L.csk_batched_area_size.restype = sz
        for f in ("csk_batched_prepare_workspace_size", "csk_batched_iterate_workspace_size"):
            getattr(L, f).argtypes = [ctypes.POINTER(csk_system), i32]
            getattr(L, f).restype = sz
        L.csk_batched_prepare.argtypes = [ctypes.POINTER(csk_system), i32, P, sz, P]
        L.csk_batched_prepare.restype = ctypes.c_int
        L.csk_batched_iterate.argtypes = [ctypes.POINTER(csk_system), i32, ctypes.POINTER(csk_params),
                                          i64, P, sz, P]
        L.csk_batched_iterate.restype = ctypes.c_int
        L.csk_solve_batched_set_plan.argtypes = [ctypes.POINTER(csk_system), i32, i32, i32]
        L.csk_solve_batched_set_plan.restype = ctypes.c_int
        L.csk_solve_batched_signature.argtypes = [ctypes.POINTER(csk_system), i32]
        L.csk_solve_batched_signature.restype = ctypes.c_uint64
        L.csk_info_sync.argtypes = [P, P, P]
        L.csk_info_sync.restype = ctypes.c_int
        L.csk_workspace_size.argtypes = [i64, i64, i64, i32, i32, i32]
        L.csk_workspace_size.restype = sz
        L.csk_exchange_floor_workspace_size.argtypes = [i32]
        L.csk_exchange_floor_workspace_size.restype = sz
        L.csk_exchange_floor.argtypes = [i32, i64, P, sz, P]
        L.csk_exchange_floor.restype = ctypes.c_int
        _lib = L
        return L


def header_functions() -> list[str]:
    """Names of the functions include/csk.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(csk_[a-z0-9_]+)\s*\(", txt)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return CSK_F32
    if t.dtype == torch.float64:
        return CSK_F64
    raise TypeError(f"unsupported dtype {t.dtype}: float32 or float64")


def _check_cuda(*ts):
    dev = None
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError("tensors on different devices")
    return dev


def _rowmajor(A: torch.Tensor) -> int:
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major tensor (unit column stride)")
    return A.stride(0)


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _workspace(nbytes: int, dev) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


def csk_params_default(**kw) -> csk_params:
    """Section 3 defaults (tol 1e-6, 20000 steps), overridden by keywords."""
    p = csk_params()
    lib().csk_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def csk_kernel_launches() -> int:
    """Kernels the library has enqueued in this process so far."""
    return int(lib().csk_kernel_launches())


def set_stage_events(params: csk_params, events) -> None:
    """Attach up to five torch.cuda.Event objects (None to skip) as the
    stage markers of csk_solve.  Each event is recorded once here so that its
    CUDA handle exists."""
    for i in range(5):
        ev = events[i] if i < len(events) else None
        if ev is None:
            params.stage_events[i] = None
            continue
        ev.record()
        params.stage_events[i] = ctypes.c_void_p(int(ev.cuda_event))


def csk_sketch_workspace_size(m: int, d: int) -> int:
    return int(lib().csk_sketch_workspace_size(m, d))


@dataclass
class Sketch:
    At: torch.Tensor
    bt: torch.Tensor | None
    norms2: torch.Tensor | None
    perm: torch.Tensor | None
    off: torch.Tensor | None


def csk_sketch(A: torch.Tensor, d: int, seed: int, b: torch.Tensor | None = None, *,
               norms: bool = True, perm: bool = False, off: bool = False,
               ws: torch.Tensor | None = None) -> Sketch:
    """At = S A and bt = S b (Algorithm 1, Initialize) on A's device."""
    dev = _check_cuda(A, b, ws)
    lda = _rowmajor(A)
    m, n = A.shape
    dt = _dtype_code(A)
    nrhs, ldb, B = 0, 0, None
    if b is not None:
        if b.dtype != A.dtype:
            raise TypeError("b must have A's dtype")
        B = b.reshape(m, -1)
        if B.stride(1) != 1:
            raise ValueError("b must be contiguous along right-hand sides")
        nrhs, ldb = B.shape[1], B.stride(0)
    At = torch.empty((d, n), dtype=A.dtype, device=dev)
    bt = torch.empty((d, nrhs), dtype=A.dtype, device=dev) if nrhs else None
    N2 = torch.empty(d, dtype=torch.float64, device=dev) if norms else None
    P = torch.empty(m, dtype=torch.int32, device=dev) if perm else None
    O = torch.empty(d + 1, dtype=torch.int32, device=dev) if off else None
    need = csk_sketch_workspace_size(m, d)
    if ws is None:
        ws = _workspace(need, dev)
    rc = lib().csk_sketch(_ptr(A), m, n, lda, _ptr(B), ldb, nrhs, dt, d, seed & (2**64 - 1),
                          _ptr(At), _ptr(bt), _ptr(N2), _ptr(P), _ptr(O), _ptr(ws), ws.numel(),
                          _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_sketch")
    if bt is not None and b.dim() == 1:
        bt = bt[:, 0]
    return Sketch(At, bt, N2, P, O)


def csk_gram(At: torch.Tensor, norms2: torch.Tensor | None = None, *, ldg: int | None = None,
             info: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """G = At At^T in split BF16 on the tensor cores (d x d FP32; the
    returned tensor is a d x d view of a d x ldg buffer)."""
    dev = _check_cuda(At, norms2, info, ws)
    if At.dtype != torch.float32 or not At.is_contiguous():
        raise TypeError("At must be contiguous float32")
    d, n = At.shape
    if norms2 is not None and (norms2.dtype != torch.float64 or norms2.numel() != d):
        raise TypeError("norms2 must be d float64 values")
    ldg = ldg or (d + 31) // 32 * 32
    G = torch.empty((d, ldg), dtype=torch.float32, device=dev)
    if ws is None:
        ws = _workspace(int(lib().csk_gram_workspace_size(d, n)), dev)
    rc = lib().csk_gram(_ptr(At), d, n, _ptr(norms2), _ptr(G), ldg, _ptr(info), _ptr(ws),
                        ws.numel(), _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_gram")
    return G[:, :d]


def csk_solve_workspace_size(m: int, n: int, dtype: int, params: csk_params) -> int:
    return int(lib().csk_solve_workspace_size(m, n, dtype, ctypes.byref(params)))


def read_info(info: torch.Tensor) -> dict:
    """Decode a csk_info record (64 bytes of device memory) on the host."""
    rec = np.frombuffer(info.cpu().numpy().tobytes(), dtype=INFO_DTYPE)[0]
    return {k: rec[k].item() for k in INFO_DTYPE.names if not k.startswith("reserved")}


def csk_info_sync(info: torch.Tensor) -> dict:
    """Copy a device csk_info record to the host through csk_info_sync (after
    the work queued on the current stream) and decode it."""
    dev = _check_cuda(info)
    host = np.zeros(1, INFO_DTYPE)
    rc = lib().csk_info_sync(_ptr(info), ctypes.c_void_p(host.ctypes.data), _stream(dev))
    if rc in (CSK_EINVAL, CSK_ECUDA):          # the call failed (no solve ends so)
        raise CskError(rc, "csk_info_sync")
    return info_dict(host)


def csk_workspace_size(m: int, n: int, d: int, nrhs: int, dtype: int, resid: int) -> int:
    """Bytes of one workspace that serves csk_sketch, csk_solve and (FP32)
    csk_solve_batched on a problem of this shape."""
    return int(lib().csk_workspace_size(m, n, d, nrhs, dtype, resid))


def csk_exchange_floor(grid: int, rounds: int, device=None, ws: torch.Tensor | None = None) -> None:
    """Enqueue the exchange-only loop (``rounds`` rounds on ``grid`` CTAs) on
    the current stream; time it with events around the call."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    need = int(lib().csk_exchange_floor_workspace_size(grid))
    if need == 0:
        raise CskError(CSK_EINVAL, "csk_exchange_floor_workspace_size")
    if ws is None:
        ws = _workspace(need, dev)
    rc = lib().csk_exchange_floor(grid, rounds, _ptr(ws), ws.numel(), _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_exchange_floor")


def csk_solve(A: torch.Tensor, b: torch.Tensor, params: csk_params, x0=None, x_star=None, *,
              x_out: torch.Tensor | None = None, info: torch.Tensor | None = None,
              ws: torch.Tensor | None = None, sync: bool = True):
    """Algorithm 1 end to end; returns (x, info dict or the device info tensor)."""
    dev = _check_cuda(A, b, x0, x_star, x_out, info, ws)
    lda = _rowmajor(A)
    m, n = A.shape
    dt = _dtype_code(A)
    for t in (b, x0, x_star):
        if t is not None and (t.dtype != A.dtype or not t.is_contiguous()):
            raise TypeError("b, x0, x_star must be contiguous with A's dtype")
    if x_out is None:
        x_out = torch.empty(n, dtype=A.dtype, device=dev)
    if info is None:
        info = torch.empty(64, dtype=torch.uint8, device=dev)
    need = csk_solve_workspace_size(m, n, dt, params)
    if need == 0:
        raise CskError(CSK_EINVAL, "csk_solve_workspace_size")
    if ws is None:
        ws = _workspace(need, dev)
    rc = lib().csk_solve(_ptr(A), m, n, lda, _ptr(b), dt, ctypes.byref(params), _ptr(x0),
                         _ptr(x_star), _ptr(x_out), _ptr(info), _ptr(ws), ws.numel(),
                         _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_solve")
    if not sync:
        return x_out, info
    return x_out, read_info(info)


def csk_solve_host_workspace_size(m: int, n: int, dtype: int, params: csk_params) -> int:
    return int(lib().csk_solve_host_workspace_size(m, n, dtype, ctypes.byref(params)))


def csk_solve_host(A: np.ndarray, b: np.ndarray, params: csk_params, x0=None, x_star=None, *,
                   ws: torch.Tensor, x_out: np.ndarray | None = None,
                   device=None) -> tuple[np.ndarray, dict, int]:
    """csk_solve with host (numpy, ideally page-locked) inputs and outputs.

    ``ws`` is a device uint8 tensor of csk_solve_host_workspace_size bytes.
    Returns (x, info dict, status code of the solve).
    """
    if A.ndim != 2 or A.strides[1] != A.itemsize:
        raise ValueError("A must be 2-D row-major")
    m, n = A.shape
    dt = CSK_F32 if A.dtype == np.float32 else CSK_F64 if A.dtype == np.float64 else None
    if dt is None:
        raise TypeError("A must be float32 or float64")
    for t in (b, x0, x_star):
        if t is not None and (t.dtype != A.dtype or not t.flags.c_contiguous):
            raise TypeError("b, x0, x_star must be contiguous with A's dtype")
    if x_out is None:
        x_out = np.empty(n, A.dtype)
    info = np.zeros(1, INFO_DTYPE)
    dev = ws.device if device is None else device

    def hp(a):
        return None if a is None else ctypes.c_void_p(a.ctypes.data)

    rc = lib().csk_solve_host(hp(A), m, n, A.strides[0] // A.itemsize, hp(b), dt,
                              ctypes.byref(params), hp(x0), hp(x_star), hp(x_out), hp(info),
                              _ptr(ws), ws.numel(), _stream(dev))
    if rc < 0 and rc != info["status"][0]:
        raise CskError(rc, "csk_solve_host")
    rec = info[0]
    return x_out, {k: rec[k].item() for k in INFO_DTYPE.names if not k.startswith("reserved")}, rc


@dataclass
class HostProblem:
    """One problem of csk_solve_host_many (host numpy arrays, ideally
    page-locked).  x_out / info are filled by the call."""
    A: np.ndarray
    b: np.ndarray
    x0: np.ndarray | None = None
    x_star: np.ndarray | None = None
    x_out: np.ndarray | None = None
    info: np.ndarray | None = None


def _host_problems(probs: list[HostProblem]):
    dt = None
    arr = (csk_host_problem * max(1, len(probs)))()
    for i, q in enumerate(probs):
        A = q.A
        if A.ndim != 2 or A.strides[1] != A.itemsize:
            raise ValueError("A must be 2-D row-major")
        t = CSK_F32 if A.dtype == np.float32 else CSK_F64 if A.dtype == np.float64 else None
        if t is None or (dt is not None and t != dt):
            raise TypeError("every A must be float32, or every A float64")
        dt = t
        for v in (q.b, q.x0, q.x_star):
            if v is not None and (v.dtype != A.dtype or not v.flags.c_contiguous):
                raise TypeError("b, x0, x_star must be contiguous with A's dtype")
        m, n = A.shape
        if q.x_out is None:                          # page-locked, so results copy back
            q.x_out = torch.empty(n, dtype=torch.float32 if t == CSK_F32 else torch.float64
                                  ).pin_memory().numpy()
        if q.info is None:
            q.info = torch.zeros(INFO_DTYPE.itemsize, dtype=torch.uint8).pin_memory().numpy(
            ).view(INFO_DTYPE)
        hp = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        arr[i] = csk_host_problem(hp(A), m, n, A.strides[0] // A.itemsize, hp(q.b), hp(q.x0),
                                  hp(q.x_star), hp(q.x_out), hp(q.info))
    return arr, (dt if dt is not None else CSK_F32)


def csk_solve_host_many_workspace_size(probs: list[HostProblem], params: csk_params) -> int:
    arr, dt = _host_problems(probs)
    return int(lib().csk_solve_host_many_workspace_size(arr, len(probs), dt, ctypes.byref(params)))


def csk_solve_host_many(probs: list[HostProblem], params: csk_params, *, ws: torch.Tensor,
                        device=None) -> int:
    """Solve every problem of ``probs`` (host memory) in order, the copies of
    the next one overlapping the current solve.  Fills each problem's x_out
    and info; returns the call's status (first non-OK solve status, else 0)."""
    arr, dt = _host_problems(probs)
    dev = ws.device if device is None else device
    rc = lib().csk_solve_host_many(arr, len(probs), dt, ctypes.byref(params), _ptr(ws), ws.numel(),
                                   _stream(dev))
    if rc < 0 and not any(q.info is not None and q.info["status"][0] == rc for q in probs):
        raise CskError(rc, "csk_solve_host_many")
    return rc


def csk_synth_systems(systems: list[tuple], device=None) -> None:
    """Fill seeded Gaussian systems on the device: ``systems`` holds tuples
    (A, X, B, seed) of contiguous FP32 device tensors (m x n, n x R, m x R);
    A and X get N(0,1) entries keyed by the seed, B = A X.  Enqueued on the
    current stream."""
    if not systems:
        return
    arr = (csk_synth_system * len(systems))()
    dev = None
    for q, (A, X, B, seed) in enumerate(systems):
        dev = _check_cuda(A, X, B)
        for t in (A, X, B):
            if t.dtype != torch.float32 or not t.is_contiguous():
                raise TypeError("synthetic systems are contiguous FP32")
        m, n = A.shape
        R = X.shape[1]
        if tuple(X.shape) != (n, R) or tuple(B.shape) != (m, R):
            raise ValueError("A m x n, X n x R, B m x R")
        arr[q] = csk_synth_system(m, n, R, 0, seed & (2**64 - 1), _ptr(A), _ptr(X), _ptr(B))
    rc = lib().csk_synth_systems(arr, len(systems), _stream(dev if device is None else device))
    if rc != CSK_OK:
        raise CskError(rc, "csk_synth_systems")


def info_dict(info: np.ndarray) -> dict:
    rec = info[0]
    return {k: rec[k].item() for k in INFO_DTYPE.names if not k.startswith("reserved")}


def csk_sketch_noalloc(A: torch.Tensor, d: int, seed: int, b: torch.Tensor | None = None, *,
                       norms: bool = True, perm: bool = False, off: bool = False) -> Sketch:
    """csk_sketch through the entry point that takes no workspace: the
    library's static scratch is used instead (m <= 2^20, d <= 2^18; calls
    must not overlap on the GPU).  Outputs are allocated here as usual."""
    dev = _check_cuda(A, b)
    lda = _rowmajor(A)
    m, n = A.shape
    dt = _dtype_code(A)
    nrhs, ldb, B = 0, 0, None
    if b is not None:
        if b.dtype != A.dtype:
            raise TypeError("b must have A's dtype")
        B = b.reshape(m, -1)
        if B.stride(1) != 1:
            raise ValueError("b must be contiguous along right-hand sides")
        nrhs, ldb = B.shape[1], B.stride(0)
    At = torch.empty((d, n), dtype=A.dtype, device=dev)
    bt = torch.empty((d, nrhs), dtype=A.dtype, device=dev) if nrhs else None
    N2 = torch.empty(d, dtype=torch.float64, device=dev) if norms else None
    P = torch.empty(m, dtype=torch.int32, device=dev) if perm else None
    O = torch.empty(d + 1, dtype=torch.int32, device=dev) if off else None
    rc = lib().csk_sketch_noalloc(_ptr(A), m, n, lda, _ptr(B), ldb, nrhs, dt, d,
                                  seed & (2**64 - 1), _ptr(At), _ptr(bt), _ptr(N2), _ptr(P),
                                  _ptr(O), _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_sketch_noalloc")
    if bt is not None and b.dim() == 1:
        bt = bt[:, 0]
    return Sketch(At, bt, N2, P, O)


@dataclass
class BatchSystem:
    """One system of a batched solve (device tensors)."""
    A: torch.Tensor               # m x n FP32
    B: torch.Tensor               # m x R FP32
    d: int
    seed: int
    X0: torch.Tensor | None = None      # n x R
    Xstar: torch.Tensor | None = None   # n x R
    Xout: torch.Tensor | None = None    # n x R (allocated when None)
    info: torch.Tensor | None = None    # R x 64 bytes (allocated when None)
    area: torch.Tensor | None = None    # resident area (csk_batched_area_size bytes)


def _systems(batch: list[BatchSystem]):
    arr = (csk_system * len(batch))()
    for i, y in enumerate(batch):
        _check_cuda(y.A, y.B, y.X0, y.Xstar, y.Xout, y.info)
        if y.A.dtype != torch.float32 or y.B.dtype != torch.float32:
            raise TypeError("batched solves take FP32 systems")
        m, n = y.A.shape
        R = y.B.shape[1]
        for t in (y.X0, y.Xstar):
            if t is not None and (tuple(t.shape) != (n, R) or not t.is_contiguous()):
                raise ValueError("X0 / Xstar must be contiguous n x R")
        if y.Xout is None:
            y.Xout = torch.empty((n, R), dtype=torch.float32, device=y.A.device)
        if y.info is None:
            y.info = torch.zeros((R, 64), dtype=torch.uint8, device=y.A.device)
        arr[i] = csk_system(_ptr(y.A), m, n, _rowmajor(y.A), _ptr(y.B), y.B.stride(0), R, 0, y.d,
                            y.seed & (2**64 - 1), _ptr(y.X0), _ptr(y.Xstar), _ptr(y.Xout),
                            _ptr(y.info), _ptr(y.area))
    return arr


def csk_solve_batched_workspace_size(batch: list[BatchSystem]) -> int:
    arr = _systems(batch)
    return int(lib().csk_solve_batched_workspace_size(arr, len(batch)))


def csk_solve_batched(batch: list[BatchSystem], params: csk_params, *, ws: torch.Tensor | None = None,
                      sync: bool = True):
    """All (system, right-hand side) solves of ``batch`` in one persistent launch.
    Returns per-system (Xout, list of info dicts) when ``sync``."""
    arr = _systems(batch)
    dev = batch[0].A.device
    if ws is None:
        ws = _workspace(int(lib().csk_solve_batched_workspace_size(arr, len(batch))), dev)
    rc = lib().csk_solve_batched(arr, len(batch), ctypes.byref(params), _ptr(ws), ws.numel(),
                                 _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_solve_batched")
    if not sync:
        return batch
    torch.cuda.synchronize(dev)
    out = []
    for y in batch:
        recs = np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=INFO_DTYPE)
        out.append((y.Xout, [{k: r[k].item() for k in INFO_DTYPE.names if not k.startswith("reserved")}
                             for r in recs]))
    return out


def csk_solve_batched_set_plan(batch: list[BatchSystem], threads: int, grid: int) -> None:
    """Install (threads, grid) as the launch shape csk_solve_batched uses for
    batches with this batch's signature when called with threads = grid = 0
    (threads = grid = 0 removes it)."""
    arr = _systems(batch)
    rc = lib().csk_solve_batched_set_plan(arr, len(batch), threads, grid)
    if rc != CSK_OK:
        raise CskError(rc, "csk_solve_batched_set_plan")


def csk_solve_batched_signature(batch: list) -> int:
    """The batch signature the tuned plans are keyed by.  Accepts BatchSystem
    objects or plain (m, n, d, nrhs) tuples (no device memory needed)."""
    arr = (csk_system * len(batch))()
    for i, y in enumerate(batch):
        if isinstance(y, BatchSystem):
            m, n = y.A.shape
            arr[i] = csk_system(None, m, n, n, None, y.B.shape[1], y.B.shape[1], 0, y.d, 0, None,
                                None, None, None)
        else:
            m, n, d, R = y
            arr[i] = csk_system(None, m, n, n, None, R, R, 0, d, 0, None, None, None, None)
    return int(lib().csk_solve_batched_signature(arr, len(batch)))


def csk_batched_area_size(n: int, d: int, nrhs: int) -> int:
    """Bytes of one system's resident area (sketch, Gram matrix, unit states)."""
    return int(lib().csk_batched_area_size(n, d, nrhs))


def csk_batched_prepare(batch: list[BatchSystem], *, ws: torch.Tensor | None = None) -> None:
    """Sketch and Gram matrix of every system into its area (allocated here
    when the system has none); resets the systems' units.  Enqueued on the
    current stream."""
    for y in batch:
        if y.area is None:
            R = y.B.shape[1]
            y.area = torch.empty(csk_batched_area_size(y.A.shape[1], y.d, R), dtype=torch.uint8,
                                 device=y.A.device)
    arr = _systems(batch)
    dev = batch[0].A.device
    if ws is None:
        ws = _workspace(int(lib().csk_batched_prepare_workspace_size(arr, len(batch))), dev)
    rc = lib().csk_batched_prepare(arr, len(batch), _ptr(ws), ws.numel(), _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_batched_prepare")


def csk_batched_iterate(batch: list[BatchSystem], params: csk_params, step_budget: int, *,
                        ws: torch.Tensor | None = None) -> None:
    """Run every unfinished unit of the prepared systems for at most
    step_budget more steps (0: to the end).  Enqueued on the current stream;
    finished units have their Xout column and info written, the others report
    CSK_INPROGRESS."""
    arr = _systems(batch)
    dev = batch[0].A.device
    if ws is None:
        ws = _workspace(int(lib().csk_batched_iterate_workspace_size(arr, len(batch))), dev)
    rc = lib().csk_batched_iterate(arr, len(batch), ctypes.byref(params), int(step_budget),
                                   _ptr(ws), ws.numel(), _stream(dev))
    if rc != CSK_OK:
        raise CskError(rc, "csk_batched_iterate")
