"""Plain CPU oracle of the Count Sketch Kaczmarz method (arXiv 2004.02480).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
library ``csk_oracle.c`` (binary64 throughout, no BLAS) with numpy arrays and
shares no code with the CUDA library in ``paper_2004_02480_gb300``.

Each wrapper names the part of the paper it restates:

* :func:`count_sketch_map`   -- Definition 1 (h : [m] -> [d], D = diag(+-1))
* :func:`stable_count_sort`  -- row order inside a bucket (ascending row index)
* :func:`sketch`             -- Algorithm 1, Initialize (At = S A, bt = S b)
* :func:`mwrk`               -- Algorithm 1, loop (selection + projection),
                                stopping rule of Section 3
* :func:`csk`                -- Algorithm 1 end to end; ``d == 0`` is MWRK
                                (Remark 1)
* :func:`final_check`        -- RES of Section 3 and ||bt - At x|| / ||bt||
* :func:`gram`, :func:`gram_split_bf16` -- G = At At^T, exact and split-BF16
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csk_oracle.c")
_HDR = os.path.join(_HERE, "csk_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_MAXITER, STATUS_ENUMERIC = 0, 1, -4


def build(force: bool = False) -> str:
    """Compile ``csk_oracle.c`` into ``_build/liboracle.so`` with gcc.

    ``-ffp-contract=off`` keeps every binary64 operation a separate rounding,
    so the oracle gives the same bits on x86-64 and on aarch64.
    """
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, dbl, cint = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.or_splitmix64_at.argtypes = [u64, u64]
        lib.or_splitmix64_at.restype = u64
        lib.or_count_sketch_map.argtypes = [u64, i64, i64, P, P]
        lib.or_stable_count_sort.argtypes = [P, i64, i64, P, P, P]
        lib.or_sketch_f64.argtypes = [P, i64, i64, i64, P, i64, i64, P, P, i64, P, P]
        lib.or_sketch_f32_same_order.argtypes = [P, i64, i64, i64, P, i64, i64, P, P, i64, P, P]
        lib.or_row_norms2_f64.argtypes = [P, i64, i64, i64, P]
        lib.or_row_norms2_of_f32.argtypes = [P, i64, i64, i64, P]
        lib.or_mwrk.argtypes = [P, P, i64, i64, i64, P, P, dbl, i64, cint, P, P,
                                i64, P, P, P, P, P]
        lib.or_mwrk.restype = cint
        lib.or_csk.argtypes = [P, P, i64, i64, i64, i64, u64, P, P, dbl, i64, cint, P, P]
        lib.or_csk.restype = cint
        lib.or_final_check.argtypes = [P, P, i64, i64, i64, P, P, P, P]
        lib.or_bf16_round.argtypes = [ctypes.c_float]
        lib.or_bf16_round.restype = ctypes.c_float
        lib.or_gram_f64.argtypes = [P, i64, i64, i64, P]
        lib.or_gram_split_bf16.argtypes = [P, i64, i64, i64, P]
        lib.or_gram_split_bf16_rows.argtypes = [P, i64, i64, i64, P, i64, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def splitmix64_at(seed: int, c: int) -> int:
    """SplitMix64 output number ``c`` (c >= 1) of the stream seeded with ``seed``."""
    return int(_load().or_splitmix64_at(seed & (2**64 - 1), c & (2**64 - 1)))


def count_sketch_map(seed: int, m: int, d: int):
    """Definition 1: bucket ``h[i]`` in [0, d) and sign ``D_ii`` in {+1, -1}."""
    h = np.empty(m, np.int32)
    s = np.empty(m, np.int8)
    _load().or_count_sketch_map(seed & (2**64 - 1), m, d, _p(h), _p(s))
    return h, s


def stable_count_sort(h, d: int):
    """Counting sort by bucket, stable in the row index: (cnt, off, perm)."""
    h = _c(h, np.int32)
    m = h.shape[0]
    cnt = np.empty(d, np.int32)
    off = np.empty(d + 1, np.int32)
    perm = np.empty(m, np.int32)
    _load().or_stable_count_sort(_p(h), m, d, _p(cnt), _p(off), _p(perm))
    return cnt, off, perm


def sketch(A, b, h, sign, d: int):
    """Algorithm 1 Initialize, binary64: (At, bt) = (S A, S b).

    ``b`` may be a vector, an (m, R) block of right-hand sides, or None.
    """
    A = _c(A, np.float64)
    m, n = A.shape
    h, sign = _c(h, np.int32), _c(sign, np.int8)
    At = np.empty((d, n), np.float64)
    if b is None:
        _load().or_sketch_f64(_p(A), m, n, n, None, 0, 0, _p(h), _p(sign), d, _p(At), None)
        return At, None
    b = _c(b, np.float64)
    vec = b.ndim == 1
    B = b.reshape(m, -1)
    R = B.shape[1]
    bt = np.empty((d, R), np.float64)
    _load().or_sketch_f64(_p(A), m, n, n, _p(B), R, R, _p(h), _p(sign), d, _p(At), _p(bt))
    return At, (bt[:, 0].copy() if vec else bt)


def sketch_f32_same_order(A, b, h, sign, d: int):
    """FP32 sketch with sequential binary32 additions in ascending row index."""
    A = _c(A, np.float32)
    m, n = A.shape
    h, sign = _c(h, np.int32), _c(sign, np.int8)
    At = np.empty((d, n), np.float32)
    if b is None:
        _load().or_sketch_f32_same_order(_p(A), m, n, n, None, 0, 0, _p(h), _p(sign), d,
                                         _p(At), None)
        return At, None
    b = _c(b, np.float32)
    vec = b.ndim == 1
    B = b.reshape(m, -1)
    R = B.shape[1]
    bt = np.empty((d, R), np.float32)
    _load().or_sketch_f32_same_order(_p(A), m, n, n, _p(B), R, R, _p(h), _p(sign), d,
                                     _p(At), _p(bt))
    return At, (bt[:, 0].copy() if vec else bt)


def row_norms2(At):
    """Squared row norms ||At_j||^2 accumulated in binary64."""
    d, n = At.shape
    N = np.empty(d, np.float64)
    if At.dtype == np.float32:
        At = _c(At, np.float32)
        _load().or_row_norms2_of_f32(_p(At), d, n, n, _p(N))
    else:
        At = _c(At, np.float64)
        _load().or_row_norms2_f64(_p(At), d, n, n, _p(N))
    return N


@dataclass
class MwrkResult:
    x: np.ndarray
    iters: int
    status: int
    ik: np.ndarray | None = None
    gap: np.ndarray | None = None
    err2: np.ndarray | None = None
    r_ik: np.ndarray | None = None
    n_ik: np.ndarray | None = None


def mwrk(At, bt, x0=None, x_star=None, tol: float = 1e-6, max_iter: int = 20000,
         nthreads: int = 1, log_len: int = 0) -> MwrkResult:
    """Algorithm 1 loop on (At, bt), literal: full residual every step."""
    At = _c(At, np.float64)
    bt = _c(bt, np.float64)
    d, n = At.shape
    x0 = _c(x0, np.float64)
    xs = _c(x_star, np.float64)
    x = np.empty(n, np.float64)
    it = ctypes.c_int64(0)
    L = int(log_len)
    ik = np.full(L, -1, np.int32) if L else None
    gap = np.full(L, np.nan) if L else None
    err2 = np.full(L, np.nan) if L else None
    rik = np.full(L, np.nan) if L else None
    nik = np.full(L, np.nan) if L else None
    st = _load().or_mwrk(_p(At), _p(bt), d, n, n, _p(x0), _p(xs), tol, max_iter,
                         nthreads, _p(x), ctypes.byref(it), L, _p(ik), _p(gap),
                         _p(err2), _p(rik), _p(nik))
    k = it.value
    if L:
        ik, gap, rik, nik = ik[:min(k, L)], gap[:min(k, L)], rik[:min(k, L)], nik[:min(k, L)]
        err2 = err2[:min(k + 1, L)]
    return MwrkResult(x, k, st, ik, gap, err2, rik, nik)


def csk(A, b, d: int, seed: int, x0=None, x_star=None, tol: float = 1e-6,
        max_iter: int = 20000, nthreads: int = 1) -> MwrkResult:
    """Algorithm 1 end to end (d == 0: MWRK on A, Remark 1)."""
    A = _c(A, np.float64)
    b = _c(b, np.float64)
    m, n = A.shape
    x = np.empty(n, np.float64)
    it = ctypes.c_int64(0)
    st = _load().or_csk(_p(A), _p(b), m, n, n, d, seed & (2**64 - 1), _p(_c(x0, np.float64)),
                        _p(_c(x_star, np.float64)), tol, max_iter, nthreads, _p(x),
                        ctypes.byref(it))
    return MwrkResult(x, it.value, st)


def final_check(At, bt, x, x_star=None):
    """(RES, ||bt - At x|| / ||bt||) in binary64."""
    At = _c(At, np.float64)
    bt = _c(bt, np.float64)
    d, n = At.shape
    rse = ctypes.c_double(0)
    res = ctypes.c_double(0)
    _load().or_final_check(_p(At), _p(bt), d, n, n, _p(_c(x, np.float64)),
                           _p(_c(x_star, np.float64)), ctypes.byref(rse), ctypes.byref(res))
    return rse.value, res.value


def bf16_round(v: float) -> float:
    return float(_load().or_bf16_round(ctypes.c_float(v)))


def gram(At):
    At = _c(At, np.float64)
    d, n = At.shape
    G = np.empty((d, d), np.float64)
    _load().or_gram_f64(_p(At), d, n, n, _p(G))
    return G


def gram_split_bf16(At):
    At = _c(At, np.float32)
    d, n = At.shape
    G = np.empty((d, d), np.float64)
    _load().or_gram_split_bf16(_p(At), d, n, n, _p(G))
    return G


def gram_split_bf16_rows(At, rows):
    """Rows ``rows`` of the split-BF16 Gram product (len(rows) x d, binary64)."""
    At = _c(At, np.float32)
    d, n = At.shape
    rows = _c(rows, np.int64)
    G = np.empty((rows.shape[0], d), np.float64)
    _load().or_gram_split_bf16_rows(_p(At), d, n, n, _p(rows), rows.shape[0], _p(G))
    return G
