"""Oracle for the embedding similarity join -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never calls
it, and it shares no code with the CUDA path (see ``sj_oracle.c`` for the
definitions it follows: Sec. 3.1 join-as-product, exact dot products of the
stored float32 rows, tie-break (score desc, index asc), inclusive threshold).

The C source is compiled with gcc into ``oracle/_build/`` on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsj_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, OpenMP) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.sjo_topk.restype = I64
        lib.sjo_topk.argtypes = [P, P, I64, I64, ctypes.c_int, P, I64, P, P, P]
        lib.sjo_threshold.restype = I64
        lib.sjo_threshold.argtypes = [P, P, I64, I64, ctypes.c_double, P, I64, P, P,
                                      P, P, P]
        lib.sjo_exact_dot.restype = ctypes.c_int
        lib.sjo_exact_dot.argtypes = [P, P, I64, P, P, P]
        lib.sjo_enclose_all.restype = None
        lib.sjo_enclose_all.argtypes = [P, P, I64, I64, I64, P, P]
        lib.sjo_exact_dot_minus.restype = ctypes.c_int
        lib.sjo_exact_dot_minus.argtypes = [P, P, I64, ctypes.c_double, P]
        lib.sjo_exact_dot_rounded.restype = None
        lib.sjo_exact_dot_rounded.argtypes = [P, P, I64, P, P]
        lib.sjo_num_threads.restype = ctypes.c_int
        lib.sjo_infonce.restype = None
        lib.sjo_infonce.argtypes = [P, P, I64, I64, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, P, P, P, P, P]
        lib.sjo_infonce_rows.restype = None
        lib.sjo_infonce_rows.argtypes = [P, P, I64, I64, ctypes.c_double,
                                         ctypes.c_double, P, I64, P, P]
        _lib = lib
        return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim != 2:
        raise ValueError("expected a 2-D array")
    return x


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS honoured)."""
    return int(_load().sjo_num_threads())


def topk(A, B, k: int, rows=None):
    """Exact top-k join: (idx int64 [r,k], score float32 [r,k], score float64 [r,k]).

    Row r of the output is left row ``rows[r]`` (all rows when ``rows`` is None).
    Order is (exact score desc, j asc); k > |B| pads with (-1, -inf).
    """
    A, B = _f32(A), _f32(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("A and B must have the same width")
    d = A.shape[1]
    if k < 1:
        raise ValueError("k must be >= 1")
    if rows is None:
        nrows, rp = A.shape[0], None
    else:
        rp = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = rp.shape[0]
    idx = np.empty((nrows, k), np.int64)
    s32 = np.empty((nrows, k), np.float32)
    s64 = np.empty((nrows, k), np.float64)
    if nrows:
        _load().sjo_topk(_p(A), _p(B), B.shape[0], d, k, _p(rp), nrows, _p(idx),
                         _p(s32), _p(s64))
    return idx, s32, s64


def _clamp_tau(tau: float) -> float:
    # |s| < 2^288 for any finite float32 rows, so clamping tau to +-2^290
    # never changes a decision and keeps it inside the fixed-point range.
    lim = 2.0 ** 290
    return float(min(max(float(tau), -lim), lim))


def threshold(A, B, tau: float, rows=None, want_s64: bool = True):
    """Exact threshold join { (i, j) : s_ij >= tau }, sorted by (i, j).

    Returns (i int64, j int64, score float32, score float64 or None).
    """
    A, B = _f32(A), _f32(B)
    d = A.shape[1]
    if rows is None:
        rows_arr = np.arange(A.shape[0], dtype=np.int64)
        rp = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        rp = rows_arr
    nrows = rows_arr.shape[0]
    tau = _clamp_tau(tau)
    lib = _load()
    counts = np.zeros(nrows, np.int64)
    if nrows:
        lib.sjo_threshold(_p(A), _p(B), B.shape[0], d, tau, _p(rp), nrows, _p(counts),
                          None, None, None, None)
    offs = np.zeros(nrows, np.int64)
    if nrows > 1:
        offs[1:] = np.cumsum(counts)[:-1]
    total = int(counts.sum())
    j = np.empty(total, np.int64)
    s32 = np.empty(total, np.float32)
    s64 = np.empty(total, np.float64) if want_s64 else None
    if total:
        lib.sjo_threshold(_p(A), _p(B), B.shape[0], d, tau, _p(rp), nrows, None,
                          _p(offs), _p(j), _p(s32), _p(s64))
    i = np.repeat(rows_arr, counts)
    return i, j, s32, s64


def exact_dot(a, b) -> Fraction:
    """Exact <a, b> of two float32 vectors as a Fraction (from the big accumulator)."""
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    mag = np.zeros(64, np.uint32)
    lsb = ctypes.c_int(0)
    nd = ctypes.c_int(0)
    sign = _load().sjo_exact_dot(_p(a), _p(b), a.shape[0], _p(mag), ctypes.byref(lsb),
                                 ctypes.byref(nd))
    v = 0
    for t in range(nd.value - 1, -1, -1):
        v = (v << 32) | int(mag[t])
    return sign * Fraction(v) * Fraction(2) ** lsb.value


def enclose_all(A, B):
    """(lo, hi), each nA x nB float64: an interval around the exact s_ij of
    every pair, from the FP64 naive sum and its rounding-error bound."""
    A, B = _f32(A), _f32(B)
    lo = np.empty((A.shape[0], B.shape[0]), np.float64)
    hi = np.empty_like(lo)
    if lo.size:
        _load().sjo_enclose_all(_p(A), _p(B), A.shape[0], B.shape[0], A.shape[1], _p(lo), _p(hi))
    return lo, hi


def exact_dot_minus(a, b, t: float) -> Fraction:
    """Exact <a, b> - t (t a double, clamped like a threshold) as a Fraction:
    the value whose sign decides s >= t."""
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    mag = np.zeros(64, np.uint32)
    lib = _load()
    sign = lib.sjo_exact_dot_minus(_p(a), _p(b), a.shape[0], _clamp_tau(t), _p(mag))
    lsb = ctypes.c_int(0)
    nd = ctypes.c_int(0)
    lib.sjo_exact_dot(_p(a), _p(b), 0, _p(np.zeros(64, np.uint32)), ctypes.byref(lsb),
                      ctypes.byref(nd))
    v = 0
    for q in range(nd.value - 1, -1, -1):
        v = (v << 32) | int(mag[q])
    return sign * Fraction(v) * Fraction(2) ** lsb.value


def exact_dot_rounded(a, b):
    """(RN_fp32, RN_fp64) of the exact <a, b>."""
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    s32 = np.zeros(1, np.float32)
    s64 = np.zeros(1, np.float64)
    _load().sjo_exact_dot_rounded(_p(a), _p(b), a.shape[0], _p(s32), _p(s64))
    return s32[0], s64[0]


def bf16_bits_to_f64(x) -> np.ndarray:
    """Exact FP64 values of bfloat16 data given as raw uint16 bit patterns."""
    x = np.ascontiguousarray(x)
    if x.dtype != np.uint16:
        raise TypeError("pass bfloat16 data as its raw uint16 bit patterns")
    return (x.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _f64_in(x) -> np.ndarray:
    x = np.asarray(x)
    if x.dtype == np.uint16:
        return bf16_bits_to_f64(x)
    return np.ascontiguousarray(x, dtype=np.float64)


def infonce(A_in, B_in, T: float, sym: bool = False, g: float = 1.0,
            grads: bool = True):
    """FP64 InfoNCE over S = A B^T / T.

    Inputs: bfloat16 data as raw uint16 bit patterns (converted exactly) or any
    real array (used as FP64, e.g. for finite differences).
    Returns (loss, lse_row, lse_col or None, dA or None, dB or None).
    """
    A, B = _f64_in(A_in), _f64_in(B_in)
    N, d = A.shape
    lse_row = np.empty(N, np.float64)
    lse_col = np.empty(N, np.float64) if sym else None
    dA = np.empty((N, d), np.float64) if grads else None
    dB = np.empty((N, d), np.float64) if grads else None
    loss = np.zeros(1, np.float64)
    _load().sjo_infonce(_p(A), _p(B), N, d, float(T), int(bool(sym)), float(g), _p(loss),
                        _p(lse_row), _p(lse_col), _p(dA), _p(dB))
    return float(loss[0]), lse_row, lse_col, dA, dB


def infonce_rows(A_in, B_in, T: float, rows, g: float = 1.0, grads: bool = True):
    """Row logsumexp and one-directional dA for the listed rows only."""
    A, B = _f64_in(A_in), _f64_in(B_in)
    N, d = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    lse = np.empty(rows.shape[0], np.float64)
    dA = np.empty((rows.shape[0], d), np.float64) if grads else None
    _load().sjo_infonce_rows(_p(A), _p(B), N, d, float(T), float(g), _p(rows),
                             rows.shape[0], _p(lse), _p(dA))
    return lse, dA
