"""Python binding of libsj.so (include/sj.h): argument marshalling only.

Every step of the join runs inside the CUDA library; this module only turns
torch tensors / numpy arrays into pointers and sizes, allocates outputs and
maps status codes to exceptions.  If the library cannot be loaded the calls
raise -- there is no CPU fallback.

The C entry points are exposed under their own names (``sj_create``,
``sj_topk``, ``sj_threshold``, ``sj_batch``, ``sj_contrastive_fwd``,
``sj_backward``, ...) through :func:`lib`; :class:`SimilarityJoin` wraps a
handle for torch users.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

SJ_OK = 0
SJ_ERR_INVALID_ARG = 1
SJ_ERR_NONFINITE = 2
SJ_ERR_NOT_UNIT_NORM = 3
SJ_ERR_CAPACITY = 4
SJ_ERR_OOM = 5
SJ_ERR_CUDA = 6
SJ_ERR_TIMEOUT = 7
SJ_ERR_UNSUPPORTED = 8
SJ_ERR_INTERNAL = 9

SJ_FP32, SJ_BF16, SJ_FP8_E4M3, SJ_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp32": SJ_FP32, "bf16": SJ_BF16, "fp8": SJ_FP8_E4M3, "bf16x3": SJ_BF16X3}

SJ_FLAG_SYM_INFONCE = 0x1
SJ_FLAG_SINGLE_SPLIT = 0x2
SJ_FLAG_NO_GRAPH = 0x4
SJ_FLAG_NARROW_TILES = 0x8
SJ_FLAG_FUSED_BACKWARD = 0x10
SJ_FLAG_BLOCK_SPARSE = 0x20
SJ_FLAG_DEBUG_TIMEOUT = 0x100

# every symbol include/sj.h declares
EXPORTS = ("sj_create", "sj_destroy", "sj_topk", "sj_threshold", "sj_batch",
           "sj_contrastive_fwd", "sj_backward", "sj_topk_noalloc", "sj_status_string",
           "sj_version", "sj_last_error_detail", "sj_autotune", "sj_autotune_load",
           "sj_debug_scores", "sj_block", "sj_join_groupby_sum", "sj_join_sum_product",
           "sj_plan", "sj_contrastive_fwd_rows", "sj_backward_rows", "sj_topk_streamed",
           "sj_threshold_streamed")

I64, P = ctypes.c_int64, ctypes.c_void_p


class SjConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", P), ("prec", ctypes.c_int),
                ("d", I64), ("flags", ctypes.c_uint32), ("workspace_limit", ctypes.c_size_t)]


class SjStats(ctypes.Structure):
    _fields_ = [("ms_prepare", ctypes.c_double), ("ms_score", ctypes.c_double),
                ("ms_select", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("n_candidates", I64), ("n_rescored", I64), ("n_exact", I64),
                ("n_overflow_rows", I64), ("n_pairs", I64),
                ("margin_max", ctypes.c_double), ("max_abs_err_lowprec", ctypes.c_double),
                ("n_launches", I64), ("n_tier2_rows", I64), ("graph_replayed", I64),
                ("padded_pair_scores", ctypes.c_double), ("n_rejoined_rows", I64),
                ("n_rejoined_again", I64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SjPair(ctypes.Structure):
    _fields_ = [("i", I64), ("j", I64), ("score", ctypes.c_float), ("_pad", ctypes.c_int32)]


class SjJob(ctypes.Structure):
    _fields_ = [("A", P), ("nA", I64), ("B", P), ("nB", I64), ("k", ctypes.c_int32),
                ("tau", ctypes.c_double), ("topk_idx", P), ("topk_score", P), ("pairs", P),
                ("capacity", I64), ("n_out", P)]


class SjGroup(ctypes.Structure):
    _fields_ = [("group", I64), ("sum_lo", ctypes.c_uint64), ("sum_hi", I64), ("count", I64)]

    def exact_sum(self) -> int:
        """The 128-bit two's complement SUM as a Python int."""
        return (int(self.sum_hi) << 64) + int(self.sum_lo)


class SjPlanInfo(ctypes.Structure):
    _fields_ = [("choice", ctypes.c_int), ("_pad", ctypes.c_int32),
                ("est_ms", ctypes.c_double * 4), ("score_ms", ctypes.c_double * 4),
                ("select_ms", ctypes.c_double * 4), ("cand_per_row", ctypes.c_double * 4),
                ("overflow_frac", ctypes.c_double * 4), ("sample_rows", I64)]

    def as_dict(self):
        names = {v: k for k, v in PRECISIONS.items()}
        per = lambda arr: {names[p]: float(arr[p]) for p in range(4)}
        return {"choice": names[int(self.choice)], "est_ms": per(self.est_ms),
                "score_ms": per(self.score_ms), "select_ms": per(self.select_ms),
                "cand_per_row": per(self.cand_per_row),
                "overflow_frac": per(self.overflow_frac), "sample_rows": int(self.sample_rows)}


class SJError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = "%s failed: %s (status %d)" % (where, status_string(code), code)
        if code in (SJ_ERR_CUDA, SJ_ERR_OOM) and _lib is not None:
            detail = _lib.sj_last_error_detail()
            if detail:
                msg += " [%s]" % detail.decode(errors="replace")
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libsj.so (building it in-tree with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
        L = ctypes.CDLL(path)
        st = ctypes.c_int
        L.sj_last_error_detail.restype = ctypes.c_char_p
        L.sj_last_error_detail.argtypes = []
        L.sj_autotune.restype = st
        L.sj_autotune.argtypes = [P, ctypes.c_int32, ctypes.c_char_p]
        L.sj_autotune_load.restype = st
        L.sj_autotune_load.argtypes = [P, ctypes.c_char_p]
        L.sj_create.restype = st
        L.sj_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(SjConfig)]
        L.sj_destroy.restype = st
        L.sj_destroy.argtypes = [P]
        L.sj_topk.restype = st
        L.sj_topk.argtypes = [P, P, I64, P, I64, ctypes.c_int32, P, P, ctypes.POINTER(SjStats)]
        L.sj_threshold.restype = st
        L.sj_threshold.argtypes = [P, P, I64, P, I64, ctypes.c_double, P, I64,
                                   ctypes.POINTER(I64), ctypes.POINTER(SjStats)]
        L.sj_batch.restype = st
        L.sj_batch.argtypes = [P, ctypes.POINTER(SjJob), ctypes.c_int32, ctypes.POINTER(SjStats)]
        L.sj_contrastive_fwd.restype = st
        L.sj_contrastive_fwd.argtypes = [P, P, P, I64, ctypes.c_float, P, P]
        L.sj_backward.restype = st
        L.sj_backward.argtypes = [P, P, P, I64, ctypes.c_float, P, P, P, P]
        L.sj_block.restype = st
        L.sj_block.argtypes = [P, P, I64, P, I64, ctypes.c_int32, ctypes.c_int32, P, I64,
                               ctypes.POINTER(I64), ctypes.POINTER(SjStats)]
        L.sj_join_groupby_sum.restype = st
        L.sj_join_groupby_sum.argtypes = [P, P, P, I64, P, P, I64, P, I64, ctypes.POINTER(I64)]
        L.sj_join_sum_product.restype = st
        L.sj_join_sum_product.argtypes = [P, P, P, I64, P, P, I64, ctypes.POINTER(SjGroup)]
        L.sj_contrastive_fwd_rows.restype = st
        L.sj_contrastive_fwd_rows.argtypes = [P, P, I64, I64, P, I64, ctypes.c_float, P, P]
        L.sj_backward_rows.restype = st
        L.sj_backward_rows.argtypes = [P, P, I64, I64, P, I64, ctypes.c_float, P, P, P, P]
        L.sj_topk_streamed.restype = st
        L.sj_topk_streamed.argtypes = [P, P, I64, P, I64, ctypes.c_int32, I64, P, P,
                                       ctypes.POINTER(SjStats)]
        L.sj_threshold_streamed.restype = st
        L.sj_threshold_streamed.argtypes = [P, P, I64, P, I64, ctypes.c_double, I64, P, I64,
                                            ctypes.POINTER(I64), ctypes.POINTER(SjStats)]
        L.sj_plan.restype = st
        L.sj_plan.argtypes = [P, P, I64, P, I64, ctypes.c_int32, ctypes.c_double, I64,
                              ctypes.POINTER(SjPlanInfo)]
        L.sj_debug_scores.restype = st
        L.sj_debug_scores.argtypes = [P, P, P]
        L.sj_topk_noalloc.restype = st
        L.sj_topk_noalloc.argtypes = [P, I64, P, I64, I64, ctypes.c_int32, P, P, P]
        L.sj_status_string.restype = ctypes.c_char_p
        L.sj_status_string.argtypes = [ctypes.c_int]
        L.sj_version.restype = ctypes.c_int
        L.sj_version.argtypes = []
        _lib = L
        return L


def status_string(code: int) -> str:
    try:
        return lib().sj_status_string(int(code)).decode()
    except Exception:  # pragma: no cover - library missing
        return "status %d" % code


def _check(code: int, where: str):
    if code != SJ_OK:
        raise SJError(code, where)


def _ptr(x) -> int:
    """Pointer of a contiguous torch tensor or numpy array (device or host)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch tensor or numpy array")


def _rows(x, d):
    if x.ndim != 2 or x.shape[1] != d:
        raise ValueError("expected an (n, %d) matrix, got %s" % (d, tuple(x.shape)))
    return int(x.shape[0])


class SimilarityJoin:
    """A handle of the similarity join library bound to one device and stream.

    Inputs are float32 (n, d) matrices of unit-norm rows, as CUDA tensors (used
    in place) or host tensors / numpy arrays (staged by the library).
    """

    def __init__(self, d: int, prec: str = "bf16", device: int = 0, stream=None,
                 flags: int = 0, workspace_limit: int = 0):
        import torch
        self.d = int(d)
        self.prec = prec
        self.flags = int(flags)
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        cfg = SjConfig(self.device, P(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                      else int(stream)),
                       PRECISIONS[prec], self.d, int(flags), int(workspace_limit))
        h = P()
        _check(lib().sj_create(ctypes.byref(h), ctypes.byref(cfg)), "sj_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().sj_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _out_like(self, A, shape, dtype):
        import torch
        dev = A.device if hasattr(A, "device") else torch.device("cpu")
        return torch.empty(shape, dtype=dtype, device=dev)

    def autotune(self, k: int, path: str | None = None):
        """Time 128- and 256-column score tiles per right-side size class for
        joins with this k; later calls use the faster width.  With `path`,
        the table is merged into that file (see sj_autotune)."""
        _check(lib().sj_autotune(self._h, int(k), path.encode() if path else None),
               "sj_autotune")

    def autotune_load(self, path: str):
        """Use the widths sj_autotune wrote to `path` (this d and precision)."""
        _check(lib().sj_autotune_load(self._h, path.encode()), "sj_autotune_load")

    def topk(self, A, B, k: int, with_stats: bool = False):
        """(idx int64 [nA, k], score float32 [nA, k]) ordered (score desc, j asc)."""
        import torch
        nA, nB = _rows(A, self.d), _rows(B, self.d)
        idx = self._out_like(A, (nA, k), torch.int64)
        sc = self._out_like(A, (nA, k), torch.float32)
        st = SjStats()
        _check(lib().sj_topk(self._h, _ptr(A), nA, _ptr(B), nB, int(k), _ptr(idx), _ptr(sc),
                             ctypes.byref(st)), "sj_topk")
        return (idx, sc, st.as_dict()) if with_stats else (idx, sc)

    def threshold(self, A, B, tau: float, capacity: int | None = None,
                  with_stats: bool = False):
        """(i int64, j int64, score float32) of every pair with s_ij >= tau."""
        import torch
        nA, nB = _rows(A, self.d), _rows(B, self.d)
        if capacity is None:
            capacity = max(1024, 8 * nA)
        for _ in range(2):
            buf = self._out_like(A, (max(int(capacity), 1), 3), torch.int64)
            n = I64(0)
            st = SjStats()
            code = lib().sj_threshold(self._h, _ptr(A), nA, _ptr(B), nB, float(tau), _ptr(buf),
                                      int(capacity), ctypes.byref(n), ctypes.byref(st))
            if code == SJ_ERR_CAPACITY:
                capacity = int(n.value)
                continue
            _check(code, "sj_threshold")
            m = int(n.value)
            i = buf[:m, 0]
            j = buf[:m, 1]
            s = buf[:m, 2:3].view(torch.float32)[:, 0]
            return (i, j, s, st.as_dict()) if with_stats else (i, j, s)
        raise SJError(SJ_ERR_CAPACITY, "sj_threshold")

    def topk_streamed(self, A, B_host, k: int, chunk_rows: int = 0, with_stats: bool = False):
        """Top-k against a B held in host memory, streamed in row chunks
        (sj_topk_streamed); outputs on A's device (A may be host: cuda:0)."""
        import torch
        nA, nB = _rows(A, self.d), _rows(B_host, self.d)
        dev = A.device if hasattr(A, "device") and A.is_cuda else torch.device("cuda", self.device)
        idx = torch.empty((nA, k), dtype=torch.int64, device=dev)
        sc = torch.empty((nA, k), dtype=torch.float32, device=dev)
        st = SjStats()
        _check(lib().sj_topk_streamed(self._h, _ptr(A), nA, _ptr(B_host), nB, int(k),
                                      int(chunk_rows), _ptr(idx), _ptr(sc), ctypes.byref(st)),
               "sj_topk_streamed")
        return (idx, sc, st.as_dict()) if with_stats else (idx, sc)

    def threshold_streamed(self, A, B_host, tau: float, chunk_rows: int = 0,
                           capacity: int | None = None):
        """(i, j, score) host tensors of every pair with s_ij >= tau against a
        B held in host memory (sj_threshold_streamed)."""
        import torch
        nA, nB = _rows(A, self.d), _rows(B_host, self.d)
        if capacity is None:
            capacity = max(1024, 8 * nA)
        for _ in range(2):
            buf = torch.empty((max(int(capacity), 1), 3), dtype=torch.int64)
            n = I64(0)
            code = lib().sj_threshold_streamed(self._h, _ptr(A), nA, _ptr(B_host), nB,
                                               float(tau), int(chunk_rows), _ptr(buf),
                                               int(capacity), ctypes.byref(n), None)
            if code == SJ_ERR_CAPACITY:
                capacity = int(n.value)
                continue
            _check(code, "sj_threshold_streamed")
            m = int(n.value)
            return buf[:m, 0], buf[:m, 1], buf[:m, 2:3].view(torch.float32)[:, 0]
        raise SJError(SJ_ERR_CAPACITY, "sj_threshold_streamed")

    def plan(self, A, B, k: int = 0, tau: float | None = None, sample_rows: int = 0):
        """sj_plan: the census and cost estimate of each scoring precision for
        this join; returns a dict (choice, est_ms, ... per precision name)."""
        info = SjPlanInfo()
        _check(lib().sj_plan(self._h, _ptr(A), _rows(A, self.d), _ptr(B), _rows(B, self.d),
                             int(k), float("nan") if tau is None else float(tau),
                             int(sample_rows), ctypes.byref(info)), "sj_plan")
        return info.as_dict()

    def block(self, ka, kb, min_match: int = 1, capacity: int | None = None,
              with_stats: bool = False):
        """(i, j, score) of every pair whose n_attr int64 key attributes (the
        columns of ka, kb; 1-D for one attribute) agree in >= min_match of
        them, sorted by (i, j) (sj_block)."""
        import torch
        if ka.ndim == 1:
            ka, kb = ka.reshape(-1, 1), kb.reshape(-1, 1)
        n_attr = int(ka.shape[1])
        if kb.shape[1] != n_attr:
            raise ValueError("ka and kb need the same attributes")
        nA, nB = int(ka.shape[0]), int(kb.shape[0])
        if capacity is None:
            capacity = max(1024, 8 * nA)
        for _ in range(2):
            buf = self._out_like(ka, (max(int(capacity), 1), 3), torch.int64)
            n = I64(0)
            st = SjStats()
            code = lib().sj_block(self._h, _ptr(ka), nA, _ptr(kb), nB, n_attr, int(min_match),
                                  _ptr(buf), int(capacity), ctypes.byref(n), ctypes.byref(st))
            if code == SJ_ERR_CAPACITY:
                capacity = int(n.value)
                continue
            _check(code, "sj_block")
            m = int(n.value)
            out = (buf[:m, 0], buf[:m, 1], buf[:m, 2:3].view(torch.float32)[:, 0])
            return out + (st.as_dict(),) if with_stats else out
        raise SJError(SJ_ERR_CAPACITY, "sj_block")

    def groupby_sum(self, a_id, a_val, b_id, b_group):
        """Q3: [(group, SUM(A.Val) as an exact int, COUNT(*))] over the join
        A.ID = B.ID, groups by value (sj_join_groupby_sum).  a_id, b_id,
        b_group int64 and a_val int32 arrays (device or host)."""
        nA, nB = int(a_id.shape[0]), int(b_id.shape[0])
        cap = nB
        for _ in range(2):
            out = (SjGroup * max(1, cap))()
            n = I64(0)
            code = lib().sj_join_groupby_sum(self._h, _ptr(a_id), _ptr(a_val), nA, _ptr(b_id),
                                             _ptr(b_group), nB, out, cap, ctypes.byref(n))
            if code == SJ_ERR_CAPACITY:
                cap = int(n.value)
                continue
            _check(code, "sj_join_groupby_sum")
            return [(int(g.group), g.exact_sum(), int(g.count)) for g in out[:int(n.value)]]
        raise SJError(SJ_ERR_CAPACITY, "sj_join_groupby_sum")

    def sum_product(self, a_id, a_val, b_id, b_val):
        """Q4: (SUM(A.Val * B.Val) as an exact int, COUNT(*)) over A.ID = B.ID
        (sj_join_sum_product)."""
        r = SjGroup()
        _check(lib().sj_join_sum_product(self._h, _ptr(a_id), _ptr(a_val), int(a_id.shape[0]),
                                         _ptr(b_id), _ptr(b_val), int(b_id.shape[0]),
                                         ctypes.byref(r)), "sj_join_sum_product")
        return r.exact_sum(), int(r.count)

    def contrastive_forward(self, A, B, T: float):
        """(loss [1], lse [N] or [2N] with the symmetric flag) on CUDA tensors.

        A, B: float32 (N, d) CUDA tensors (rounded to BF16 inside the library).
        """
        import torch
        N = _rows(A, self.d)
        if _rows(B, self.d) != N:
            raise ValueError("A and B must have the same number of rows")
        sym = bool(self.flags & SJ_FLAG_SYM_INFONCE)
        loss = torch.empty(1, dtype=torch.float32, device=A.device)
        lse = torch.empty(2 * N if sym else N, dtype=torch.float32, device=A.device)
        _check(lib().sj_contrastive_fwd(self._h, _ptr(A), _ptr(B), N, float(T), _ptr(loss),
                                        _ptr(lse)), "sj_contrastive_fwd")
        return loss, lse

    def contrastive_backward(self, A, B, T: float, lse, grad_loss):
        """(dA, dB) float32 for the upstream gradient grad_loss [1] (CUDA)."""
        import torch
        N = _rows(A, self.d)
        dA = torch.empty_like(A, dtype=torch.float32)
        dB = torch.empty_like(B, dtype=torch.float32)
        g = grad_loss.reshape(1).to(torch.float32).contiguous()
        _check(lib().sj_backward(self._h, _ptr(A), _ptr(B), N, float(T), _ptr(lse), _ptr(g),
                                 _ptr(dA), _ptr(dB)), "sj_backward")
        return dA, dB

    def contrastive_forward_rows(self, A_rows, r0: int, B, T: float):
        """Row shard rows [r0, r0 + n) of the contrastive join against all of
        B: (loss_part [1], lse_rows [n]); loss_part sums over shards to the
        loss (sj_contrastive_fwd_rows)."""
        import torch
        n, N = _rows(A_rows, self.d), _rows(B, self.d)
        loss = torch.empty(1, dtype=torch.float32, device=A_rows.device)
        lse = torch.empty(n, dtype=torch.float32, device=A_rows.device)
        _check(lib().sj_contrastive_fwd_rows(self._h, _ptr(A_rows), n, int(r0), _ptr(B), N,
                                             float(T), _ptr(loss), _ptr(lse)),
               "sj_contrastive_fwd_rows")
        return loss, lse

    def contrastive_backward_rows(self, A_rows, r0: int, B, T: float, lse_rows, grad_loss):
        """(dA_rows, dB_part) of the row shard; dB_part sums over shards to dB
        (sj_backward_rows)."""
        import torch
        n, N = _rows(A_rows, self.d), _rows(B, self.d)
        dA = torch.empty_like(A_rows, dtype=torch.float32)
        dB = torch.empty_like(B, dtype=torch.float32)
        g = grad_loss.reshape(1).to(torch.float32).contiguous()
        _check(lib().sj_backward_rows(self._h, _ptr(A_rows), n, int(r0), _ptr(B), N, float(T),
                                      _ptr(lse_rows), _ptr(g), _ptr(dA), _ptr(dB)),
               "sj_backward_rows")
        return dA, dB

    def batch(self, jobs, with_stats: bool = False):
        """Run independent joins in one call.

        jobs: list of dicts with A, B and any of k (top-k) / tau (threshold,
        with optional capacity).  Returns per job a dict with 'idx', 'score'
        and/or 'i', 'j', 'pair_score'.  Jobs whose pairs exceed their capacity
        are issued once more with the required capacity.
        """
        import torch
        caps = {}
        for q, jb in enumerate(jobs):
            if jb.get("tau") is not None:
                nA, nB = _rows(jb["A"], self.d), _rows(jb["B"], self.d)
                caps[q] = int(jb.get("capacity", min(nA * nB, max(1024, 8 * nA))))
        todo = list(range(len(jobs)))
        outs = [None] * len(jobs)
        total = SjStats()
        for _ in range(2):
            arr = (SjJob * max(1, len(todo)))()
            cur = []
            for slot, q in enumerate(todo):
                jb = jobs[q]
                A, B = jb["A"], jb["B"]
                nA, nB = _rows(A, self.d), _rows(B, self.d)
                o = {}
                arr[slot].A, arr[slot].nA, arr[slot].B, arr[slot].nB = _ptr(A), nA, _ptr(B), nB
                if jb.get("k"):
                    o["idx"] = self._out_like(A, (nA, int(jb["k"])), torch.int64)
                    o["score"] = self._out_like(A, (nA, int(jb["k"])), torch.float32)
                    arr[slot].k = int(jb["k"])
                    arr[slot].topk_idx, arr[slot].topk_score = _ptr(o["idx"]), _ptr(o["score"])
                if q in caps:
                    o["_buf"] = self._out_like(A, (max(caps[q], 1), 3), torch.int64)
                    o["_n"] = I64(0)
                    arr[slot].tau = float(jobs[q]["tau"])
                    arr[slot].pairs = _ptr(o["_buf"])
                    arr[slot].capacity = caps[q]
                    arr[slot].n_out = ctypes.cast(ctypes.byref(o["_n"]), P)
                cur.append((q, o))
            st = SjStats()
            code = lib().sj_batch(self._h, arr, len(todo), ctypes.byref(st))
            for name, _t in SjStats._fields_:
                setattr(total, name, getattr(total, name) + getattr(st, name))
            if code not in (SJ_OK, SJ_ERR_CAPACITY):
                _check(code, "sj_batch")
            retry = []
            for q, o in cur:
                if "_buf" in o and int(o["_n"].value) > caps[q]:
                    caps[q] = int(o["_n"].value)
                    retry.append(q)
                    continue
                if "_buf" in o:
                    m = int(o["_n"].value)
                    buf = o.pop("_buf")
                    o.pop("_n")
                    o["i"], o["j"] = buf[:m, 0], buf[:m, 1]
                    o["pair_score"] = buf[:m, 2:3].view(torch.float32)[:, 0]
                outs[q] = o
            if not retry:
                break
            todo = retry
        if any(o is None for o in outs):
            raise SJError(SJ_ERR_CAPACITY, "sj_batch")
        return (outs, total.as_dict()) if with_stats else outs


def _contrastive_function():
    import torch

    class ContrastiveJoin(torch.autograd.Function):
        """InfoNCE over S = A B^T / T with the library's forward and backward.

        The backward recomputes score tiles on the tensor cores; no N x N
        matrix is stored.
        """

        @staticmethod
        def forward(ctx, A, B, T, join):
            A = A.contiguous()
            B = B.contiguous()
            loss, lse = join.contrastive_forward(A, B, T)
            ctx.save_for_backward(A, B, lse)
            ctx.T = T
            ctx.join = join
            return loss.reshape(())

        @staticmethod
        def backward(ctx, grad):
            A, B, lse = ctx.saved_tensors
            dA, dB = ctx.join.contrastive_backward(A, B, ctx.T, lse, grad.reshape(1))
            return dA, dB, None, None

    return ContrastiveJoin


def contrastive_loss(A, B, T: float, join: "SimilarityJoin"):
    """Differentiable InfoNCE loss of paired rows (positives on the diagonal)."""
    return _contrastive_function().apply(A, B, T, join)
