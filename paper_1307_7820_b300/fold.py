"""Thin ctypes binding of libfold_b300 (C-ABI in include/fold.h).

Every function here only marshals arguments: each step of the fold runs in
the CUDA library.  The functions keep the C names (``fold_init``,
``fold_score``, ...); :class:`Folder` wraps a context for convenience.  The
library is loaded from this directory; if it is missing, :func:`lib` raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfold_b300.so")

FOLD_OK, FOLD_EINVAL, FOLD_ENOMEM, FOLD_EAGAIN, FOLD_ETIMEOUT, FOLD_ECUDA, FOLD_ENOTREADY = range(7)
FOLD_METHOD_TWO_VECTOR, FOLD_METHOD_PLAIN, FOLD_METHOD_SLIDING, FOLD_METHOD_FG = 0, 1, 2, 3
FOLD_OPT_METHOD, FOLD_OPT_GRID, FOLD_OPT_TIMEOUT_MS, FOLD_OPT_KCHUNK = 1, 2, 3, 4
FOLD_OPT_Q, FOLD_OPT_TILE, FOLD_OPT_LAUNCHES, FOLD_OPT_TEST_DROP_TASK = 5, 6, 7, 8
FOLD_OPT_TIMING, FOLD_OPT_KERNEL_NS, FOLD_OPT_TRACE, FOLD_OPT_NEAR_CTAS, FOLD_OPT_COLUMNS = 9, 10, 11, 12, 13
FOLD_OPT_BATCH_FLAT, FOLD_OPT_R_MEMO, FOLD_OPT_BATCH_GATHER = 14, 15, 16
FOLD_OPT_COL_HELPERS = 17
FOLD_OPT_SERVE_RING = 18
FOLD_OPT_SERVE_LONG_TILES = 20
FOLD_OPT_SERVE_LONG_CAP = 21
FOLD_OPT_COL_JOIN = 19
FOLD_PAIRS_DEFAULT = 0x5A48   # AU UA CG GC GU UG
FOLD_PAIRS_PAPER = 0x1248     # AU UA CG GC
FOLD_ABI_VERSION = 1
FOLD_MAX_N = 65535
FOLD_STATIC_MAX_N = 1024

#: every symbol include/fold.h declares
ABI_SYMBOLS = (
    "fold_init", "fold_destroy", "fold_strerror", "fold_encode", "fold_set_option", "fold_get_option", "fold_rtable",
    "fold_score", "fold_workspace_bytes", "fold_score_dev", "fold_batch",
    "fold_serve_start", "fold_serve_submit", "fold_serve_poll", "fold_serve_stop", "fold_serve_stats_get",
    "fold_serve_warm", "fold_serve_wait_any",
    "fold_trace_copy",
    "fold_score_static", "fold_schedule_check", "fold_batch_schedule_check", "fold_tune", "fold_tune_q", "fold_tune_save", "fold_tune_load",
    "fold_structure", "fold_structure_workspace_bytes", "fold_structure_dev", "fold_lookup_rate",
    "fold_batch_plan_create", "fold_batch_plan_workspace_bytes", "fold_batch_plan_codes_bytes",
    "fold_batch_plan_destroy", "fold_batch_dev", "fold_batch_dev_table",
)


class TraceRec(ctypes.Structure):
    """struct fold_trace_rec"""
    _fields_ = [("worker", ctypes.c_int32), ("task", ctypes.c_int32), ("type", ctypes.c_int32),
                ("I", ctypes.c_int32), ("J", ctypes.c_int32), ("seq", ctypes.c_int32),
                ("sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_start", ctypes.c_int64), ("t_deps", ctypes.c_int64), ("t_mid", ctypes.c_int64),
                ("t_end", ctypes.c_int64), ("t_aux", ctypes.c_int64 * 3)]



class TuneResult(ctypes.Structure):
    """struct fold_tune_result"""
    _fields_ = [("q", ctypes.c_int32), ("near_ctas", ctypes.c_int32), ("columns", ctypes.c_int32),
                ("kchunk", ctypes.c_int32), ("ms", ctypes.c_float), ("default_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeStats(ctypes.Structure):
    """struct fold_serve_stats"""
    _fields_ = [("slices", ctypes.c_uint64), ("tasks", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("finished", ctypes.c_uint64), ("gpu_ms", ctypes.c_double), ("slice_ms", ctypes.c_double),
                ("prep_ms", ctypes.c_double), ("queued", ctypes.c_int32), ("inflight", ctypes.c_int32),
                ("solo", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


class FoldError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = fold_strerror(code) if _lib is not None else f"status {code}"
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def lib():
    """Load libfold_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1307_7820_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u16 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint16
    P = ctypes.POINTER
    L.fold_init.argtypes = [ctypes.c_int, u16, ctypes.c_int, P(vp)]
    L.fold_init.restype = ctypes.c_int
    L.fold_destroy.argtypes = [vp]
    L.fold_destroy.restype = None
    L.fold_strerror.argtypes = [ctypes.c_int]
    L.fold_strerror.restype = ctypes.c_char_p
    L.fold_set_option.argtypes = [vp, ctypes.c_int, i64]
    L.fold_get_option.argtypes = [vp, ctypes.c_int, P(i64)]
    L.fold_rtable.argtypes = [vp, vp, i64]
    L.fold_score.argtypes = [vp, ctypes.c_char_p, i32, P(i32), vp]
    L.fold_workspace_bytes.argtypes = [vp, i32]
    L.fold_workspace_bytes.restype = i64
    L.fold_score_dev.argtypes = [vp, vp, i32, vp, i64, vp, vp, vp]
    L.fold_batch.argtypes = [vp, i32, P(ctypes.c_char_p), P(i32), P(i32), P(vp)]
    L.fold_serve_start.argtypes = [vp, i64, i32]
    L.fold_serve_submit.argtypes = [vp, ctypes.c_char_p, i32, P(ctypes.c_uint64)]
    L.fold_serve_poll.argtypes = [vp, ctypes.c_uint64, P(i32), vp]
    L.fold_serve_stop.argtypes = [vp]
    L.fold_serve_stats_get.argtypes = [vp, P(ServeStats)]
    L.fold_serve_warm.argtypes = [vp, i32]
    L.fold_serve_wait_any.argtypes = [vp, i32, P(ctypes.c_uint64)]
    L.fold_serve_wait_any.restype = ctypes.c_int
    L.fold_trace_copy.argtypes = [vp, vp, i64]
    L.fold_score_static.argtypes = [vp, i32, u16, vp, vp, vp]
    L.fold_encode.argtypes = [ctypes.c_char_p, i32, vp]
    L.fold_lookup_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i32, P(ctypes.c_double), P(ctypes.c_double)]
    L.fold_lookup_rate.restype = ctypes.c_int
    L.fold_batch_plan_create.argtypes = [vp, i32, P(i32), P(vp)]
    L.fold_batch_plan_create.restype = ctypes.c_int
    L.fold_batch_plan_workspace_bytes.argtypes = [vp]
    L.fold_batch_plan_workspace_bytes.restype = i64
    L.fold_batch_plan_codes_bytes.argtypes = [vp]
    L.fold_batch_plan_codes_bytes.restype = i64
    L.fold_batch_plan_destroy.argtypes = [vp]
    L.fold_batch_plan_destroy.restype = None
    L.fold_batch_dev.argtypes = [vp, vp, vp, vp, i64, vp, vp]
    L.fold_batch_dev.restype = ctypes.c_int
    L.fold_batch_dev_table.argtypes = [vp, vp, vp, i32, vp, vp]
    L.fold_batch_dev_table.restype = ctypes.c_int
    L.fold_encode.restype = ctypes.c_int
    L.fold_score_static.restype = ctypes.c_int
    L.fold_schedule_check.argtypes = [i32, ctypes.c_int, ctypes.c_int, i32]
    L.fold_schedule_check.restype = ctypes.c_int
    L.fold_batch_schedule_check.argtypes = [i32, P(i32), ctypes.c_int, ctypes.c_int, i32]
    L.fold_batch_schedule_check.restype = ctypes.c_int
    L.fold_trace_copy.restype = i64
    L.fold_structure.argtypes = [vp, ctypes.c_char_p, i32, P(i32), vp, vp]
    L.fold_structure.restype = ctypes.c_int
    L.fold_structure_workspace_bytes.argtypes = [vp, i32]
    L.fold_structure_workspace_bytes.restype = i64
    L.fold_structure_dev.argtypes = [vp, vp, i32, vp, i64, vp, vp, vp]
    L.fold_structure_dev.restype = ctypes.c_int
    L.fold_tune.argtypes = [vp, i32, i32, P(TuneResult)]
    L.fold_tune_q.argtypes = [ctypes.c_int, u16, ctypes.c_int, P(i32), i32, i32, i32, P(TuneResult)]
    L.fold_tune_save.argtypes = [vp, ctypes.c_char_p]
    L.fold_tune_load.argtypes = [vp, ctypes.c_char_p]
    for name in ("fold_tune", "fold_tune_q", "fold_tune_save", "fold_tune_load"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("fold_set_option", "fold_get_option", "fold_rtable", "fold_score", "fold_score_dev", "fold_batch",
                 "fold_serve_start", "fold_serve_submit", "fold_serve_poll", "fold_serve_stop"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != FOLD_OK:
        raise FoldError(rc, what)


# ---------------------------------------------------------------- C names
def fold_strerror(code: int) -> str:
    return lib().fold_strerror(code).decode()


def fold_init(q: int = 8, pair_mask: int = FOLD_PAIRS_DEFAULT, device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().fold_init(q, pair_mask, device, ctypes.byref(h)), "fold_init")
    return h.value


def fold_destroy(ctx: int) -> None:
    lib().fold_destroy(ctx)


def fold_set_option(ctx: int, option: int, value: int) -> None:
    _check(lib().fold_set_option(ctx, option, value), "fold_set_option")


def fold_get_option(ctx: int, option: int) -> int:
    v = ctypes.c_int64()
    _check(lib().fold_get_option(ctx, option, ctypes.byref(v)), "fold_get_option")
    return v.value


def fold_rtable(ctx: int) -> np.ndarray:
    q = fold_get_option(ctx, FOLD_OPT_Q)
    out = np.zeros(1 << (2 * (q - 1)), dtype=np.uint8)
    _check(lib().fold_rtable(ctx, out.ctypes.data, out.size), "fold_rtable")
    return out


def fold_score(ctx: int, seq: str, want_D: bool = False):
    """D(0,n-1) (and the n*n int16 table if want_D) for a host string."""
    b = seq.encode("ascii")
    n = len(b)
    mp = ctypes.c_int32()
    D = np.zeros((n, n), dtype=np.int16) if want_D else None
    _check(lib().fold_score(ctx, b, n, ctypes.byref(mp), D.ctypes.data if want_D and n else None), "fold_score")
    return (mp.value, D) if want_D else mp.value


def fold_workspace_bytes(ctx: int, n: int) -> int:
    v = lib().fold_workspace_bytes(ctx, n)
    if v < 0:
        raise FoldError(-v, "fold_workspace_bytes")
    return v


def fold_score_dev(ctx: int, d_codes: int, n: int, d_ws: int, ws_bytes: int, d_max_pairs: int,
                   d_D_out: int | None = None, stream: int | None = None) -> None:
    """Enqueue a fold on device pointers (ints, e.g. torch ``data_ptr()``)."""
    _check(lib().fold_score_dev(ctx, d_codes, n, d_ws, ws_bytes, d_max_pairs, d_D_out, stream), "fold_score_dev")


def fold_batch(ctx: int, seqs, want_D: bool = False):
    bs = [s.encode("ascii") for s in seqs]
    k = len(bs)
    # one buffer holds every sequence; the pointer array points into it (kept alive by `blob`)
    blob = b"".join(bs)
    lens = np.fromiter((len(x) for x in bs), dtype=np.int32, count=k)
    offs = np.zeros(k, dtype=np.uint64)
    if k > 1:
        np.cumsum(lens[:-1], dtype=np.uint64, out=offs[1:])
    base = ctypes.cast(ctypes.c_char_p(blob), ctypes.c_void_p).value or 0
    ptrs = offs + np.uint64(base)
    out = np.zeros(max(k, 1), dtype=np.int32)
    Ds = None
    dptr = None
    if want_D:
        Ds = [np.zeros((len(x), len(x)), dtype=np.int16) for x in bs]
        dptr = (ctypes.c_void_p * k)(*[D.ctypes.data if D.size else None for D in Ds])
    _check(lib().fold_batch(ctx, k, ptrs.ctypes.data_as(ctypes.POINTER(ctypes.c_char_p)),
                            lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), dptr), "fold_batch")
    res = out[:k].copy()
    return (res, Ds) if want_D else res


def fold_trace_copy(ctx: int, cap: int = 1 << 24) -> np.ndarray:
    """Trace of the last traced launch as a numpy structured array."""
    buf = (TraceRec * cap)()
    k = lib().fold_trace_copy(ctx, buf, cap)
    if k < 0:
        raise FoldError(-k, "fold_trace_copy")
    dt = np.dtype([("worker", "i4"), ("task", "i4"), ("type", "i4"), ("I", "i4"), ("J", "i4"), ("seq", "i4"),
                   ("sm", "i4"), ("reserved", "i4"), ("t_start", "i8"), ("t_deps", "i8"), ("t_mid", "i8"), ("t_end", "i8"), ("t_aux", "i8", (3,))])
    return np.frombuffer(bytes(buf)[: k * ctypes.sizeof(TraceRec)], dtype=dt).copy()


def fold_score_static(d_codes: int | None, n: int, pair_mask: int, d_max_pairs: int,
                      d_D_out: int | None = None, stream: int | None = None) -> None:
    """Allocation-free fold of up to FOLD_STATIC_MAX_N bases (device pointers as ints)."""
    _check(lib().fold_score_static(d_codes, n, pair_mask, d_max_pairs, d_D_out, stream), "fold_score_static")


class BatchPlan:
    """A batch planned once (fold_batch_plan_create) and folded from device buffers by
    fold_batch_dev, which stream capture can record into a CUDA graph."""

    def __init__(self, ctx: int, lens):
        self.lens = np.ascontiguousarray(lens, dtype=np.int32)
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(lib().fold_batch_plan_create(ctx, len(self.lens), self.lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            ctypes.byref(h)), "fold_batch_plan_create")
        self.h = h.value
        self.offsets = np.concatenate([[0], np.cumsum(self.lens.astype(np.int64))[:-1]]) if len(self.lens) else np.zeros(0)

    @property
    def workspace_bytes(self) -> int:
        return int(lib().fold_batch_plan_workspace_bytes(self.h))

    @property
    def codes_bytes(self) -> int:
        return int(lib().fold_batch_plan_codes_bytes(self.h))

    def encode(self, seqs) -> np.ndarray:
        """The batch's sequences as one concatenated code array (the layout fold_batch_dev reads)."""
        assert [len(x) for x in seqs] == self.lens.tolist()
        return np.concatenate([encode_codes(x) for x in seqs]) if len(seqs) else np.zeros(0, np.uint8)

    def fold_dev(self, d_codes: int, d_ws: int, ws_bytes: int, d_max_pairs: int, stream: int | None = None) -> None:
        _check(lib().fold_batch_dev(self.ctx, self.h, d_codes, d_ws, ws_bytes, d_max_pairs, stream), "fold_batch_dev")

    def table_dev(self, d_ws: int, k: int, d_D_out: int, stream: int | None = None) -> None:
        _check(lib().fold_batch_dev_table(self.ctx, self.h, d_ws, k, d_D_out, stream), "fold_batch_dev_table")

    def close(self) -> None:
        if self.h:
            lib().fold_batch_plan_destroy(self.h)
            self.h = None


def fold_lookup_rate(device: int = 0, q: int = 8, mode: int = 0, iters: int = 4096):
    """(lookups per SM clock per SM, kernel ms) of the shared-memory R-lookup microbenchmark."""
    r = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(lib().fold_lookup_rate(device, q, mode, iters, ctypes.byref(r), ctypes.byref(ms)), "fold_lookup_rate")
    return r.value, ms.value


def fold_batch_schedule_check(lens, q: int = 8, method: int = FOLD_METHOD_TWO_VECTOR, kchunk: int = 0) -> int:
    """Host check of fold_batch's interleaved list for these lengths (0 = valid)."""
    arr = np.ascontiguousarray(lens, dtype=np.int32)
    return lib().fold_batch_schedule_check(len(arr), arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), q, method,
                                           kchunk)


def fold_schedule_check(n: int, q: int = 8, method: int = FOLD_METHOD_TWO_VECTOR, kchunk: int = 0) -> int:
    """0 if the task list for length n is valid (host only, no GPU)."""
    return lib().fold_schedule_check(n, q, method, kchunk)


def fold_structure(ctx: int, seq: str):
    """(max pairs, partner array int32, dot-bracket string) of one optimal structure."""
    b = seq.encode("ascii")
    n = len(b)
    mp = ctypes.c_int32()
    partner = np.full(max(n, 1), -1, dtype=np.int32)
    db = ctypes.create_string_buffer(n + 1)
    _check(lib().fold_structure(ctx, b, n, ctypes.byref(mp), partner.ctypes.data, db), "fold_structure")
    return mp.value, partner[:n], db.value.decode("ascii")


def fold_structure_workspace_bytes(ctx: int, n: int) -> int:
    r = lib().fold_structure_workspace_bytes(ctx, n)
    if r < 0:
        raise FoldError(-r, "fold_structure_workspace_bytes")
    return r


def fold_structure_dev(ctx: int, d_codes: int | None, n: int, d_ws: int, ws_bytes: int, d_max_pairs: int,
                       d_partner: int | None, stream: int | None = None) -> None:
    _check(lib().fold_structure_dev(ctx, d_codes, n, d_ws, ws_bytes, d_max_pairs, d_partner, stream),
           "fold_structure_dev")


def fold_tune(ctx: int, n: int, reps: int = 3) -> dict:
    """Times the single-fold settings for length n; the fastest is kept for that size."""
    r = TuneResult()
    _check(lib().fold_tune(ctx, n, reps, ctypes.byref(r)), "fold_tune")
    return r.as_dict()


def fold_tune_q(lens, q_min: int = 4, q_max: int = 10, pair_mask: int = FOLD_PAIRS_DEFAULT,
                method: int = FOLD_METHOD_TWO_VECTOR, device: int = 0) -> dict:
    """Fastest q for one length (tuned) or a batch of lengths (timed fold_batch)."""
    arr = (ctypes.c_int32 * len(lens))(*[int(x) for x in lens])
    r = TuneResult()
    _check(lib().fold_tune_q(device, pair_mask, method, arr, len(lens), q_min, q_max, ctypes.byref(r)), "fold_tune_q")
    return r.as_dict()


def fold_tune_save(ctx: int, path: str) -> None:
    _check(lib().fold_tune_save(ctx, path.encode()), "fold_tune_save")


def fold_tune_load(ctx: int, path: str) -> None:
    _check(lib().fold_tune_load(ctx, path.encode()), "fold_tune_load")


def fold_serve_start(ctx: int, budget_bytes: int, max_inflight: int = 4096) -> None:
    _check(lib().fold_serve_start(ctx, budget_bytes, max_inflight), "fold_serve_start")


def fold_serve_submit(ctx: int, seq: str) -> int:
    """Ticket, or raises FoldError(FOLD_EAGAIN) when the request must wait."""
    b = seq.encode("ascii")
    t = ctypes.c_uint64()
    _check(lib().fold_serve_submit(ctx, b, len(b), ctypes.byref(t)), "fold_serve_submit")
    return t.value


def fold_serve_wait_any(ctx: int, timeout_ms: int = 100) -> int | None:
    """Ticket of a finished request not reported before (collect it with fold_serve_poll), or None
    after timeout_ms."""
    t = ctypes.c_uint64()
    rc = lib().fold_serve_wait_any(ctx, timeout_ms, ctypes.byref(t))
    if rc == FOLD_ENOTREADY:
        return None
    _check(rc, "fold_serve_wait_any")
    return t.value


def fold_serve_poll(ctx: int, ticket: int, D_out: np.ndarray | None = None):
    """max pairs once done, None while the request is in flight."""
    mp = ctypes.c_int32()
    rc = lib().fold_serve_poll(ctx, ticket, ctypes.byref(mp), D_out.ctypes.data if D_out is not None else None)
    if rc == FOLD_ENOTREADY:
        return None
    _check(rc, "fold_serve_poll")
    return mp.value


def fold_serve_stop(ctx: int) -> None:
    _check(lib().fold_serve_stop(ctx), "fold_serve_stop")


def fold_serve_warm(ctx: int, max_n: int) -> None:
    """Build the task lists for every length up to max_n now instead of at first use."""
    _check(lib().fold_serve_warm(ctx, max_n), "fold_serve_warm")


def fold_serve_stats(ctx: int) -> dict:
    """Counters of the running serving loop (slices, tasks, requests, device and host time)."""
    st = ServeStats()
    _check(lib().fold_serve_stats_get(ctx, ctypes.byref(st)), "fold_serve_stats_get")
    return st.as_dict()


# ---------------------------------------------------------------- convenience
class Folder:
    """A context: ``Folder(q=8).score("GGGAAAUCC")``."""

    def __init__(self, q: int = 8, pair_mask: int = FOLD_PAIRS_DEFAULT, device: int = 0, method: str = "two_vector"):
        self.ctx = fold_init(q, pair_mask, device)
        self.set_method(method)

    def set_method(self, method: str) -> None:
        fold_set_option(self.ctx, FOLD_OPT_METHOD,
                        {"two_vector": FOLD_METHOD_TWO_VECTOR, "plain": FOLD_METHOD_PLAIN,
                         "sliding": FOLD_METHOD_SLIDING, "fg": FOLD_METHOD_FG}[method])

    @property
    def q(self) -> int:
        return fold_get_option(self.ctx, FOLD_OPT_Q)

    @property
    def tile(self) -> int:
        return fold_get_option(self.ctx, FOLD_OPT_TILE)

    @property
    def launches(self) -> int:
        return fold_get_option(self.ctx, FOLD_OPT_LAUNCHES)

    def option(self, opt: int, value: int | None = None):
        if value is None:
            return fold_get_option(self.ctx, opt)
        fold_set_option(self.ctx, opt, value)

    def rtable(self) -> np.ndarray:
        return fold_rtable(self.ctx)

    def score(self, seq: str, want_D: bool = False):
        return fold_score(self.ctx, seq, want_D)

    def batch(self, seqs, want_D: bool = False):
        return fold_batch(self.ctx, seqs, want_D)

    def structure(self, seq: str):
        """(max pairs, partner array, dot-bracket) of one optimal structure."""
        return fold_structure(self.ctx, seq)

    def tune(self, n: int, reps: int = 3) -> dict:
        return fold_tune(self.ctx, n, reps)

    def workspace_bytes(self, n: int) -> int:
        return fold_workspace_bytes(self.ctx, n)

    def score_dev(self, codes, ws, out, D_out=None, stream=None) -> None:
        """codes: uint8 CUDA tensor of codes 0..3; ws: uint8 CUDA tensor of
        workspace_bytes(n); out: int32 CUDA tensor (1 element)."""
        n = int(codes.numel())
        fold_score_dev(self.ctx, codes.data_ptr() if n else None, n, ws.data_ptr(), ws.numel(), out.data_ptr(),
                       D_out.data_ptr() if D_out is not None else None, stream)

    def close(self) -> None:
        if self.ctx:
            fold_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode_codes(seq: str) -> np.ndarray:
    """Base letters to codes 0..3 for the device entry points, by the library's fold_encode
    (raises FoldError with FOLD_EINVAL on other letters)."""
    raw = seq.encode("ascii", errors="replace")
    out = np.empty(len(raw), dtype=np.uint8)
    _check(lib().fold_encode(raw, len(raw), out.ctypes.data if len(raw) else None), "fold_encode")
    return out
