"""Thin Python binding of the C ABI in include/qpadl_pir.h (argument marshalling only).

Every function here has the name of the C entry point it calls, takes torch
tensors (device tensors for *_dev arguments, CPU tensors for *_host ones),
checks dtype/shape/device, passes raw pointers and the current CUDA stream,
and raises QpadlError on a non-zero status.  All arithmetic runs in the CUDA
library; there is no CPU fallback: if the library cannot be loaded every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

QPADL_OK = 0
QPADL_EINVAL = -1
QPADL_ENOMEM = -2
QPADL_ECUDA = -3
QPADL_ETIMEOUT = -4
QPADL_EBUSY = -5
QPADL_EAGAIN = -6
QPADL_SETUP_TENSOR_COPY = 0x1
QPADL_OPT_STREAM_CHUNK = 1
QPADL_OPT_TENSOR_MIN_BATCH = 2
QPADL_OPT_STREAM_RAW = 3
QPADL_OPT_U8_MAX_BATCH = 4
QPADL_OPT_U8_KSTEP = 5
QPADL_OPT_PAIR_GEMM = 6


class QpadlError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class qpadl_params(ctypes.Structure):
    _fields_ = [
        ("rows", ctypes.c_uint64),
        ("cols", ctypes.c_uint64),
        ("n", ctypes.c_uint32),
        ("log_q", ctypes.c_uint32),
        ("p", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("sigma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def params(rows: int, cols: int, n: int, p: int = 256, sigma: float = 6.4, seed: int = 1,
           flags: int = 0) -> qpadl_params:
    return qpadl_params(rows, cols, n, 32, p, flags, sigma, seed & (2**64 - 1))


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_SIGS = {
    "qpadl_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "qpadl_version": ([], ctypes.c_int),
    "qpadl_pir_setup": ([_P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "qpadl_pir_destroy": ([_P], ctypes.c_int),
    "qpadl_pir_status": ([_P], ctypes.c_int),
    "qpadl_pir_device_bytes": ([_P], ctypes.c_uint64),
    "qpadl_pir_set_option": ([_P, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "qpadl_pir_get_option": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "qpadl_pir_gen_a": ([_P, _P, _P], ctypes.c_int),
    "qpadl_pir_hint": ([_P, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_query": ([_P, _P, _P, _P, ctypes.c_uint64, _P, _P], ctypes.c_int),
    "qpadl_pir_query_batch": ([_P, _P, _P, _P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_pir_answer": ([_P, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_answer_batch": ([_P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_pir_answer_batch_path": ([_P, _P, ctypes.c_uint32, _P, ctypes.c_int, _P], ctypes.c_int),
    "qpadl_pir_answer_host": ([_P, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_answer_noalloc": ([_P, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_noalloc_status": ([], ctypes.c_int),
    "qpadl_pir_recover": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_shape": ([_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qpadl_pir_reserve": ([_P, ctypes.c_uint32, _P], ctypes.c_int),
    "qpadl_pir_shard_rows": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qpadl_client_create": ([_P, _P, _P, ctypes.c_uint32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "qpadl_client_query_batch": ([_P, _P, _P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_client_recover_batch": ([_P, _P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_client_status": ([_P], ctypes.c_int),
    "qpadl_client_device_bytes": ([_P], ctypes.c_uint64),
    "qpadl_client_set_option": ([_P, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "qpadl_client_destroy": ([_P], ctypes.c_int),
    "qpadl_goldberg_setup": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P, ctypes.POINTER(_P)],
                             ctypes.c_int),
    "qpadl_goldberg_answer_batch": ([_P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_goldberg_set_option": ([_P, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "qpadl_goldberg_status": ([_P], ctypes.c_int),
    "qpadl_goldberg_destroy": ([_P], ctypes.c_int),
    "qpadl_chor_setup": ([ctypes.c_uint64, ctypes.c_uint64, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "qpadl_chor_answer_batch": ([_P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_chor_status": ([_P], ctypes.c_int),
    "qpadl_chor_set_option": ([_P, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "qpadl_chor_get_option": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "qpadl_chor_destroy": ([_P], ctypes.c_int),
    "qpadl_pir_autotune": ([_P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_selftest_bounded_wait": ([ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "qpadl_server_create": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "qpadl_server_add_db": ([_P, _P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qpadl_server_start": ([_P], ctypes.c_int),
    "qpadl_server_submit": ([_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qpadl_server_poll": ([_P, ctypes.c_uint64, _P, _P], ctypes.c_int),
    "qpadl_server_stats": ([_P, _P], ctypes.c_int),
    "qpadl_server_destroy": ([_P], ctypes.c_int),
    "qpadl_server_replay": ([_P, ctypes.c_uint64, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "qpadl_pir_recover_batch": ([_P, _P, _P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_pir_client_status": ([], ctypes.c_int),
    "qpadl_pir_delta_width": ([_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), _P], ctypes.c_int),
    "qpadl_pir_delta_encode": ([_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "qpadl_pir_delta_decode": ([_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _P, _P], ctypes.c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqpadl_pir.so (building it first if asked); raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (argt, rest) in _SIGS.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = argt
                fn.restype = rest
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    try:
        return load(build_if_missing=False).qpadl_strerror(code).decode()
    except Exception:
        return {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error",
                -4: "device wait timed out", -5: "busy", -6: "not ready"}.get(code, "unknown error")


def _check(rc: int, what: str):
    if rc != QPADL_OK:
        raise QpadlError(rc, what)


def _dev(t: torch.Tensor, dtype: torch.dtype, numel: int, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _host(t: torch.Tensor, dtype: torch.dtype, numel: int, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name}: need contiguous {dtype} with >= {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Database:
    """Handle returned by qpadl_pir_setup (owns the C handle, keeps D alive)."""

    def __init__(self, handle: ctypes.c_void_p, prm: qpadl_params, db: torch.Tensor):
        self.handle = handle
        self.prm = prm
        self.db = db

    @property
    def rows(self) -> int:
        return int(self.prm.rows)

    @property
    def cols(self) -> int:
        return int(self.prm.cols)

    def close(self):
        if self.handle:
            load().qpadl_pir_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qpadl_version() -> int:
    return int(load().qpadl_version())


def qpadl_pir_setup(prm: qpadl_params, db: torch.Tensor, stream=None) -> Database:
    _dev(db, torch.uint8, int(prm.rows) * int(prm.cols), "db")
    h = ctypes.c_void_p()
    _check(load().qpadl_pir_setup(ctypes.byref(prm), ctypes.c_void_p(db.data_ptr()), _stream(stream),
                                  ctypes.byref(h)), "qpadl_pir_setup")
    return Database(h, prm, db)


def qpadl_pir_destroy(db: Database):
    db.close()


def qpadl_pir_status(db: Database) -> int:
    return int(load().qpadl_pir_status(db.handle))


def qpadl_pir_device_bytes(db: Database) -> int:
    return int(load().qpadl_pir_device_bytes(db.handle))


def qpadl_pir_set_option(db: Database, option: int, value: int):
    _check(load().qpadl_pir_set_option(db.handle, int(option), int(value)), "qpadl_pir_set_option")


def qpadl_pir_get_option(db: Database, option: int) -> int:
    v = ctypes.c_int64()
    _check(load().qpadl_pir_get_option(db.handle, int(option), ctypes.byref(v)), "qpadl_pir_get_option")
    return int(v.value)


def qpadl_pir_gen_a(prm: qpadl_params, A: torch.Tensor, stream=None) -> torch.Tensor:
    p = _dev(A, torch.int32, int(prm.cols) * int(prm.n), "A")
    _check(load().qpadl_pir_gen_a(ctypes.byref(prm), p, _stream(stream)), "qpadl_pir_gen_a")
    return A


def qpadl_pir_hint(db: Database, A: torch.Tensor, H: torch.Tensor, stream=None) -> torch.Tensor:
    n = int(db.prm.n)
    pa = _dev(A, torch.int32, db.cols * n, "A")
    ph = _dev(H, torch.int32, db.rows * n, "H")
    _check(load().qpadl_pir_hint(db.handle, pa, ph, _stream(stream)), "qpadl_pir_hint")
    return H


def qpadl_pir_query(prm: qpadl_params, A: torch.Tensor, s: torch.Tensor, e: torch.Tensor, col: int,
                    q: torch.Tensor, stream=None) -> torch.Tensor:
    C, n = int(prm.cols), int(prm.n)
    args = (_dev(A, torch.int32, C * n, "A"), _dev(s, torch.int32, n, "s"), _dev(e, torch.int32, C, "e"))
    _check(load().qpadl_pir_query(ctypes.byref(prm), *args, int(col), _dev(q, torch.int32, C, "q"),
                                  _stream(stream)), "qpadl_pir_query")
    return q


def qpadl_pir_query_batch(prm: qpadl_params, A: torch.Tensor, S: torch.Tensor, E: torch.Tensor,
                          cols: torch.Tensor, Q: torch.Tensor, stream=None) -> torch.Tensor:
    C, n = int(prm.cols), int(prm.n)
    B = int(cols.numel())
    _check(load().qpadl_pir_query_batch(
        ctypes.byref(prm), _dev(A, torch.int32, C * n, "A"), _dev(S, torch.int32, B * n, "S"),
        _dev(E, torch.int32, B * C, "E"), _dev(cols, torch.int32, B, "cols"), B,
        _dev(Q, torch.int32, B * C, "Q"), _stream(stream)), "qpadl_pir_query_batch")
    return Q


def qpadl_pir_answer(db: Database, q: torch.Tensor, ans: torch.Tensor, stream=None) -> torch.Tensor:
    _check(load().qpadl_pir_answer(db.handle, _dev(q, torch.int32, db.cols, "q"),
                                   _dev(ans, torch.int32, db.rows, "ans"), _stream(stream)),
           "qpadl_pir_answer")
    return ans


def qpadl_pir_answer_batch(db: Database, Q: torch.Tensor, ans: torch.Tensor, stream=None,
                           path: int | None = None) -> torch.Tensor:
    B = Q.numel() // db.cols
    if B * db.cols != Q.numel() or B == 0:
        raise ValueError("Q must hold B x C words")
    pq = _dev(Q, torch.int32, B * db.cols, "Q")
    pa = _dev(ans, torch.int32, B * db.rows, "ans")
    if path is None:
        rc = load().qpadl_pir_answer_batch(db.handle, pq, B, pa, _stream(stream))
    else:
        rc = load().qpadl_pir_answer_batch_path(db.handle, pq, B, pa, int(path), _stream(stream))
    _check(rc, "qpadl_pir_answer_batch")
    return ans


def qpadl_pir_answer_host(db: Database, q: torch.Tensor, ans: torch.Tensor, stream=None) -> torch.Tensor:
    _check(load().qpadl_pir_answer_host(db.handle, _host(q, torch.int32, db.cols, "q"),
                                        _host(ans, torch.int32, db.rows, "ans"), _stream(stream)),
           "qpadl_pir_answer_host")
    return ans


def qpadl_pir_answer_noalloc(db: torch.Tensor, rows: int, cols: int, q: torch.Tensor, ans: torch.Tensor,
                             stream=None) -> torch.Tensor:
    """Allocation-free single-query Response on a caller-resident database (no handle)."""
    _check(load().qpadl_pir_answer_noalloc(_dev(db, torch.uint8, rows * cols, "db"), rows, cols,
                                           _dev(q, torch.int32, cols, "q"), _dev(ans, torch.int32, rows, "ans"),
                                           _stream(stream)), "qpadl_pir_answer_noalloc")
    return ans


def qpadl_pir_noalloc_status() -> int:
    """Waits for the current device; returns and clears the status word of the
    allocation-free Response (QPADL_OK or QPADL_ETIMEOUT)."""
    return int(load().qpadl_pir_noalloc_status())


def qpadl_pir_recover(prm: qpadl_params, ans: torch.Tensor, H: torch.Tensor, s: torch.Tensor,
                      out: torch.Tensor, stream=None) -> torch.Tensor:
    R, n = int(prm.rows), int(prm.n)
    _check(load().qpadl_pir_recover(
        ctypes.byref(prm), _dev(ans, torch.int32, R, "ans"), _dev(H, torch.int32, R * n, "H"),
        _dev(s, torch.int32, n, "s"), _dev(out, torch.uint8, R, "out"), _stream(stream)), "qpadl_pir_recover")
    return out


def qpadl_pir_recover_batch(prm: qpadl_params, ans: torch.Tensor, H: torch.Tensor, S: torch.Tensor,
                            out: torch.Tensor, stream=None) -> torch.Tensor:
    R, n = int(prm.rows), int(prm.n)
    B = S.numel() // n
    _check(load().qpadl_pir_recover_batch(
        ctypes.byref(prm), _dev(ans, torch.int32, B * R, "ans"), _dev(H, torch.int32, R * n, "H"),
        _dev(S, torch.int32, B * n, "S"), B, _dev(out, torch.uint8, B * R, "out"), _stream(stream)),
        "qpadl_pir_recover_batch")
    return out


def delta_rows(E: int, w: int) -> int:
    """Rows R' = 4 + w (E - 1) of a compressed database (Sec. 5.3)."""
    return 4 + w * (E - 1)


def qpadl_pir_delta_width(entries: torch.Tensor, E: int, stream=None) -> int:
    """Bytes per stored difference for the entries in blocks of E (synchronises the stream)."""
    w = ctypes.c_uint32(0)
    _check(load().qpadl_pir_delta_width(_dev(entries, torch.int32, entries.numel(), "entries"), entries.numel(), E,
                                        ctypes.byref(w), _stream(stream)), "qpadl_pir_delta_width")
    return int(w.value)


def qpadl_pir_delta_encode(entries: torch.Tensor, E: int, w: int, db: torch.Tensor, stream=None) -> torch.Tensor:
    """Compressed database (R' x C uint8 digits) of the entries (Sec. 5.3)."""
    n = entries.numel()
    C = (n + E - 1) // E
    _check(load().qpadl_pir_delta_encode(_dev(entries, torch.int32, n, "entries"), n, E, w,
                                         _dev(db, torch.uint8, delta_rows(E, w) * C, "db"), _stream(stream)),
           "qpadl_pir_delta_encode")
    return db


def qpadl_pir_delta_decode(digits: torch.Tensor, B: int, E: int, w: int, out: torch.Tensor,
                           stream=None) -> torch.Tensor:
    """Entries (B x E) of B recovered blocks (B x R' digits)."""
    _check(load().qpadl_pir_delta_decode(_dev(digits, torch.uint8, B * delta_rows(E, w), "digits"), B, E, w,
                                         _dev(out, torch.int32, B * E, "out"), _stream(stream)),
           "qpadl_pir_delta_decode")
    return out


def qpadl_pir_client_status() -> int:
    """Waits for the current device; returns and clears the status word of the
    handle-free Query/Recover kernels (QPADL_OK or QPADL_ETIMEOUT)."""
    return int(load().qpadl_pir_client_status())


class Client:
    """Handle returned by qpadl_client_create (owns the C context)."""

    def __init__(self, handle: ctypes.c_void_p, prm: qpadl_params, has_hint: bool):
        self.handle = handle
        self.prm = prm
        self.has_hint = has_hint

    def close(self):
        if self.handle:
            load().qpadl_client_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qpadl_client_create(prm: qpadl_params, A: torch.Tensor, H: torch.Tensor | None = None, max_batch: int = 1024,
                        stream=None) -> Client:
    C, R, n = int(prm.cols), int(prm.rows), int(prm.n)
    pa = _dev(A, torch.int32, C * n, "A")
    ph = _dev(H, torch.int32, R * n, "H") if H is not None else None
    h = ctypes.c_void_p()
    _check(load().qpadl_client_create(ctypes.byref(prm), pa, ph, int(max_batch), _stream(stream), ctypes.byref(h)),
           "qpadl_client_create")
    return Client(h, prm, H is not None)


def qpadl_client_query_batch(c: Client, S: torch.Tensor, E: torch.Tensor, cols: torch.Tensor, Q: torch.Tensor,
                             stream=None) -> torch.Tensor:
    C, n = int(c.prm.cols), int(c.prm.n)
    B = int(cols.numel())
    _check(load().qpadl_client_query_batch(
        c.handle, _dev(S, torch.int32, B * n, "S"), _dev(E, torch.int32, B * C, "E"),
        _dev(cols, torch.int32, B, "cols"), B, _dev(Q, torch.int32, B * C, "Q"), _stream(stream)),
        "qpadl_client_query_batch")
    return Q


def qpadl_client_recover_batch(c: Client, ans: torch.Tensor, S: torch.Tensor, out: torch.Tensor,
                               stream=None) -> torch.Tensor:
    R, n = int(c.prm.rows), int(c.prm.n)
    B = S.numel() // n
    _check(load().qpadl_client_recover_batch(
        c.handle, _dev(ans, torch.int32, B * R, "ans"), _dev(S, torch.int32, B * n, "S"), B,
        _dev(out, torch.uint8, B * R, "out"), _stream(stream)), "qpadl_client_recover_batch")
    return out


def qpadl_client_status(c: Client) -> int:
    return int(load().qpadl_client_status(c.handle))


QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS = 1
QPADL_CLIENT_OPT_PAIR_GEMM = 2


def qpadl_client_set_option(c: Client, option: int, value: int):
    _check(load().qpadl_client_set_option(c.handle, int(option), int(value)), "qpadl_client_set_option")


def qpadl_client_device_bytes(c: Client) -> int:
    return int(load().qpadl_client_device_bytes(c.handle))


class GoldbergDatabase:
    """Handle returned by qpadl_goldberg_setup (owns the C handle, keeps the database alive)."""

    def __init__(self, handle: ctypes.c_void_p, rows: int, cols: int, p: int, db: torch.Tensor):
        self.handle = handle
        self.rows = rows
        self.cols = cols
        self.p = p
        self.db = db

    def close(self):
        if self.handle:
            load().qpadl_goldberg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


QPADL_GOLDBERG_OPT_GEMM_MIN_BATCH = 1
QPADL_GOLDBERG_OPT_U8_MAX_BATCH = 2
QPADL_GOLDBERG_OPT_PAIR_GEMM = 3


def qpadl_goldberg_setup(rows: int, cols: int, p: int, db: torch.Tensor, stream=None) -> GoldbergDatabase:
    """db: rows x cols uint8 field elements (record j = column j)."""
    pd = _dev(db, torch.uint8, int(rows) * int(cols), "db")
    h = ctypes.c_void_p()
    _check(load().qpadl_goldberg_setup(int(rows), int(cols), int(p), pd, _stream(stream), ctypes.byref(h)),
           "qpadl_goldberg_setup")
    return GoldbergDatabase(h, int(rows), int(cols), int(p), db)


def qpadl_goldberg_answer_batch(h: GoldbergDatabase, Q: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Q: B x cols int32 field elements; out: B x rows int32."""
    B = Q.numel() // h.cols
    if B * h.cols != Q.numel() or B == 0:
        raise ValueError("Q must hold B x cols elements")
    _check(load().qpadl_goldberg_answer_batch(h.handle, _dev(Q, torch.int32, B * h.cols, "Q"), B,
                                              _dev(out, torch.int32, B * h.rows, "out"), _stream(stream)),
           "qpadl_goldberg_answer_batch")
    return out


def qpadl_goldberg_set_option(h: GoldbergDatabase, option: int, value: int):
    _check(load().qpadl_goldberg_set_option(h.handle, int(option), int(value)), "qpadl_goldberg_set_option")


def qpadl_goldberg_status(h: GoldbergDatabase) -> int:
    return int(load().qpadl_goldberg_status(h.handle))


class ChorDatabase:
    """Handle returned by qpadl_chor_setup (owns the C handle, keeps the database alive)."""

    def __init__(self, handle: ctypes.c_void_p, rows: int, bits: int, db: torch.Tensor):
        self.handle = handle
        self.rows = rows
        self.bits = bits
        self.db = db

    @property
    def words(self) -> int:
        return self.bits // 32

    @property
    def query_words(self) -> int:
        return (self.rows + 31) // 32

    def close(self):
        if self.handle:
            load().qpadl_chor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qpadl_chor_setup(rows: int, bits: int, db: torch.Tensor, stream=None) -> ChorDatabase:
    """db: rows x bits/32 int32 words (bit c of record i = bit c % 32 of word c / 32)."""
    pd = _dev(db, torch.int32, int(rows) * (int(bits) // 32), "db")
    h = ctypes.c_void_p()
    _check(load().qpadl_chor_setup(int(rows), int(bits), pd, _stream(stream), ctypes.byref(h)), "qpadl_chor_setup")
    return ChorDatabase(h, int(rows), int(bits), db)


def qpadl_chor_answer_batch(h: ChorDatabase, Q: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Q: B x ceil(rows/32) int32 words; out: B x bits/32 int32 words."""
    B = Q.numel() // h.query_words
    if B * h.query_words != Q.numel() or B == 0:
        raise ValueError("Q must hold B x ceil(rows/32) words")
    _check(load().qpadl_chor_answer_batch(h.handle, _dev(Q, torch.int32, B * h.query_words, "Q"), B,
                                          _dev(out, torch.int32, B * h.words, "out"), _stream(stream)),
           "qpadl_chor_answer_batch")
    return out


QPADL_CHOR_OPT_M4RM_MIN_BATCH = 1
QPADL_CHOR_OPT_SCAN_FORM = 2


def qpadl_chor_set_option(h: ChorDatabase, option: int, value: int):
    _check(load().qpadl_chor_set_option(h.handle, int(option), int(value)), "qpadl_chor_set_option")


def qpadl_chor_get_option(h: ChorDatabase, option: int) -> int:
    v = ctypes.c_int64()
    _check(load().qpadl_chor_get_option(h.handle, int(option), ctypes.byref(v)), "qpadl_chor_get_option")
    return int(v.value)


def qpadl_chor_status(h: ChorDatabase) -> int:
    return int(load().qpadl_chor_status(h.handle))


def as_u32(t: torch.Tensor):
    """View an int32 torch tensor's bits as numpy uint32 (host copy)."""
    return t.detach().cpu().numpy().view("uint32")


def from_u32(a, device="cuda") -> torch.Tensor:
    """numpy uint32 -> int32 torch tensor with the same bits."""
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(device)


# ----------------------------------------------------------------------------- serving
class qpadl_server_config(ctypes.Structure):
    _fields_ = [
        ("host_budget_bytes", ctypes.c_uint64),
        ("device_budget_bytes", ctypes.c_uint64),
        ("max_inflight", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint32),
        ("num_streams", ctypes.c_uint32),
        ("test_drop_completion_launch", ctypes.c_uint32),
        ("hold_us", ctypes.c_double),
        ("watchdog_ms", ctypes.c_double),
        ("group_size_ratio", ctypes.c_double),
    ]


class qpadl_request_times(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("launch_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class qpadl_server_stats_t(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
        ("refused", ctypes.c_uint64), ("inflight", ctypes.c_uint32), ("queued", ctypes.c_uint32),
        ("mean_launch_requests", ctypes.c_double), ("host_bytes_used", ctypes.c_uint64),
        ("device_bytes_used", ctypes.c_uint64), ("grouped_launches", ctypes.c_uint64),
        ("mean_enqueue_us", ctypes.c_double), ("stream_kernels", ctypes.c_uint64),
        ("gemm_kernels", ctypes.c_uint64),
    ]


def server_config(host_budget_bytes=1 << 30, device_budget_bytes=1 << 30, max_inflight=4096, max_batch=256,
                  num_streams=4, hold_us=0.0, watchdog_ms=10000.0, test_drop_completion_launch=0,
                  group_size_ratio=2.0):
    return qpadl_server_config(host_budget_bytes, device_budget_bytes, max_inflight, max_batch, num_streams,
                               test_drop_completion_launch, hold_us, watchdog_ms, group_size_ratio)


def qpadl_pir_shape(db: Database):
    r, c = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().qpadl_pir_shape(db.handle, ctypes.byref(r), ctypes.byref(c)), "qpadl_pir_shape")
    return int(r.value), int(c.value)


def qpadl_pir_shard_rows(rows: int, world: int, rank: int):
    """Rows [r0, r1) that rank `rank` of `world` holds (host only)."""
    r0, r1 = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().qpadl_pir_shard_rows(int(rows), int(world), int(rank), ctypes.byref(r0), ctypes.byref(r1)),
           "qpadl_pir_shard_rows")
    return int(r0.value), int(r1.value)


class qpadl_tune_report(ctypes.Structure):
    _fields_ = [
        ("single_ms", (ctypes.c_double * 2) * 3),
        ("u8_kstep_ms", ctypes.c_double * 2),
        ("stream_ms", ctypes.c_double * 3),
        ("tensor_ms", ctypes.c_double * 3),
        ("tuned_batch", ctypes.c_uint32),
        ("stream_chunk", ctypes.c_int32), ("stream_raw", ctypes.c_int32), ("u8_kstep", ctypes.c_int32),
        ("tensor_min_batch", ctypes.c_uint32),
        ("u8_vs_f16_ms", (ctypes.c_double * 2) * 2), ("u8_max_batch", ctypes.c_uint32),
    ]


def qpadl_pir_autotune(db: Database, max_batch: int, stream=None) -> dict:
    """Time the handle's exact-path choices on the device and keep the fastest; returns the report."""
    rep = qpadl_tune_report()
    _check(load().qpadl_pir_autotune(db.handle, int(max_batch), _stream(stream), ctypes.byref(rep)),
           "qpadl_pir_autotune")
    return {"single_ms": [[rep.single_ms[c][r] for r in range(2)] for c in range(3)],
            "u8_kstep_ms": list(rep.u8_kstep_ms), "stream_ms": list(rep.stream_ms), "tensor_ms": list(rep.tensor_ms),
            "tuned_batch": rep.tuned_batch, "stream_chunk": rep.stream_chunk, "stream_raw": rep.stream_raw,
            "u8_kstep": rep.u8_kstep, "tensor_min_batch": rep.tensor_min_batch,
            "u8_vs_f16_ms": [[rep.u8_vs_f16_ms[b][k] for k in range(2)] for b in range(2)],
            "u8_max_batch": rep.u8_max_batch}


def qpadl_pir_reserve(db: Database, max_batch: int, stream=None):
    _check(load().qpadl_pir_reserve(db.handle, int(max_batch), _stream(stream)), "qpadl_pir_reserve")


class Server:
    """Handle of a qpadl_server (keeps its databases alive)."""

    def __init__(self, handle, dbs):
        self.handle = handle
        self.dbs = dbs

    def close(self):
        if self.handle:
            load().qpadl_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qpadl_server_create(cfg: qpadl_server_config) -> Server:
    h = ctypes.c_void_p()
    _check(load().qpadl_server_create(ctypes.byref(cfg), ctypes.byref(h)), "qpadl_server_create")
    return Server(h, [])


def qpadl_server_add_db(srv: Server, db: Database) -> int:
    i = ctypes.c_int()
    _check(load().qpadl_server_add_db(srv.handle, db.handle, ctypes.byref(i)), "qpadl_server_add_db")
    srv.dbs.append(db)
    return int(i.value)


def qpadl_server_start(srv: Server):
    _check(load().qpadl_server_start(srv.handle), "qpadl_server_start")


def qpadl_server_submit(srv: Server, db_id: int, q_host) -> int:
    """Returns the ticket; raises QpadlError (code QPADL_EBUSY) when admission refuses.
    q_host: numpy uint32 array (C words)."""
    import numpy as np
    q = np.ascontiguousarray(q_host, dtype=np.uint32)
    t = ctypes.c_uint64()
    _check(load().qpadl_server_submit(srv.handle, int(db_id), ctypes.c_void_p(q.ctypes.data), ctypes.byref(t)),
           "qpadl_server_submit")
    return int(t.value)


def qpadl_server_poll(srv: Server, ticket: int, ans_host=None):
    """Returns (status, times); status QPADL_EAGAIN while pending.  ans_host: numpy uint32 (R words) or None."""
    tm = qpadl_request_times()
    p = ctypes.c_void_p(ans_host.ctypes.data) if ans_host is not None else None
    rc = load().qpadl_server_poll(srv.handle, ctypes.c_uint64(ticket), p, ctypes.byref(tm))
    return int(rc), (tm.submit_s, tm.launch_s, tm.done_s)


def qpadl_server_stats(srv: Server) -> dict:
    st = qpadl_server_stats_t()
    _check(load().qpadl_server_stats(srv.handle, ctypes.byref(st)), "qpadl_server_stats")
    return {f: getattr(st, f) for f, _ in qpadl_server_stats_t._fields_}


def qpadl_server_destroy(srv: Server):
    srv.close()


def qpadl_server_replay(srv: Server, arrival_s, db_ids, queries, answers=None, with_times: bool = False):
    """Open-loop replay (native): returns (latency_s, status) numpy arrays, plus an
    n x 3 array of (submit, launch, done) seconds after each scheduled arrival when
    with_times.  queries / answers: lists of numpy uint32 arrays (kept alive by the caller)."""
    import numpy as np
    n = len(arrival_s)
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    ids = np.ascontiguousarray(db_ids, dtype=np.int32)
    qp = (ctypes.c_void_p * n)(*[q.ctypes.data for q in queries])
    ap = (ctypes.c_void_p * n)(*[a.ctypes.data for a in answers]) if answers is not None else None
    lat = np.zeros(n, dtype=np.float64)
    st = np.zeros(n, dtype=np.int32)
    tm = np.zeros((n, 3), dtype=np.float64) if with_times else None
    _check(load().qpadl_server_replay(srv.handle, n, ctypes.c_void_p(arr.ctypes.data),
                                      ctypes.c_void_p(ids.ctypes.data), qp, ap, ctypes.c_void_p(lat.ctypes.data),
                                      ctypes.c_void_p(st.ctypes.data),
                                      ctypes.c_void_p(tm.ctypes.data) if with_times else None),
           "qpadl_server_replay")
    return (lat, st, tm) if with_times else (lat, st)


def qpadl_selftest_bounded_wait(arrive: bool, stream=None):
    """Run the library's bounded mbarrier wait on a barrier nothing arrives on (arrive=False)
    or on a completed one; returns (device status code, nanoseconds waited)."""
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check(load().qpadl_selftest_bounded_wait(1 if arrive else 0, ctypes.c_void_p(st.data_ptr()),
                                              ctypes.c_void_p(ns.data_ptr()), _stream(stream)),
           "qpadl_selftest_bounded_wait")
    torch.cuda.synchronize()
    return int(st.item()), int(ns.item())
