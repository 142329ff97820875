"""CPU oracle of the LWE-style PIR path (plain C, loaded through ctypes).

TEST INFRASTRUCTURE ONLY.  The tests, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` are the only callers; the product package never
imports this module, and this module imports nothing from the product.

Each function is the plain definition of one step (see qpadl_oracle.c for the
passages of arxiv 2510.03631 it follows and the readings taken where the paper
is silent).  Arrays are numpy; all arithmetic is uint32 with wraparound.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qpadl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libqpadl_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over independent rows only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # QPADL_ORACLE_LIB names an alternative build of qpadl_oracle.c: the
            # mutation tests load deliberately broken copies through it to show
            # that the pins catch each planted mistake
            lib = ctypes.CDLL(os.environ.get("QPADL_ORACLE_LIB") or build())
            u64, i32, u32 = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
            P = ctypes.c_void_p
            lib.oracle_splitmix64.argtypes = [u64, u64]
            lib.oracle_splitmix64.restype = u64
            lib.oracle_gen_a.argtypes = [u64, u64, u64, P]
            lib.oracle_hint.argtypes = [P, u64, u64, P, u64, P, i32]
            lib.oracle_query.argtypes = [P, u64, u64, P, P, u64, u32, P]
            lib.oracle_answer.argtypes = [P, u64, u64, P, P, i32]
            lib.oracle_answer_batch.argtypes = [P, u64, u64, P, u64, P, i32]
            lib.oracle_recover.argtypes = [P, P, u64, u64, P, u32, P]
            lib.oracle_chor_answer.argtypes = [P, u64, u64, P, u64, u64, P, i32]
            lib.oracle_chor_query.argtypes = [P, u64, u64, u64, P]
            lib.oracle_chor_reconstruct.argtypes = [P, u64, u64, P]
            lib.oracle_goldberg_answer.argtypes = [P, u64, u64, P, u64, u32, P, i32]
            lib.oracle_delta_width.argtypes = [P, u64, u64]
            lib.oracle_delta_width.restype = u32
            lib.oracle_delta_encode.argtypes = [P, u64, u64, u32, P]
            lib.oracle_delta_decode.argtypes = [P, u64, u32, P]
            lib.oracle_goldberg_query.argtypes = [P, u64, u64, u64, P, u64, u32, P]
            lib.oracle_goldberg_reconstruct.argtypes = [P, P, u64, u64, u32, P]
            lib.oracle_max_threads.restype = i32
            for f in ("oracle_gen_a", "oracle_hint", "oracle_query", "oracle_answer",
                      "oracle_answer_batch", "oracle_recover", "oracle_chor_answer", "oracle_chor_query",
                      "oracle_chor_reconstruct", "oracle_goldberg_answer", "oracle_goldberg_query",
                      "oracle_goldberg_reconstruct"):
                getattr(lib, f).restype = None
            _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != dtype:
        raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
    return a


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def splitmix64(seed: int, i: int) -> int:
    """Output number i of SplitMix64 started from state `seed`."""
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), i))


def gen_a(seed: int, cols: int, n: int) -> np.ndarray:
    """Setup: public matrix A (cols x n, uint32) from its seed."""
    A = np.empty((cols, n), dtype=np.uint32)
    _load().oracle_gen_a(seed & (2**64 - 1), cols, n, _p(A))
    return A


def hint(D: np.ndarray, A: np.ndarray, threads: int = 1) -> np.ndarray:
    """Offline hint H = D * A mod 2^32 (R x n)."""
    D = _c(D, np.uint8)
    A = _c(A, np.uint32)
    R, C = D.shape
    if A.shape[0] != C:
        raise ValueError("A must have C rows")
    n = A.shape[1]
    H = np.empty((R, n), dtype=np.uint32)
    _load().oracle_hint(_p(D), R, C, _p(A), n, _p(H), threads)
    return H


def query(A: np.ndarray, s: np.ndarray, e: np.ndarray, col: int, delta: int) -> np.ndarray:
    """Client query qu = A s + e + delta * u_col mod 2^32 (length C)."""
    A = _c(A, np.uint32)
    s = _c(s, np.uint32)
    e = _c(e, np.int32)
    C, n = A.shape
    if s.shape != (n,) or e.shape != (C,):
        raise ValueError("shape mismatch")
    qu = np.empty(C, dtype=np.uint32)
    _load().oracle_query(_p(A), C, n, _p(s), _p(e), col, delta & 0xFFFFFFFF, _p(qu))
    return qu


def answer(D: np.ndarray, qu: np.ndarray, threads: int = 1) -> np.ndarray:
    """Server response ans = D * qu mod 2^32 (length R)."""
    D = _c(D, np.uint8)
    qu = _c(qu, np.uint32)
    R, C = D.shape
    if qu.shape != (C,):
        raise ValueError("query length must equal C")
    ans = np.empty(R, dtype=np.uint32)
    _load().oracle_answer(_p(D), R, C, _p(qu), _p(ans), threads)
    return ans


def answer_batch(D: np.ndarray, Q: np.ndarray, threads: int = 1) -> np.ndarray:
    """Batched responses: Q is B x C (query b in row b); returns B x R."""
    D = _c(D, np.uint8)
    Q = _c(Q, np.uint32)
    R, C = D.shape
    B = Q.shape[0]
    if Q.shape != (B, C):
        raise ValueError("Q must be B x C")
    ans = np.empty((B, R), dtype=np.uint32)
    _load().oracle_answer_batch(_p(D), R, C, _p(Q), B, _p(ans), threads)
    return ans


def recover(ans: np.ndarray, H: np.ndarray, s: np.ndarray, p: int = 256) -> np.ndarray:
    """Client recovery of the queried column: R digits in [0, p)."""
    ans = _c(ans, np.uint32)
    H = _c(H, np.uint32)
    s = _c(s, np.uint32)
    R, n = H.shape
    if ans.shape != (R,) or s.shape != (n,):
        raise ValueError("shape mismatch")
    lp = int(p).bit_length() - 1
    if p < 2 or p > 256 or (1 << lp) != p:
        raise ValueError("p must be a power of two in [2, 256]")
    out = np.empty(R, dtype=np.uint8)
    _load().oracle_recover(_p(ans), _p(H), R, n, _p(s), lp, _p(out))
    return out


def delta_for(p: int) -> int:
    """Scale Delta = q / p with q = 2^32."""
    return (1 << 32) // p


def chor_answer(DB: np.ndarray, r: int, Q: np.ndarray, threads: int = 1) -> np.ndarray:
    """Chor Response over GF(2): DB is r x w uint32 words (r rows of 32 w bits),
    Q is B x qw words (qw = ceil(r / 32), bit i of query b = row i selected);
    returns B x w words, the XOR of the selected rows for each query."""
    DB = _c(DB, np.uint32)
    Q = _c(Q, np.uint32)
    if DB.ndim != 2 or DB.shape[0] != r:
        raise ValueError("DB must be r x w words")
    w = DB.shape[1]
    qw = (r + 31) // 32
    if Q.ndim != 2 or Q.shape[1] != qw:
        raise ValueError("Q must be B x ceil(r/32) words")
    B = Q.shape[0]
    out = np.empty((B, w), dtype=np.uint32)
    _load().oracle_chor_answer(_p(DB), r, w, _p(Q), qw, B, _p(out), threads)
    return out


def chor_query(shares: np.ndarray, theta: int) -> np.ndarray:
    """ENS client query: (ell-1) x qw random words -> ell x qw query words, the
    last being the XOR of the others with the unit vector at theta."""
    shares = _c(shares, np.uint32)
    ell = shares.shape[0] + 1
    qw = shares.shape[1]
    if not 0 <= theta < 32 * qw:
        raise ValueError("theta out of range")
    out = np.empty((ell, qw), dtype=np.uint32)
    _load().oracle_chor_query(_p(shares), ell, qw, theta, _p(out))
    return out


def chor_reconstruct(responses: np.ndarray) -> np.ndarray:
    """ENS reconstruction: XOR of the ell responses (ell x w words)."""
    responses = _c(responses, np.uint32)
    ell, w = responses.shape
    out = np.empty(w, dtype=np.uint32)
    _load().oracle_chor_reconstruct(_p(responses), ell, w, _p(out))
    return out


def goldberg_answer(D: np.ndarray, Q: np.ndarray, p: int, threads: int = 1) -> np.ndarray:
    """Goldberg Response over Z_p: D is R x C bytes (record j = column j), Q is
    B x C field elements (uint32 < p); returns B x R, rho = D q mod p."""
    D = _c(D, np.uint8)
    Q = _c(np.atleast_2d(Q), np.uint32)
    R, C = D.shape
    B = Q.shape[0]
    if Q.shape != (B, C):
        raise ValueError("Q must be B x C")
    out = np.empty((B, R), dtype=np.uint32)
    _load().oracle_goldberg_answer(_p(D), R, C, _p(Q), B, p, _p(out), threads)
    return out


def goldberg_query(coef: np.ndarray, theta: int, alpha: np.ndarray, p: int) -> np.ndarray:
    """FTR client: coef is C x t (the non-constant coefficients of the C
    polynomials); returns ell x C queries, query k = the polynomials at alpha[k]."""
    coef = _c(coef, np.uint32)
    alpha = _c(alpha, np.uint32)
    C, t = coef.shape
    ell = alpha.shape[0]
    out = np.empty((ell, C), dtype=np.uint32)
    _load().oracle_goldberg_query(_p(coef), C, t, theta, _p(alpha), ell, p, _p(out))
    return out


def goldberg_reconstruct(responses: np.ndarray, alpha: np.ndarray, p: int) -> np.ndarray:
    """Lagrange interpolation at 0 of k responses (k x R) at the points alpha (k)."""
    responses = _c(responses, np.uint32)
    alpha = _c(alpha, np.uint32)
    k, R = responses.shape
    out = np.empty(R, dtype=np.uint32)
    _load().oracle_goldberg_reconstruct(_p(responses), _p(alpha), k, R, p, _p(out))
    return out


def delta_width(x: np.ndarray, E: int) -> int:
    """Bytes per stored difference for entries x grouped in blocks of E (Sec. 5.3)."""
    x = _c(x, np.uint32)
    if x.ndim != 1 or x.size == 0 or E < 1:
        raise ValueError("x: non-empty 1-D entries; E >= 1")
    return int(_load().oracle_delta_width(_p(x), x.size, E))


def delta_encode(x: np.ndarray, E: int, w: int) -> np.ndarray:
    """Compressed database (R' x C digits, record j = column j) of entries x (Sec. 5.3)."""
    x = _c(x, np.uint32)
    if x.ndim != 1 or x.size == 0 or E < 1 or not 1 <= w <= 4:
        raise ValueError("x: non-empty 1-D entries; E >= 1; w in 1..4")
    C = (x.size + E - 1) // E
    db = np.empty((4 + w * (E - 1), C), dtype=np.uint8)
    _load().oracle_delta_encode(_p(x), x.size, E, w, _p(db))
    return db


def delta_decode(digits: np.ndarray, E: int, w: int) -> np.ndarray:
    """The E entries of one block from its R' = 4 + w (E - 1) digits (Sec. 5.3)."""
    digits = _c(digits, np.uint8)
    if digits.shape != (4 + w * (E - 1),):
        raise ValueError("digits: one block of 4 + w (E - 1) digits")
    out = np.empty(E, dtype=np.uint32)
    _load().oracle_delta_decode(_p(digits), E, w, _p(out))
    return out
