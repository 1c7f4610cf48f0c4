"""Plain CPU oracle for the heterogeneity-aware majority voter (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product path (the CUDA library
and its binding in ``paper_1405_2912_b300``) never imports it, and the two share
no source: this package wraps ``ref_vote.c`` (a scalar C loop, built with gcc)
through ctypes.

What the oracle computes is stated at the top of ``ref_vote.c``; it follows the
voter of Sec. IV.D of Kicherer & Karl (bit-wise comparison for integer types,
comparison within a programmer-set maximum difference for floating point) with
the readings listed there for what the paper leaves open.

All functions take and return numpy arrays in host memory.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ref_vote.c")
_LIB = os.path.join(_HERE, "libftref.so")
_lock = threading.Lock()
_lib = None

# Element-type codes shared by the C ABI of both libraries (an interface, not
# arithmetic): the integer values are part of the public header.
DTYPES = {"i32": 0, "u32": 1, "i64": 2, "u64": 3, "u8": 4, "f32": 5, "f64": 6}
NP_OF = {"i32": np.int32, "u32": np.uint32, "i64": np.int64, "u64": np.uint64,
         "u8": np.uint8, "f32": np.float32, "f64": np.float64}
BLOCK_BYTES = 4096


def build(force: bool = False) -> str:
    """Compile ref_vote.c into libftref.so next to it (gcc, no fast-math, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.ref_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            L.ref_crc32c.restype = ctypes.c_uint32
            L.ref_crc32c_bitwise.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            L.ref_crc32c_bitwise.restype = ctypes.c_uint32
            L.ref_block_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_void_p]
            L.ref_block_crc32c.restype = ctypes.c_int
            L.ref_eq.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_double]
            L.ref_eq.restype = ctypes.c_int
            L.ref_vote.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
            L.ref_vote.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _as_bytes(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    return np.frombuffer(bytes(data), dtype=np.uint8)


def crc32c(data) -> int:
    """CRC32C of a bytes-like object or array (table form)."""
    b = _as_bytes(data)
    return int(lib().ref_crc32c(_ptr(b), b.size))


def crc32c_bitwise(data) -> int:
    """CRC32C of a bytes-like object or array (bit-at-a-time form)."""
    b = _as_bytes(data)
    return int(lib().ref_crc32c_bitwise(_ptr(b), b.size))


def block_crc32c(buf: np.ndarray, block_bytes: int = BLOCK_BYTES) -> np.ndarray:
    """Independent CRC32C of each block_bytes block of buf's bytes (last block partial)."""
    b = np.ascontiguousarray(buf).view(np.uint8).reshape(-1)
    nblocks = (b.size + block_bytes - 1) // block_bytes
    out = np.zeros(nblocks, dtype=np.uint32)
    rc = lib().ref_block_crc32c(_ptr(b), b.size, block_bytes, _ptr(out))
    if rc != 0:
        raise ValueError("ref_block_crc32c: invalid arguments")
    return out


def eq(dtype: str, a, b, abs_tol: float = 0.0, rel_tol: float = 0.0) -> bool:
    """The voter's comparison of two scalars of the given element type."""
    t = NP_OF[dtype]
    x = np.array([a], dtype=t) if not isinstance(a, np.ndarray) else a.astype(t, copy=False).reshape(1)
    y = np.array([b], dtype=t) if not isinstance(b, np.ndarray) else b.astype(t, copy=False).reshape(1)
    rc = lib().ref_eq(DTYPES[dtype], _ptr(x), _ptr(y), float(abs_tol), float(rel_tol))
    if rc < 0:
        raise ValueError("unknown dtype")
    return bool(rc)


def vote(replicas, dtype: str, abs_tol: float = 0.0, rel_tol: float = 0.0,
         with_ties: bool = False, with_crc: bool = True) -> dict:
    """Vote R same-length host arrays.  Returns a dict with keys
    out, block_crc, mismatch (u64[R]), first_mismatch (i64[R]), no_majority (int),
    first_no_majority (int) and, if with_ties, tie (u8[n])."""
    t = NP_OF[dtype]
    reps = [np.ascontiguousarray(np.asarray(r).view(t).reshape(-1)) for r in replicas]
    R = len(reps)
    n = reps[0].size if R else 0
    if any(r.size != n for r in reps):
        raise ValueError("replicas differ in length")
    ptrs = (ctypes.c_void_p * max(R, 1))(*[_ptr(r) for r in reps])
    out = np.empty(n, dtype=t)
    nbytes = n * np.dtype(t).itemsize
    crc = np.zeros((nbytes + BLOCK_BYTES - 1) // BLOCK_BYTES, dtype=np.uint32)
    mism = np.zeros(max(R, 1), dtype=np.uint64)
    first = np.zeros(max(R, 1), dtype=np.int64)
    nomaj = np.zeros(1, dtype=np.uint64)
    fnomaj = np.zeros(1, dtype=np.int64)
    tie = np.zeros(n, dtype=np.uint8) if with_ties else None
    rc = lib().ref_vote(ctypes.cast(ptrs, ctypes.c_void_p), R, n, DTYPES[dtype],
                        float(abs_tol), float(rel_tol), _ptr(out),
                        _ptr(crc) if with_crc and crc.size else None,
                        _ptr(mism), _ptr(first), _ptr(nomaj), _ptr(fnomaj),
                        _ptr(tie) if tie is not None and tie.size else None)
    if rc != 0:
        raise ValueError("ref_vote: invalid arguments")
    res = {"out": out, "block_crc": crc if with_crc else None,
           "mismatch": mism[:R].copy(), "first_mismatch": first[:R].copy(),
           "no_majority": int(nomaj[0]), "first_no_majority": int(fnomaj[0])}
    if with_ties:
        res["tie"] = tie
    return res
