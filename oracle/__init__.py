"""CPU oracle for exact Smith-Waterman database search (recurrence (1), Section II.A).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The GPU library
never calls it and shares no code with it.

``sw_oracle.c`` holds the arithmetic (plain scalar int32, one cell at a time);
this module compiles it with gcc and marshals numpy arrays to it.

Pins (in ``tests/test_oracle_pins.py``): brute-force enumeration of every
local alignment on sequences of at most 8 residues, an O(n^3) explicit-gap
formulation, a no-gap special case that reduces to Kadane's maximum subarray
per diagonal, and invariants (non-negativity, self-score bound, swap symmetry,
reversal, integer scaling, zero-padding, concatenation monotonicity, upper
bound). Top-k is pinned against a plain sort.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_handle = None


def build(src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle with gcc (idempotent). ``src``/``out`` override the paths."""
    src = src or os.path.join(_HERE, "sw_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    out = out or os.path.join(_BUILD, "libsw_oracle.so")
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", src, "-o", tmp],
                       check=True)
        os.replace(tmp, out)
    return out


def _declare(lib):
    p, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    for name in ("oracle_sw_score", "oracle_sw_score_full"):
        f = getattr(lib, name)
        f.argtypes = [p, u32, p, u32, p, u32, i32, i32]
        f.restype = i32
    lib.oracle_scores.argtypes = [p, u32, p, p, p, u64, p, u32, i32, i32, p, ctypes.c_int]
    lib.oracle_scores.restype = ctypes.c_int
    lib.oracle_top_k.argtypes = [p, u64, u32, p, p, p]
    lib.oracle_top_k.restype = ctypes.c_int
    lib.oracle_sw_align.argtypes = [p, u32, p, u32, p, u32, i32, i32, p, p, u32, p]
    lib.oracle_sw_align.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load the compiled oracle; ``path`` loads another build of it (e.g. a mutant)."""
    global _handle
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _handle is None:
            _handle = _declare(ctypes.CDLL(build()))
        return _handle


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else np.empty(1, a.dtype).ctypes.data


def _matrix(matrix) -> tuple[np.ndarray, int]:
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    assert m.ndim == 2 and m.shape[0] == m.shape[1]
    return m, int(m.shape[0])


def sw_score(q, d, matrix, alpha: int, beta: int, lib=None, full: bool = False) -> int:
    """Score of one pair under recurrence (1); q indexes rows of ``matrix``."""
    lib = lib or load()
    q, d = _u8(q), _u8(d)
    M, A = _matrix(matrix)
    f = lib.oracle_sw_score_full if full else lib.oracle_sw_score
    return int(f(_ptr(q), q.size, _ptr(d), d.size, _ptr(M), A, int(alpha), int(beta)))


def scores(query, residues, offsets, matrix, alpha: int, beta: int, which=None,
           nthreads: int | None = None, lib=None) -> np.ndarray:
    """Scores of ``query`` against every database sequence (or those listed in ``which``)."""
    lib = lib or load()
    q = _u8(query)
    db = _u8(residues)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    M, A = _matrix(matrix)
    if which is None:
        count, wp = off.size - 1, None
    else:
        w = np.ascontiguousarray(which, dtype=np.uint64)
        count, wp = w.size, _ptr(w)
    out = np.zeros(count, dtype=np.int32)
    nt = nthreads or (os.cpu_count() or 1)
    lib.oracle_scores(_ptr(q), q.size, _ptr(db), _ptr(off), wp, count, _ptr(M), A, int(alpha),
                      int(beta), _ptr(out), nt)
    return out


def top_k(score_array, k: int, lib=None):
    """(top_scores int32, top_index uint64): score descending, then index ascending."""
    lib = lib or load()
    s = np.ascontiguousarray(score_array, dtype=np.int32)
    kk = min(int(k), s.size)
    ts = np.zeros(max(kk, 1), dtype=np.int32)
    ti = np.zeros(max(kk, 1), dtype=np.uint64)
    n = ctypes.c_uint32(0)
    lib.oracle_top_k(_ptr(s), s.size, int(k), _ptr(ts), _ptr(ti), ctypes.byref(n))
    return ts[: n.value].copy(), ti[: n.value].copy()


def search(query, residues, offsets, matrix, alpha: int, beta: int, k: int,
           nthreads: int | None = None, lib=None):
    """Every score plus the top-k list, as stage (iv) of the workflow orders them."""
    s = scores(query, residues, offsets, matrix, alpha, beta, nthreads=nthreads, lib=lib)
    ts, ti = top_k(s, k, lib=lib)
    return s, ts, ti


def align(q, d, matrix, alpha: int, beta: int, lib=None):
    """One optimal local alignment (the oracle's traceback): a dict with score, the 0-based
    half-open query and database ranges and the op string ('M', 'I', 'D')."""
    lib = lib or load()
    q, d = _u8(q), _u8(d)
    m, A = _matrix(matrix)
    out = np.zeros(5, dtype=np.int32)
    cap = int(q.size + d.size + 1)
    ops = ctypes.create_string_buffer(cap)
    n_ops = ctypes.c_uint32(0)
    rc = lib.oracle_sw_align(_ptr(q), q.size, _ptr(d), d.size, _ptr(m), A, int(alpha), int(beta),
                             _ptr(out), ops, cap, ctypes.byref(n_ops))
    if rc != 0:
        raise RuntimeError("oracle_sw_align failed")
    return {"score": int(out[0]), "q_begin": int(out[1]), "q_end": int(out[2]),
            "d_begin": int(out[3]), "d_end": int(out[4]), "ops": ops.raw[:n_ops.value].decode()}
