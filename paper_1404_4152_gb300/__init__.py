"""Python binding of libswgb300: exact Smith-Waterman protein database search on a GB300.

Thin ctypes marshalling over the C ABI in ``include/sw.h``; every step of a
search runs in the library's CUDA kernels. The functions carry the C names:

    db = sw_db_load(residues, offsets, alphabet=20)
    scores, top_scores, top_index, stats = sw_search(db, query, matrix, alpha, beta, top_k)
    sw_search_device(db, d_query, d_matrix, alpha, beta, top_k, d_scores, d_top_s, d_top_i, stream)
    sw_db_free(db)

Scoring follows recurrence (1) of Section II.A of the SWAPHI paper: alpha is
the gap extension penalty, beta the sum of the gap open and extension
penalties, and matrix[a, b] scores query residue a against database residue b.

There is no CPU fallback: importing the binding fails loudly if the compiled
library is missing (run ``__graft_entry__.build()`` or ``python -m
paper_1404_4152_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SW_MAX_ALPHABET = 32
SW_MAX_TOP_K = 1024
SW_DB_FLAG_FORCE_INT32 = 1
SW_DB_FLAG_PROFILE = 2
SW_DB_FLAG_QUERY_PROFILE = 4
PHASES = ("wavefront", "rescore_int32", "topk", "batch")

_STATUS = {0: "SW_OK", 1: "SW_ERR_INVALID_ARG", 2: "SW_ERR_OOM", 3: "SW_ERR_CUDA",
           4: "SW_ERR_TIMEOUT", 5: "SW_ERR_BUSY", 6: "SW_ERR_INTERNAL"}


class SwError(RuntimeError):
    """A non-OK status from the library; ``status`` holds the code name."""

    def __init__(self, code: int, message: str):
        self.code = code
        self.status = _STATUS.get(code, str(code))
        super().__init__(f"{self.status}: {message}")


class sw_db_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("long_threshold", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("block_threshold", ctypes.c_uint32)]


class sw_db_info(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_uint64), ("total_residues", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("alphabet", ctypes.c_uint32),
                ("max_length", ctypes.c_uint32), ("n_long", ctypes.c_uint64),
                ("device", ctypes.c_int), ("n_block", ctypes.c_uint64),
                ("block_threshold", ctypes.c_uint32)]


class sw_stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_uint64), ("recomputed", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class sw_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("calls", ctypes.c_uint64 * 4),
                ("cells", ctypes.c_uint64 * 4), ("ms", ctypes.c_double * 4)]


class sw_server_opts(ctypes.Structure):
    _fields_ = [("max_queue", ctypes.c_uint32), ("max_active", ctypes.c_uint32),
                ("max_qlen", ctypes.c_uint32), ("slices", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64)]


class sw_latency(ctypes.Structure):
    _fields_ = [("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double)]


class sw_server_stats(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("cells", ctypes.c_uint64),
                ("busy_ms", ctypes.c_double), ("pending", ctypes.c_uint32),
                ("active", ctypes.c_uint32), ("max_active", ctypes.c_uint32),
                ("slices", ctypes.c_uint32), ("gpu_ms", ctypes.c_double)]


class sw_alignment(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("q_begin", ctypes.c_uint32), ("q_end", ctypes.c_uint32),
                ("db_index", ctypes.c_uint64), ("d_begin", ctypes.c_uint32),
                ("d_end", ctypes.c_uint32), ("ops_offset", ctypes.c_uint64),
                ("ops_len", ctypes.c_uint32)]


class sw_tuning(ctypes.Structure):
    _fields_ = [("ns_per_row_residue", (ctypes.c_double * 5) * 4),
                ("fastest_R", ctypes.c_uint32 * 4), ("int32_over_int16", ctypes.c_double),
                ("cutover_fraction", ctypes.c_double), ("from_cache", ctypes.c_int)]


# Every entry point the header declares: (name, restype, argtypes).
_P, _U8, _U32, _U64, _I32 = (ctypes.c_void_p, ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64,
                             ctypes.c_int32)
SIGNATURES = {
    "sw_db_load": (ctypes.c_int, [_P, _P, _U64, _U32, _P, ctypes.POINTER(_P)]),
    "sw_db_free": (None, [_P]),
    "sw_db_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "sw_db_open": (ctypes.c_int, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "sw_db_get_info": (ctypes.c_int, [_P, _P]),
    "sw_search": (ctypes.c_int, [_P, _P, _U32, _P, _I32, _I32, _U32, _P, _P, _P, _P, _P]),
    "sw_search_device": (ctypes.c_int, [_P, _P, _U32, _P, _I32, _I32, _U32, _P, _P, _P, _P]),
    "sw_search_batch": (ctypes.c_int, [_P, _U32, _P, _P, _P, _I32, _I32, _U32, _P, _P, _P, _P,
                                       _P]),
    "sw_search_batch_device": (ctypes.c_int, [_P, _U32, _P, _P, _P, _I32, _I32, _U32, _P, _P, _P,
                                              _P]),
    "sw_search_noalloc": (ctypes.c_int, [_P, _U32, _P, _U32, _I32, _I32, _P, _P, _U32, _U32, _P,
                                         _P]),
    "sw_server_create": (ctypes.c_int, [_P, _P, ctypes.POINTER(_P)]),
    "sw_server_submit": (ctypes.c_int, [_P, _P, _U32, _P, _I32, _I32, _U32, _P]),
    "sw_server_wait": (ctypes.c_int, [_P, _U64, _U32, _P, _P, _P, _P]),
    "sw_server_cancel": (ctypes.c_int, [_P, _U64]),
    "sw_server_get_stats": (ctypes.c_int, [_P, _P]),
    "sw_server_destroy": (None, [_P]),
    "sw_db_autotune": (ctypes.c_int, [_P, _P, _I32, _I32, ctypes.c_char_p, _P]),
    "sw_db_get_profile": (ctypes.c_int, [_P, _P]),
    "sw_db_reset_profile": (ctypes.c_int, [_P]),
    "sw_db_debug_check": (ctypes.c_int, [_P, _P]),
    "sw_align": (ctypes.c_int, [_P, _P, _U32, _P, _I32, _I32, _P, _U32, _P, _P, _U64, _P]),
    "sw_align_batch": (ctypes.c_int, [_P, _U32, _P, _P, _P, _I32, _I32, _P, _P, _U32, _P, _P, _U64,
                                      _P]),
    "sw_last_error": (ctypes.c_char_p, []),
    "sw_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str | None = None):
    """Load libswgb300.so (raises if it has not been built); with SWGB_DEBUG_BOUNDS=1 in
    the environment, the bounds-checked build libswgb300_debug.so instead."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.lib_path(debug=os.environ.get("SWGB_DEBUG_BOUNDS") == "1")
    if not os.path.exists(p):
        raise ImportError(f"{os.path.basename(p)} is not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(code: int):
    if code != 0:
        raise SwError(code, load_library().sw_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


class Database:
    """A database resident on the device (an ``sw_db*``)."""

    def __init__(self, handle, n_seqs: int, alphabet: int):
        self.handle = handle
        self.n_seqs = n_seqs
        self.alphabet = alphabet

    def info(self) -> dict:
        return sw_db_get_info(self)

    def free(self):
        if self.handle:
            load_library().sw_db_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


SW_BLOCK_ROUTE_OFF = 0xFFFFFFFF  # block_threshold: never use the block-wavefront route


def sw_db_load(residues, offsets, alphabet: int = 20, device: int = 0, long_threshold: int = 0,
               device_budget: int = 0, flags: int = 0, block_threshold: int = 0) -> Database:
    """Load database sequences (uint8 codes, uint64 offsets of n+1 entries) onto the GPU.
    Sequences above ``block_threshold`` (0 = automatic, SW_BLOCK_ROUTE_OFF = never) are
    scored by a block of 8 warps each beside the warp-per-pair kernel."""
    lib = load_library()
    res = np.ascontiguousarray(residues, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    opts = sw_db_opts(device, long_threshold, device_budget, flags, block_threshold)
    h = ctypes.c_void_p()
    _check(lib.sw_db_load(_ptr(res), _ptr(off), off.size - 1, alphabet, ctypes.byref(opts),
                          ctypes.byref(h)))
    return Database(h, off.size - 1, alphabet)


def sw_db_free(db: Database):
    db.free()


def sw_db_save(db: Database, path: str):
    """Write the loaded database (sorted tiles and index) to ``path``."""
    _check(load_library().sw_db_save(db.handle, str(path).encode()))


def sw_db_open(path: str, device: int = 0, device_budget: int = 0, flags: int = 0,
               block_threshold: int = 0) -> Database:
    """Open a database written by sw_db_save (no sorting or tiling)."""
    opts = sw_db_opts(device, 0, device_budget, flags, block_threshold)
    h = ctypes.c_void_p()
    _check(load_library().sw_db_open(str(path).encode(), ctypes.byref(opts), ctypes.byref(h)))
    db = Database(h, 0, 0)
    info = db.info()
    db.n_seqs, db.alphabet = info["n_seqs"], info["alphabet"]
    return db


def sw_db_get_info(db: Database) -> dict:
    info = sw_db_info()
    _check(load_library().sw_db_get_info(db.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in sw_db_info._fields_}


def sw_search(db: Database, query, matrix, alpha: int, beta: int, top_k: int = 10,
              want_scores: bool = True):
    """One query, host buffers -> (scores int32 | None, top_scores, top_index, stats dict)."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    scores = np.empty(db.n_seqs, dtype=np.int32) if want_scores else None
    ts = np.empty(max(top_k, 1), dtype=np.int32)
    ti = np.empty(max(top_k, 1), dtype=np.uint64)
    n_top = ctypes.c_uint32(0)
    st = sw_stats()
    _check(load_library().sw_search(db.handle, _ptr(q), q.size, _ptr(m), int(alpha), int(beta),
                                    int(top_k), _ptr(scores) if scores is not None else None,
                                    _ptr(ts), _ptr(ti), ctypes.byref(n_top), ctypes.byref(st)))
    k = n_top.value
    return scores, ts[:k].copy(), ti[:k].copy(), {f: getattr(st, f) for f, _ in sw_stats._fields_}


def sw_search_device(db: Database, d_query, qlen: int, d_matrix, alpha: int, beta: int,
                     top_k: int, d_scores, d_top_scores, d_top_index, stream=None):
    """One query on DEVICE buffers (torch tensors or raw pointers), enqueued on ``stream``."""

    def addr(x):
        if x is None:
            return None
        if isinstance(x, int):
            return x
        return x.data_ptr()

    s = stream
    if s is not None and not isinstance(s, int):
        s = s.cuda_stream
    _check(load_library().sw_search_device(db.handle, addr(d_query), int(qlen), addr(d_matrix),
                                           int(alpha), int(beta), int(top_k), addr(d_scores),
                                           addr(d_top_scores), addr(d_top_index), s))


def sw_search_batch(db: Database, queries, matrix, alpha: int, beta: int, top_k: int = 10,
                    want_scores: bool = False):
    """Several queries -> (list of score arrays | None, top_scores [nq,k], top_index [nq,k],
    n_top [nq], stats dict)."""
    qs = [np.ascontiguousarray(q, dtype=np.uint8) for q in queries]
    nq = len(qs)
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    qptr = (ctypes.c_void_p * nq)(*[q.ctypes.data for q in qs])
    qlen = np.array([q.size for q in qs], dtype=np.uint32)
    score_rows = [np.empty(db.n_seqs, dtype=np.int32) for _ in qs] if want_scores else None
    sptr = (ctypes.c_void_p * nq)(*[s.ctypes.data for s in score_rows]) if want_scores else None
    ts = np.zeros((nq, max(top_k, 1)), dtype=np.int32)
    ti = np.zeros((nq, max(top_k, 1)), dtype=np.uint64)
    nt = np.zeros(nq, dtype=np.uint32)
    st = sw_stats()
    _check(load_library().sw_search_batch(db.handle, nq, qptr, _ptr(qlen), _ptr(m), int(alpha),
                                          int(beta), int(top_k), sptr, _ptr(ts), _ptr(ti),
                                          _ptr(nt), ctypes.byref(st)))
    return (score_rows, ts[:, :top_k], ti[:, :top_k], nt,
            {f: getattr(st, f) for f, _ in sw_stats._fields_})


def sw_search_batch_device(db: Database, d_queries, qoffsets, d_matrix, alpha: int, beta: int,
                           top_k: int, d_scores, d_top_scores, d_top_index, stream=None):
    """Batch on DEVICE buffers: d_queries concatenated, qoffsets (host, nq+1), d_scores [nq, n]."""

    def addr(x):
        if x is None or isinstance(x, int):
            return x
        return x.data_ptr()

    off = np.ascontiguousarray(qoffsets, dtype=np.uint64)
    s = stream
    if s is not None and not isinstance(s, int):
        s = s.cuda_stream
    _check(load_library().sw_search_batch_device(db.handle, off.size - 1, addr(d_queries),
                                                 _ptr(off), addr(d_matrix), int(alpha), int(beta),
                                                 int(top_k), addr(d_scores), addr(d_top_scores),
                                                 addr(d_top_index), s))


def sw_search_noalloc(d_query, qlen: int, d_matrix, alphabet: int, alpha: int, beta: int,
                      d_residues, d_offsets, n_seqs: int, max_len: int, d_scores, stream=None):
    """Score one query against caller-owned device sequences without any device allocation.

    For callers that may not allocate device memory (their application owns the
    whole device pool, or cannot afford cudaMalloc's synchronisation): every
    buffer is the caller's (torch tensors or raw device pointers), and the
    library's fixed 32 MiB scratch array does the rest. Calls that overlap on
    the GPU share that array and race; run them one after another. Scores the
    kernel cannot compute are marked: -1 for a sequence longer than 2048 residues
    when the query is longer than 512, -2 for a code outside the alphabet.
    """

    def addr(x):
        if x is None or isinstance(x, int):
            return x
        return x.data_ptr()

    s = stream
    if s is not None and not isinstance(s, int):
        s = s.cuda_stream
    _check(load_library().sw_search_noalloc(addr(d_query), int(qlen), addr(d_matrix), int(alphabet),
                                            int(alpha), int(beta), addr(d_residues),
                                            addr(d_offsets), int(n_seqs), int(max_len),
                                            addr(d_scores), s))


def sw_db_get_profile(db: Database) -> dict:
    """Per-phase device time of a handle loaded with SW_DB_FLAG_PROFILE."""
    p = sw_profile()
    _check(load_library().sw_db_get_profile(db.handle, ctypes.byref(p)))
    return {"launches": p.launches,
            "phases": {name: {"calls": p.calls[i], "cells": p.cells[i], "ms": p.ms[i]}
                       for i, name in enumerate(PHASES)}}


def sw_db_reset_profile(db: Database):
    _check(load_library().sw_db_reset_profile(db.handle))


class Server:
    """A continuous-batching search server (an ``sw_server*``) over a loaded database."""

    def __init__(self, handle, db: Database):
        self.handle = handle
        self.db = db

    def submit(self, query, matrix, alpha: int, beta: int, top_k: int = 10) -> int:
        return sw_server_submit(self, query, matrix, alpha, beta, top_k)

    def wait(self, ticket: int, timeout_ms: int = 600_000, top_k: int = SW_MAX_TOP_K):
        return sw_server_wait(self, ticket, timeout_ms, top_k)

    def cancel(self, ticket: int):
        sw_server_cancel(self, ticket)

    def stats(self) -> dict:
        return sw_server_get_stats(self)

    def destroy(self):
        if self.handle:
            load_library().sw_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sw_server_create(db: Database, max_queue: int = 0, max_active: int = 0, max_qlen: int = 0,
                     slices: int = 0, device_budget: int = 0) -> Server:
    opts = sw_server_opts(max_queue, max_active, max_qlen, slices, device_budget)
    h = ctypes.c_void_p()
    _check(load_library().sw_server_create(db.handle, ctypes.byref(opts), ctypes.byref(h)))
    return Server(h, db)


def sw_server_submit(srv: Server, query, matrix, alpha: int, beta: int, top_k: int = 10) -> int:
    q = np.ascontiguousarray(query, dtype=np.uint8)
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    t = ctypes.c_uint64()
    _check(load_library().sw_server_submit(srv.handle, _ptr(q), q.size, _ptr(m), int(alpha),
                                           int(beta), int(top_k), ctypes.byref(t)))
    return t.value


def sw_server_wait(srv: Server, ticket: int, timeout_ms: int = 600_000,
                   top_k: int = SW_MAX_TOP_K):
    """-> (top_scores, top_index, latency dict); raises SwError (SW_ERR_TIMEOUT, ...)."""
    ts = np.zeros(max(top_k, 1), np.int32)
    ti = np.zeros(max(top_k, 1), np.uint64)
    n = ctypes.c_uint32()
    lat = sw_latency()
    _check(load_library().sw_server_wait(srv.handle, int(ticket), int(timeout_ms), _ptr(ts),
                                         _ptr(ti), ctypes.byref(n), ctypes.byref(lat)))
    k = n.value
    return ts[:k].copy(), ti[:k].copy(), {f: getattr(lat, f) for f, _ in sw_latency._fields_}


def sw_server_cancel(srv: Server, ticket: int):
    _check(load_library().sw_server_cancel(srv.handle, int(ticket)))


def sw_server_get_stats(srv: Server) -> dict:
    st = sw_server_stats()
    _check(load_library().sw_server_get_stats(srv.handle, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in sw_server_stats._fields_}


def sw_server_destroy(srv: Server):
    srv.destroy()


def sw_db_autotune(db: Database, matrix, alpha: int, beta: int, cache_path: str | None = None):
    """Measure every kernel shape on a sample of the database; later searches use the best."""
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    t = sw_tuning()
    _check(load_library().sw_db_autotune(db.handle, _ptr(m), int(alpha), int(beta),
                                         cache_path.encode() if cache_path else None,
                                         ctypes.byref(t)))
    modes = ("pair_db", "query_pair", "int32", "pair_ring")
    return {"ns_per_row_residue": {modes[i]: list(t.ns_per_row_residue[i]) for i in range(4)},
            "rows_per_lane": [8, 12, 16, 20, 24],
            "fastest_R": {modes[i]: t.fastest_R[i] for i in range(4)},
            "int32_over_int16": t.int32_over_int16, "cutover_fraction": t.cutover_fraction,
            "from_cache": bool(t.from_cache)}


def sw_last_error() -> str:
    return load_library().sw_last_error().decode()


def sw_version() -> str:
    return load_library().sw_version().decode()


def sw_align(db: Database, query, matrix, alpha: int, beta: int, db_index):
    """One optimal local alignment per listed database sequence (host buffers): a list of
    dicts with score, 0-based half-open query / database ranges and the op string."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    idx = np.ascontiguousarray(db_index, dtype=np.uint64)
    n = int(idx.size)
    out = (sw_alignment * max(n, 1))()
    used = ctypes.c_uint64(0)
    cap = max(1, n * (int(q.size) + int(db.info()["max_length"])))  # an alignment has at most
    ops = ctypes.create_string_buffer(cap)                          # |query| + |sequence| letters
    _check(load_library().sw_align(db.handle, _ptr(q), q.size, _ptr(m), int(alpha), int(beta),
                                   _ptr(idx), n, out, ops, cap, ctypes.byref(used)))
    raw = ops.raw
    res = []
    for k in range(n):
        o = out[k]
        res.append({"score": o.score, "q_begin": o.q_begin, "q_end": o.q_end,
                    "db_index": o.db_index, "d_begin": o.d_begin, "d_end": o.d_end,
                    "ops": raw[o.ops_offset:o.ops_offset + o.ops_len].decode()})
    return res


def sw_db_debug_check(db: Database) -> int:
    """Site of the first out-of-bounds device access the handle's kernels recorded since the
    last check (0: none), then cleared; always 0 unless the bounds-checked build is loaded."""
    site = ctypes.c_uint32(0)
    _check(load_library().sw_db_debug_check(db.handle, ctypes.byref(site)))
    return int(site.value)


def sw_align_batch(db: Database, queries, matrix, alpha: int, beta: int, hits):
    """Alignments for several queries in one call: ``hits`` is a sequence of (query number,
    database index) pairs; returns one dict per hit, as sw_align."""
    qs = [np.ascontiguousarray(q, dtype=np.uint8) for q in queries]
    cat = np.concatenate(qs) if qs else np.zeros(0, np.uint8)
    qoff = np.zeros(len(qs) + 1, dtype=np.uint64)
    qoff[1:] = np.cumsum([q.size for q in qs])
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    hq = np.ascontiguousarray([h[0] for h in hits], dtype=np.uint32)
    hi = np.ascontiguousarray([h[1] for h in hits], dtype=np.uint64)
    n = int(hi.size)
    out = (sw_alignment * max(n, 1))()
    used = ctypes.c_uint64(0)
    maxq = max([q.size for q in qs] + [0])
    cap = max(1, n * (int(maxq) + int(db.info()["max_length"])))
    ops = ctypes.create_string_buffer(cap)
    _check(load_library().sw_align_batch(db.handle, len(qs), _ptr(cat), _ptr(qoff), _ptr(m),
                                         int(alpha), int(beta), _ptr(hq), _ptr(hi), n, out, ops,
                                         cap, ctypes.byref(used)))
    raw = ops.raw
    return [{"score": out[k].score, "q_begin": out[k].q_begin, "q_end": out[k].q_end,
             "db_index": out[k].db_index, "d_begin": out[k].d_begin, "d_end": out[k].d_end,
             "ops": raw[out[k].ops_offset:out[k].ops_offset + out[k].ops_len].decode()}
            for k in range(n)]
