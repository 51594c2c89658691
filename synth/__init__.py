"""Seeded synthetic protein workloads shared by the oracle tests, the GPU tests and bench.py.

This module generates inputs only. It holds no Smith-Waterman arithmetic: it
draws residue codes, sequence lengths and query sets from a seed, and it
carries the public scoring-matrix and composition tables that those inputs
are drawn with.

Workload shapes follow the paper's experiments (Section IV.A): protein
queries of 144 to 5,478 residues searched against a large protein database
(UniProtKB/TrEMBL, mean length 318, longest 36,805), scored with BLOSUM62.
The real databases and query accessions are not used; residues are drawn
i.i.d. at the Robinson-Robinson background frequencies and lengths from a
clipped log-normal distribution.

Everything is integer-driven (splitmix64 / xoshiro256** in ``synth.c``), so
x86-64 and aarch64 hosts produce the same bytes. The only floating-point step
is the log-normal quantile table, built once per distribution from
``statistics.NormalDist`` and rounded to integers; ``qtable_digest`` exposes
its hash so a test can check that both hosts built the same table.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import statistics
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")

# The 20 standard amino acids in the conventional BLOSUM row order.
ALPHABET = "ARNDCQEGHILKMFPSTWYV"

# BLOSUM62 (Henikoff & Henikoff 1992), rows/columns in ALPHABET order, as
# distributed with NCBI BLAST. Symmetric, entries in [-4, 11].
BLOSUM62 = np.array(
    [
        # A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V
        [4, -1, -2, -2, 0, -1, -1, 0, -2, -1, -1, -1, -1, -2, -1, 1, 0, -3, -2, 0],  # A
        [-1, 5, 0, -2, -3, 1, 0, -2, 0, -3, -2, 2, -1, -3, -2, -1, -1, -3, -2, -3],  # R
        [-2, 0, 6, 1, -3, 0, 0, 0, 1, -3, -3, 0, -2, -3, -2, 1, 0, -4, -2, -3],  # N
        [-2, -2, 1, 6, -3, 0, 2, -1, -1, -3, -4, -1, -3, -3, -1, 0, -1, -4, -3, -3],  # D
        [0, -3, -3, -3, 9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1],  # C
        [-1, 1, 0, 0, -3, 5, 2, -2, 0, -3, -2, 1, 0, -3, -1, 0, -1, -2, -1, -2],  # Q
        [-1, 0, 0, 2, -4, 2, 5, -2, 0, -3, -3, 1, -2, -3, -1, 0, -1, -3, -2, -2],  # E
        [0, -2, 0, -1, -3, -2, -2, 6, -2, -4, -4, -2, -3, -3, -2, 0, -2, -2, -3, -3],  # G
        [-2, 0, 1, -1, -3, 0, 0, -2, 8, -3, -3, -1, -2, -1, -2, -1, -2, -2, 2, -3],  # H
        [-1, -3, -3, -3, -1, -3, -3, -4, -3, 4, 2, -3, 1, 0, -3, -2, -1, -3, -1, 3],  # I
        [-1, -2, -3, -4, -1, -2, -3, -4, -3, 2, 4, -2, 2, 0, -3, -2, -1, -2, -1, 1],  # L
        [-1, 2, 0, -1, -3, 1, 1, -2, -1, -3, -2, 5, -1, -3, -1, 0, -1, -3, -2, -2],  # K
        [-1, -1, -2, -3, -1, 0, -2, -3, -2, 1, 2, -1, 5, 0, -2, -1, -1, -1, -1, 1],  # M
        [-2, -3, -3, -3, -2, -3, -3, -3, -1, 0, 0, -3, 0, 6, -4, -2, -2, 1, 3, -1],  # F
        [-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7, -1, -1, -4, -3, -2],  # P
        [1, -1, 1, 0, -1, 0, 0, 0, -1, -2, -2, 0, -1, -2, -1, 4, 1, -3, -2, -2],  # S
        [0, -1, 0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1, 5, -2, -2, 0],  # T
        [-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1, -4, -3, -2, 11, 2, -3],  # W
        [-2, -2, -2, -3, -2, -1, -2, -3, 2, -1, -1, -2, -1, 3, -3, -2, -2, 2, 7, -1],  # Y
        [0, -3, -3, -3, -1, -2, -2, -3, -3, 3, 1, -2, 1, -1, -2, -2, 0, -3, -1, 4],  # V
    ],
    dtype=np.int8,
)

# Robinson & Robinson (1991) background amino-acid frequencies, in units of
# 1e-5, ALPHABET order (the composition NCBI BLAST uses). Sums to 100,000.
ROBINSON_WEIGHTS = np.array(
    [7805, 5129, 4487, 5364, 1925, 4264, 6295, 7377, 2199, 5142,
     9019, 5744, 2243, 3856, 5203, 7120, 5841, 1330, 3216, 6441],
    dtype=np.uint32,
)

QTABLE_BITS = 16
_lib_lock = threading.Lock()
_lib_handle = None


def _compile() -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "synth.c")
    out = os.path.join(_BUILD, "libsynth.so")
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", src, "-o", tmp],
                       check=True)
        os.replace(tmp, out)
    return out


def build() -> str:
    """Compile ``synth.c`` (idempotent); returns the shared-library path."""
    return _compile()


def _lib():
    global _lib_handle
    with _lib_lock:
        if _lib_handle is None:
            lib = ctypes.CDLL(_compile())
            u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            lib.synth_lengths.argtypes = [u64, u64, u64, p, p]
            lib.synth_residues.argtypes = [u64, u64, p, u64, p, u32, p, ctypes.c_int]
            lib.synth_residues.restype = ctypes.c_int
            lib.synth_mutate.argtypes = [u64, u64, u64, p, u64, p, u32, u32, p]
            lib.synth_uniform_u32.argtypes = [u64, u64, u64, u32, u32, p]
            lib.synth_draws.argtypes = [u64, u64, u64, p]
            _lib_handle = lib
        return _lib_handle


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def robinson_cdf() -> np.ndarray:
    return np.cumsum(ROBINSON_WEIGHTS).astype(np.uint32)


def lognormal_params(mean: float, sd: float) -> tuple[float, float]:
    """(mu, sigma) of the log-normal with the given mean and standard deviation."""
    s2 = math.log(1.0 + (sd / mean) ** 2)
    return math.log(mean) - s2 / 2.0, math.sqrt(s2)


def lognormal_qtable(mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    """65,536 clipped, rounded log-normal quantiles at probabilities (k + 0.5) / 65536."""
    nd = statistics.NormalDist()
    n = 1 << QTABLE_BITS
    out = np.empty(n, dtype=np.uint32)
    for k in range(n):
        v = math.exp(mu + sigma * nd.inv_cdf((k + 0.5) / n))
        out[k] = min(max(int(math.floor(v + 0.5)), lo), hi)
    return out


def qtable_digest(table: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(table, dtype=np.uint32).tobytes()).hexdigest()


def gen_lengths(n: int, qtable: np.ndarray, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    qt = np.ascontiguousarray(qtable, dtype=np.uint32)
    assert qt.size == 1 << QTABLE_BITS
    _lib().synth_lengths(seed, stream, n, _ptr(qt), _ptr(out))
    return out


def gen_residues(lengths: np.ndarray, seed: int, stream: int, nthreads: int | None = None):
    """Residue codes for sequences of the given lengths -> (residues uint8, offsets uint64)."""
    lengths = np.asarray(lengths, dtype=np.uint64)
    offsets = np.zeros(lengths.size + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    res = np.empty(int(offsets[-1]), dtype=np.uint8)
    cdf = robinson_cdf()
    nt = nthreads or min(32, os.cpu_count() or 1)
    rc = _lib().synth_residues(seed, stream, _ptr(offsets), lengths.size, _ptr(cdf), len(cdf),
                               _ptr(res) if res.size else _ptr(np.empty(1, np.uint8)), nt)
    if rc != 0:
        raise RuntimeError("synth_residues failed")
    return res, offsets


def mutate(src: np.ndarray, seed: int, stream: int, index: int, rate_per_10000: int) -> np.ndarray:
    src = np.ascontiguousarray(src, dtype=np.uint8)
    out = np.empty_like(src)
    cdf = robinson_cdf()
    _lib().synth_mutate(seed, stream, index, _ptr(src), src.size, _ptr(cdf), len(cdf),
                        rate_per_10000, _ptr(out))
    return out


def uniform_u32(n: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    _lib().synth_uniform_u32(seed, stream, n, lo, hi, _ptr(out))
    return out


def draws(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _lib().synth_draws(seed, stream, n, _ptr(out))
    return out


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    """A database, a list of queries and the scoring scheme of recurrence (1)."""

    name: str
    residues: np.ndarray          # uint8 codes, all DB sequences concatenated
    offsets: np.ndarray           # uint64, n_seqs + 1
    queries: list                 # list of uint8 arrays
    matrix: np.ndarray            # int8 [A, A], row = query residue, column = DB residue
    alpha: int                    # gap extension penalty
    beta: int                     # gap open + extension penalty
    top_k: int
    alphabet: int = 20
    notes: dict = field(default_factory=dict)

    @property
    def n_seqs(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def db_residues(self) -> int:
        return int(self.offsets[-1])

    def cells(self) -> int:
        return sum(int(q.size) for q in self.queries) * self.db_residues


# Streams: distinct generator streams per array so that every array can be
# regenerated alone.
_S_DB_LEN, _S_DB_RES, _S_Q_LEN, _S_Q_RES, _S_PLANT_POS, _S_PLANT_MUT = 1, 2, 3, 4, 5, 6
_S_ARRIVAL = 7
_S_TAIL_POS, _S_TAIL_LEN = 8, 9

DB_MEAN, DB_SD, DB_LO, DB_HI = 350.0, 250.0, 10, 5000
_qtable_cache: dict = {}


def _qtable(mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    key = (mu, sigma, lo, hi)
    if key not in _qtable_cache:
        _qtable_cache[key] = lognormal_qtable(mu, sigma, lo, hi)
    return _qtable_cache[key]


def db_qtable() -> np.ndarray:
    """Length table of the standard synthetic database: mean 350, sd 250, clipped [10, 5000]."""
    mu, sigma = lognormal_params(DB_MEAN, DB_SD)
    return _qtable(mu, sigma, DB_LO, DB_HI)


def make_db(n_seqs: int, seed: int, qtable: np.ndarray | None = None):
    qt = db_qtable() if qtable is None else qtable
    lengths = gen_lengths(n_seqs, qt, seed, _S_DB_LEN)
    return gen_residues(lengths, seed, _S_DB_RES)


def make_queries(lengths, seed: int) -> list:
    res, off = gen_residues(np.asarray(lengths, dtype=np.uint64), seed, _S_Q_RES)
    return [res[int(off[i]):int(off[i + 1])].copy() for i in range(len(lengths))]


def stream_query_lengths() -> list:
    """20 lengths geometrically spaced from 144 to 5,478 (the paper's query range)."""
    return [int(math.floor(144.0 * (5478.0 / 144.0) ** (k / 19.0) + 0.5)) for k in range(20)]


def small_search(seed: int = 1404) -> Workload:
    """One 144-residue query against 10,000 sequences; BLOSUM62, beta=11, alpha=1, top 10."""
    res, off = make_db(10_000, seed)
    return Workload("small_search", res, off, make_queries([144], seed), BLOSUM62.copy(), 1, 11, 10)


def query_stream(seed: int = 1405, n_seqs: int = 2_000_000, n_queries: int = 20) -> Workload:
    """20 queries of 144..5478 residues (one at a time) against 2,000,000 sequences."""
    res, off = make_db(n_seqs, seed)
    qs = make_queries(stream_query_lengths()[:n_queries], seed)
    return Workload("query_stream", res, off, qs, BLOSUM62.copy(), 1, 11, 10)


def query_batch(seed: int = 1406, n_seqs: int = 1_000_000, n_queries: int = 256) -> Workload:
    """256 queries with lengths uniform in [50, 2000] against 1,000,000 sequences."""
    res, off = make_db(n_seqs, seed)
    lens = uniform_u32(n_queries, 50, 2000, seed, _S_Q_LEN)
    return Workload("query_batch", res, off, make_queries(lens, seed), BLOSUM62.copy(), 1, 11, 10)


def served_query_lengths(n: int, seed: int) -> np.ndarray:
    """Serving queries: log-normal, median 300, sigma 0.642, clipped to [20, 5000]."""
    qt = _qtable(math.log(300.0), 0.642, 20, 5000)
    return gen_lengths(n, qt, seed, _S_Q_LEN)


def served_stream(seed: int = 1407, n_seqs: int = 20_000_000, n_queries: int = 200) -> Workload:
    res, off = make_db(n_seqs, seed)
    qs = make_queries(served_query_lengths(n_queries, seed), seed)
    return Workload("served_stream", res, off, qs, BLOSUM62.copy(), 1, 11, 10)


def arrival_times(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Poisson arrival times (seconds) by inverse-CDF of exponential gaps from keyed draws."""
    d = draws(n, seed, _S_ARRIVAL)
    u = ((d >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    return np.cumsum(-np.log(u) / rate_per_s)


def long_sequences(seed: int = 1408, n_seqs: int = 100_000, n_planted: int = 1000,
            scale: int = 1, long_tail: int = 0) -> Workload:
    """A 5,478-residue query against 100,000 long-ish sequences (mean 2000, up to 35,000)
    with near-duplicates of the query (5% substitutions) planted at random positions.

    scale > 1 multiplies the matrix and both penalties by that integer; every score then
    scales exactly, which pushes the planted pairs past the 16-bit range.

    long_tail > 0 also sets that many other sequences to lengths uniform in [20,000, 35,000]
    (the log-normal alone stays below ~27,000 at this size; the paper's database reaches
    36,805), the tail that one warp per pair would leave running after the rest.
    """
    mu = math.log(2000.0) - 0.642 ** 2 / 2.0
    qt = _qtable(mu, 0.642, 10, 35000)
    q = make_queries([5478], seed)[0]
    lengths = gen_lengths(n_seqs, qt, seed, _S_DB_LEN)
    pos = np.unique((draws(n_planted * 2, seed, _S_PLANT_POS) % np.uint64(n_seqs)).astype(np.int64))
    pos = pos[:n_planted]
    lengths[pos] = q.size
    if long_tail:
        cand = (draws(long_tail * 4 + 16, seed, _S_TAIL_POS) % np.uint64(n_seqs)).astype(np.int64)
        cand = [int(c) for c in dict.fromkeys(cand.tolist()) if c not in set(pos.tolist())]
        tail = np.array(cand[:long_tail], dtype=np.int64)
        lengths[tail] = uniform_u32(tail.size, 20000, 35000, seed, _S_TAIL_LEN)
    res, off = gen_residues(lengths, seed, _S_DB_RES)
    for k, p in enumerate(pos):
        res[int(off[p]):int(off[p + 1])] = mutate(q, seed, _S_PLANT_MUT, k, 500)
    m = (BLOSUM62.astype(np.int32) * scale).astype(np.int8)
    name = "long_sequences" + ("_tail" if long_tail else "") + (
        "_x3" if scale == 3 else f"_x{scale}" if scale > 1 else "")
    w = Workload(name, res, off, [q], m, 1 * scale, 11 * scale, 10)
    w.notes["planted"] = pos
    if long_tail:
        w.notes["tail"] = tail
    return w
