"""Write the stored expected results of the full-size workloads.

Every value written here comes from the CPU oracle (``oracle/``) run on inputs drawn by
the seeded generator (``synth/``); nothing else is imported. For each listed query of a
workload the file records:

  - sha256 of the oracle's whole int32 score vector (little-endian, original database
    order), plus one sha256 per sixteenth of the vector, so a mismatch can be localised;
  - the oracle's top-k list (score descending, then database index ascending: stage (iv)
    of the workflow in Section III, ties completed by index);
  - the score-vector sum, minimum and maximum, and sha256 digests of the generated inputs
    (database residues and offsets, the query), so a consumer can tell a generator
    mismatch from a scoring mismatch.

Run (resumable; each finished query is saved at once):

    python tests/golden/make_golden.py [--only NAME ...] [--threads N]

The workloads are the benchmark configurations: the 20-query stream against 2,000,000
sequences, a seeded subset of the 256-query batch against 1,000,000 sequences, four
served queries against the 20,000,000-sequence resident database, and the long-sequence
workload (5,478-residue query, 100,000 sequences up to 35,000 residues, 1,000 planted
near-duplicates) with its matrix and penalties scaled by 1 and by 3, and with a tail of 64
sequences of 20,000-35,000 residues at 100,000 and at 10,000 sequences.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

N_CHUNKS = 16
BATCH_SUBSET_SEED = 11
BATCH_SUBSET_SIZE = 16


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def chunk_bounds(n: int) -> list[int]:
    return [(n * c) // N_CHUNKS for c in range(N_CHUNKS + 1)]


def score_digest(scores: np.ndarray) -> dict:
    s = np.ascontiguousarray(scores, dtype="<i4")
    b = chunk_bounds(s.size)
    return {"sha256": sha(s), "chunks": [sha(s[b[c]:b[c + 1]]) for c in range(N_CHUNKS)],
            "sum": int(s.astype(np.int64).sum()), "min": int(s.min()), "max": int(s.max())}


def batch_subset(n_queries: int = 256) -> list[int]:
    """The seeded subset of batch queries that carries full-size expected results."""
    rng = np.random.default_rng(BATCH_SUBSET_SEED)
    return sorted(int(i) for i in rng.choice(n_queries, size=BATCH_SUBSET_SIZE, replace=False))


def workloads() -> dict:
    """name -> (generator, ordered query indices). Order = the order queries are scored."""
    return {
        "long_sequences": (lambda: synth.long_sequences(scale=1), [0]),
        "long_sequences_x3": (lambda: synth.long_sequences(scale=3), [0]),
        # with 64 sequences of 20,000-35,000 residues, at 100,000 and at 10,000 sequences
        "long_sequences_tail": (lambda: synth.long_sequences(long_tail=64), [0]),
        "long_sequences_tail_10k": (lambda: synth.long_sequences(n_seqs=10_000, n_planted=100,
                                                                 long_tail=64), [0]),
        # the four lengths named first are scored first, then the rest
        "query_stream": (synth.query_stream, [0, 9, 14, 19] + [i for i in range(20)
                                                               if i not in (0, 9, 14, 19)]),
        "query_batch": (synth.query_batch, batch_subset()),
        "served_stream": (lambda: synth.served_stream(n_queries=4), [0, 1, 2, 3]),
    }


def path_of(name: str) -> str:
    return os.path.join(HERE, f"{name}.json")


def load(name: str) -> dict | None:
    p = path_of(name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def save(name: str, doc: dict) -> None:
    p = path_of(name)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, p)


def run(name: str, threads: int) -> None:
    gen, order = workloads()[name]
    t0 = time.time()
    w = gen()
    inputs = {"residues_sha256": sha(w.residues), "offsets_sha256": sha(w.offsets.astype("<u8")),
              "n_seqs": w.n_seqs, "db_residues": w.db_residues}
    doc = load(name)
    if doc is None or doc.get("inputs") != inputs:
        doc = {"workload": w.name, "inputs": inputs, "alpha": w.alpha, "beta": w.beta,
               "top_k": w.top_k, "n_chunks": N_CHUNKS, "queries": {},
               "written_by": "tests/golden/make_golden.py (oracle/ + synth/ only)"}
    print(f"[{name}] inputs ready in {time.time() - t0:.1f} s: {w.n_seqs} sequences, "
          f"{w.db_residues} residues", flush=True)
    for qi in order:
        q = w.queries[qi]
        key = str(qi)
        if key in doc["queries"] and doc["queries"][key]["query_sha256"] == sha(q):
            continue
        t = time.time()
        s = oracle.scores(q, w.residues, w.offsets, w.matrix, w.alpha, w.beta, nthreads=threads)
        ts, ti = oracle.top_k(s, w.top_k)
        dt = time.time() - t
        doc["queries"][key] = {"qlen": int(q.size), "query_sha256": sha(q),
                               "scores": score_digest(s),
                               "top_scores": [int(v) for v in ts],
                               "top_index": [int(v) for v in ti],
                               "oracle_s": round(dt, 1), "threads": threads}
        save(name, doc)
        print(f"[{name}] query {qi} ({q.size} aa) in {dt:.0f} s "
              f"({q.size * w.db_residues / dt / 1e9:.2f} GCUPS)", flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--only", nargs="*", default=None, help="workload names (default: all)")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    names = a.only or list(workloads())
    for n in names:
        run(n, a.threads)


if __name__ == "__main__":
    main()
