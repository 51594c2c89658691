"""Full-size workloads, bit-exact on every score, against stored oracle results.

``tests/golden/*.json`` holds, for every query the generator lists, the sha256 of the CPU
oracle's whole int32 score vector (plus one sha256 per sixteenth of it) and the oracle's
top-k list. They are written by ``tests/golden/make_golden.py``, which calls only the
oracle and the seeded input generator. Each test regenerates the same inputs, checks their
digests (so a generator difference is reported as such, not as a scoring error), runs the
GPU search exactly as the benchmark does, hashes the GPU's score vector and compares both
the hash and the top-k list. A mismatch names the sixteenths of the vector that differ.

Workloads: the 20-query stream against 2,000,000 sequences (each query alone), a seeded
subset of the 256-query batch against 1,000,000 sequences (all 256 in one graph-captured
batch), four served queries against the 20,000,000-sequence resident database (plain
search for the score vectors, the continuous-batching server for the top-k lists), the
long-sequence workload scaled by 1 and by 3 (int32 rescoring of the planted pairs), and
its long-tail variants at 100,000 and 10,000 sequences with and without the block route.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _golden(name):
    p = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(p):
        pytest.skip(f"no stored oracle results for {name}")
    with open(p) as f:
        doc = json.load(f)
    if not doc["queries"]:
        pytest.skip(f"no stored oracle results for {name}")
    return doc


def _check_inputs(doc, w):
    got = {"residues_sha256": _sha(w.residues), "offsets_sha256": _sha(w.offsets.astype("<u8")),
           "n_seqs": w.n_seqs, "db_residues": w.db_residues}
    assert got == doc["inputs"], "the generator drew different inputs than the stored results'"


def _check_scores(entry, scores, ts, ti, tag):
    s = np.ascontiguousarray(scores, dtype="<i4")
    if _sha(s) != entry["scores"]["sha256"]:
        n = doc_chunks = len(entry["scores"]["chunks"])
        b = [(s.size * c) // n for c in range(n + 1)]
        bad = [c for c in range(doc_chunks) if _sha(s[b[c]:b[c + 1]]) != entry["scores"]["chunks"][c]]
        raise AssertionError(f"{tag}: score vector differs from the oracle's in sixteenths {bad} "
                             f"(sum {int(s.astype(np.int64).sum())} vs {entry['scores']['sum']}, "
                             f"max {int(s.max())} vs {entry['scores']['max']})")
    assert list(map(int, ts)) == entry["top_scores"], tag
    assert list(map(int, ti)) == entry["top_index"], tag


def test_query_stream_every_score():
    doc = _golden("query_stream")
    w = synth.query_stream()
    _check_inputs(doc, w)
    with sw.sw_db_load(w.residues, w.offsets) as db:
        for key, entry in sorted(doc["queries"].items(), key=lambda kv: int(kv[0])):
            q = w.queries[int(key)]
            assert _sha(q) == entry["query_sha256"]
            scores, ts, ti, _ = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, doc["top_k"])
            _check_scores(entry, scores, ts, ti, f"query {key} ({q.size} aa)")


def test_query_batch_every_score_of_the_stored_subset():
    doc = _golden("query_batch")
    w = synth.query_batch()
    _check_inputs(doc, w)
    with sw.sw_db_load(w.residues, w.offsets) as db:
        rows, ts, ti, nt, _ = sw.sw_search_batch(db, w.queries, w.matrix, w.alpha, w.beta,
                                                 doc["top_k"], want_scores=True)
    for key, entry in doc["queries"].items():
        qi = int(key)
        assert _sha(w.queries[qi]) == entry["query_sha256"]
        _check_scores(entry, rows[qi], ts[qi], ti[qi], f"batch query {qi}")


@pytest.mark.parametrize("name,scale", [("long_sequences", 1), ("long_sequences_x3", 3)])
def test_long_sequences_every_score(name, scale):
    doc = _golden(name)
    w = synth.long_sequences(scale=scale)
    _check_inputs(doc, w)
    q = w.queries[0]
    entry = doc["queries"]["0"]
    assert _sha(q) == entry["query_sha256"]
    with sw.sw_db_load(w.residues, w.offsets, long_threshold=3000) as db:
        scores, ts, ti, st = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, doc["top_k"])
    assert (st["recomputed"] > 0) == (scale > 1)
    _check_scores(entry, scores, ts, ti, name)


@pytest.mark.parametrize("name,n_seqs", [("long_sequences_tail", 100_000),
                                         ("long_sequences_tail_10k", 10_000)])
def test_long_tail_every_score_with_and_without_the_block_route(name, n_seqs):
    """The long-sequence workload with 64 sequences of 20,000-35,000 residues: every score
    with the block route (the automatic threshold, and one forced low enough to route
    several hundred sequences) and without it."""
    doc = _golden(name)
    w = synth.long_sequences(n_seqs=n_seqs, n_planted=1000 * n_seqs // 100_000, long_tail=64)
    _check_inputs(doc, w)
    q = w.queries[0]
    entry = doc["queries"]["0"]
    assert _sha(q) == entry["query_sha256"]
    for bt in (0, 6000, sw.SW_BLOCK_ROUTE_OFF):
        with sw.sw_db_load(w.residues, w.offsets, long_threshold=3000, block_threshold=bt) as db:
            scores, ts, ti, _ = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, doc["top_k"])
        _check_scores(entry, scores, ts, ti, f"{name} block_threshold={bt}")


def test_served_stream_every_score_and_served_top_k():
    doc = _golden("served_stream")
    w = synth.served_stream(n_queries=4)
    _check_inputs(doc, w)
    keys = sorted(doc["queries"], key=int)
    with sw.sw_db_load(w.residues, w.offsets) as db:
        for key in keys:
            q = w.queries[int(key)]
            assert _sha(q) == doc["queries"][key]["query_sha256"]
            scores, ts, ti, _ = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, doc["top_k"])
            _check_scores(doc["queries"][key], scores, ts, ti, f"served query {key} (plain)")
        # the same queries through the server, submitted together (continuous batching)
        with sw.sw_server_create(db, max_active=8, slices=8) as srv:
            tickets = [srv.submit(w.queries[int(k)], w.matrix, w.alpha, w.beta, doc["top_k"])
                       for k in keys]
            got = [srv.wait(t) for t in tickets]
    for key, (gs, gi, _) in zip(keys, got):
        assert list(map(int, gs)) == doc["queries"][key]["top_scores"], key
        assert list(map(int, gi)) == doc["queries"][key]["top_index"], key
