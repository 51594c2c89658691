"""Full-size workloads in the configuration the benchmark runs, checked on sampled outputs.

At these sizes the oracle cannot score every pair in a test's time, so each
test checks (a) a seeded random sample of scores and every top-k hit against
the oracle one by one, and (b) that the returned top-k list is exactly the
ranked top-k of the returned score vector.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")


def _check_sampled(w, q, scores, ts, ti, sample, extra=()):
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.integers(0, w.n_seqs, size=sample), ti.astype(np.int64),
                                    np.asarray(extra, dtype=np.int64)]))
    es = oracle.scores(q, w.residues, w.offsets, w.matrix, w.alpha, w.beta, which=idx)
    bad = np.nonzero(scores[idx] != es)[0]
    assert bad.size == 0, (idx[bad[:8]], scores[idx[bad[:8]]], es[bad[:8]])
    ets, eti = pins.ranked_top_k(scores, w.top_k)
    assert np.array_equal(ts, ets) and np.array_equal(ti, eti)


def test_two_million_sequences_sampled():
    w = synth.query_stream()
    with sw.sw_db_load(w.residues, w.offsets) as db:
        for q in (w.queries[0], w.queries[10], w.queries[19]):
            scores, ts, ti, st = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, w.top_k)
            _check_sampled(w, q, scores, ts, ti, sample=400 if q.size > 2000 else 1500)


@pytest.mark.parametrize("scale", [1, 3])
def test_long_sequences_and_planted_duplicates(scale):
    """A 5,478-residue query against 100,000 sequences of mean length 2,000 (up to 35,000),
    1,000 of them near-copies of the query. scale 3 multiplies the matrix and penalties by 3,
    which pushes the planted pairs past the 16-bit range and through int32 rescoring."""
    w = synth.long_sequences(scale=scale)
    q = w.queries[0]
    planted = w.notes["planted"]
    with sw.sw_db_load(w.residues, w.offsets, long_threshold=3000) as db:
        assert db.info()["n_long"] > 10000
        scores, ts, ti, st = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, w.top_k)
        assert (st["recomputed"] > 0) == (scale > 1)
        _check_sampled(w, q, scores, ts, ti, sample=120, extra=planted[:200])
        # every top hit is a planted near-duplicate
        assert set(ti.tolist()) <= set(int(p) for p in planted)
        if scale > 1:
            assert scores[planted].min() > 32767


def test_traceback_of_planted_long_pairs_above_16_bits():
    """The long-sequence workload with matrix and penalties x3: alignments of planted
    5,478-residue near-copies whose scores pass the 16-bit range, letter for letter
    against the oracle."""
    w = synth.long_sequences(scale=3)
    q = w.queries[0]
    planted = np.asarray(w.notes["planted"][:6], dtype=np.uint64)
    rng = np.random.default_rng(5)
    others = rng.integers(0, w.n_seqs, size=6).astype(np.uint64)
    idx = np.concatenate([planted, others])
    with sw.sw_db_load(w.residues, w.offsets, long_threshold=3000) as db:
        got = sw.sw_align(db, q, w.matrix, w.alpha, w.beta, idx)
    for g, i in zip(got, idx):
        d = w.residues[int(w.offsets[i]):int(w.offsets[i + 1])]
        e = oracle.align(q, d, w.matrix, w.alpha, w.beta)
        assert all(g[k] == e[k] for k in e), (int(i), g["score"], e["score"])
    assert min(g["score"] for g in got[:6]) > 32767


def test_batch_of_256_queries_against_a_million_sequences_sampled():
    """The batched workload as the benchmark runs it (256 queries, lengths uniform in
    [50, 2000], against 1,000,000 sequences, one graph-captured launch): for a seeded sample
    of 24 queries, a sample of scores and every top-k hit against the oracle, and each
    top-k list against the ranked top-k of its returned row."""
    w = synth.query_batch()
    with sw.sw_db_load(w.residues, w.offsets) as db:
        rows, ts, ti, nt, st = sw.sw_search_batch(db, w.queries, w.matrix, w.alpha, w.beta,
                                                  w.top_k, want_scores=True)
    rng = np.random.default_rng(11)
    for qi in sorted(rng.choice(len(w.queries), size=24, replace=False).tolist()):
        _check_sampled(w, w.queries[qi], rows[qi], ts[qi], ti[qi], sample=60)


def test_served_stream_at_full_size_matches_plain_search():
    """The serving workload's resident database (20,000,000 sequences, 7 G residues): eight
    queries of the served length mix submitted together, so waves pair some of them and run
    others alone over 8 slices; every top-k list must equal the single-query search's on the
    same handle, and its hits' scores the oracle's."""
    res, off = synth.make_db(20_000_000, 1407)
    qs = synth.make_queries(synth.served_query_lengths(8, 1417), 1417)
    with sw.sw_db_load(res, off) as db:
        plain = [sw.sw_search(db, q, synth.BLOSUM62, 1, 11, 10, want_scores=False) for q in qs]
        with sw.sw_server_create(db, max_active=8, slices=8) as srv:
            tickets = [srv.submit(q, synth.BLOSUM62, 1, 11, 10) for q in qs]
            got = [srv.wait(t) for t in tickets]
    for q, (s, ts, ti, _), g in zip(qs, plain, got):
        assert np.array_equal(g[0], ts) and np.array_equal(g[1], ti)
        es = oracle.scores(q, res, off, synth.BLOSUM62, 1, 11, which=ti.astype(np.int64))
        assert np.array_equal(es, ts)
