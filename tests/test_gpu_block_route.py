"""The block-wavefront route for very long database sequences, element by element against
the CPU oracle.

Sequences above ``block_threshold`` (and above ``long_threshold``) are scored by a whole
block of 8 warps each, the multi-warp wavefront of the intra-sequence model (Section
III.C), beside the warp-per-pair search kernel; everything else takes the usual kernels.
The databases here put sequence lengths on both sides of an explicit threshold (and of the
long-sequence threshold), so whole tiles go to each side and one tile holds both; the
queries span several 256-row bands of the block wavefront and several passes of the
search kernels.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")

M = synth.BLOSUM62


def _straddling_db(seed=2201, threshold=4000):
    """Lengths just below, at and above the threshold, mixed with ordinary ones."""
    rng = np.random.default_rng(seed)
    near = np.concatenate([np.arange(threshold - 12, threshold + 13),          # 25 around it
                           rng.integers(threshold + 1, threshold + 3000, 22),  # above
                           rng.integers(1001, threshold, 20)])                 # long, below
    short = synth.gen_lengths(260, synth.db_qtable(), seed, 1).astype(np.int64)
    lengths = np.concatenate([near, short, [0, 1, 5]])
    lengths = lengths[rng.permutation(lengths.size)].astype(np.uint64)
    return synth.gen_residues(lengths, seed, 2)


def test_single_query_across_the_block_threshold():
    res, off = _straddling_db()
    q = synth.make_queries([2600], 2202)[0]
    exp = oracle.scores(q, res, off, M, 1, 11)
    lengths = np.diff(off)
    for bt in (4000, sw.SW_BLOCK_ROUTE_OFF):
        with sw.sw_db_load(res, off, long_threshold=1000, block_threshold=bt) as db:
            info = db.info()
            if bt == 4000:
                assert info["block_threshold"] == 4000
                n_above = int((lengths > 4000).sum())
                assert n_above <= info["n_block"] < n_above + 8
            else:
                assert info["n_block"] == 0
            scores, ts, ti, _ = sw.sw_search(db, q, M, 1, 11, 10)
        bad = np.nonzero(scores != exp)[0]
        assert bad.size == 0, (bt, bad[:10], lengths[bad[:10]], scores[bad[:10]], exp[bad[:10]])


def test_batch_and_int32_across_the_block_threshold():
    """A batch of queries (two per lane pair, graph-captured) and the forced int32 path with
    the route, both against the oracle; the batch twice (graph replay)."""
    res, off = _straddling_db(seed=2203, threshold=3500)
    qs = synth.make_queries([700, 1300, 333], 2204)
    exp = [oracle.scores(q, res, off, M, 1, 11) for q in qs]
    with sw.sw_db_load(res, off, long_threshold=800, block_threshold=3500) as db:
        assert db.info()["n_block"] > 0
        for _ in range(2):
            rows, ts, ti, nt, _ = sw.sw_search_batch(db, qs, M, 1, 11, 10, want_scores=True)
            for r, e in zip(rows, exp):
                assert np.array_equal(r, e), np.nonzero(r != e)[0][:10]
    with sw.sw_db_load(res, off, long_threshold=800, block_threshold=3500,
                       flags=sw.SW_DB_FLAG_FORCE_INT32) as db:
        for q, e in zip(qs, exp):
            scores, _, _, _ = sw.sw_search(db, q, M, 1, 11, 5)
            assert np.array_equal(scores, e)


def test_block_threshold_below_long_threshold_is_raised_to_it():
    res, off = _straddling_db(seed=2205, threshold=2000)
    q = synth.make_queries([300], 2206)[0]
    with sw.sw_db_load(res, off, long_threshold=2500, block_threshold=100) as db:
        info = db.info()
        assert info["block_threshold"] == 2500
        assert info["n_block"] == min(-(-info["n_long"] // 8) * 8, info["n_seqs"])
        scores, _, _, _ = sw.sw_search(db, q, M, 1, 11, 5)
    assert np.array_equal(scores, oracle.scores(q, res, off, M, 1, 11))


def test_long_tail_workload_with_and_without_the_route():
    """A 10,000-sequence version of the long-sequence workload with 64 sequences of
    20,000-35,000 residues, where the automatic threshold routes the tail: the route and no
    route give the same scores, and a seeded sample plus the tail and the top hits equal
    the oracle's."""
    w = synth.long_sequences(n_seqs=10_000, n_planted=100, long_tail=64)
    q = w.queries[0]
    out = {}
    for bt in (0, sw.SW_BLOCK_ROUTE_OFF):
        with sw.sw_db_load(w.residues, w.offsets, long_threshold=3000, block_threshold=bt) as db:
            if bt == 0:
                assert db.info()["n_block"] >= 64
            out[bt] = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, w.top_k)
    assert np.array_equal(out[0][0], out[sw.SW_BLOCK_ROUTE_OFF][0])
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([rng.integers(0, w.n_seqs, 40), w.notes["tail"][:24],
                                    out[0][2].astype(np.int64)]))
    exp = oracle.scores(q, w.residues, w.offsets, w.matrix, w.alpha, w.beta, which=idx)
    assert np.array_equal(out[0][0][idx], exp)


def test_block_route_after_save_and_reopen(tmp_path):
    """A database written by sw_db_save and reopened routes the same sequences (the route
    is a load option, applied to the reopened sorted order) and scores them exactly."""
    res, off = _straddling_db(seed=2207, threshold=3000)
    q = synth.make_queries([900], 2208)[0]
    exp = oracle.scores(q, res, off, M, 1, 11)
    path = str(tmp_path / "db.swgb")
    with sw.sw_db_load(res, off, long_threshold=1000, block_threshold=3000) as db:
        n_block = db.info()["n_block"]
        assert n_block > 0
        sw.sw_db_save(db, path)
    with sw.sw_db_open(path, block_threshold=3000) as db:
        assert db.info()["n_block"] == n_block
        scores, ts, ti, _ = sw.sw_search(db, q, M, 1, 11, 10)
    assert np.array_equal(scores, exp)
    ets, eti = pins.ranked_top_k(exp, 10)
    assert np.array_equal(ts, ets) and np.array_equal(ti, eti)
