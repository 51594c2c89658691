"""The autotuner: it measures every kernel shape, caches the table, and searches stay exact."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")


def test_autotune_cache_and_exact_results(tmp_path):
    lengths = synth.gen_lengths(6000, synth.db_qtable(), 401, 1)
    res, off = synth.gen_residues(lengths, 401, 2)
    cache = str(tmp_path / "tune.json")
    with sw.sw_db_load(res, off) as db:
        t1 = sw.sw_db_autotune(db, synth.BLOSUM62, 1, 11, cache)
        assert not t1["from_cache"]
        for mode in ("pair_db", "query_pair", "pair_ring"):
            row = t1["ns_per_row_residue"][mode]
            assert all(v > 0 for v in row), (mode, row)
        assert t1["ns_per_row_residue"]["int32"][2] > 0  # int32 runs with 16 rows per lane only
        assert t1["int32_over_int16"] > 1.0 and 0 < t1["cutover_fraction"] < 1
        assert os.path.exists(cache) and "query_pair" in json.load(open(cache))
        t2 = sw.sw_db_autotune(db, synth.BLOSUM62, 1, 11, cache)
        assert t2["from_cache"]
        for mode in ("pair_db", "pair_ring"):
            assert np.allclose(t2["ns_per_row_residue"][mode], t1["ns_per_row_residue"][mode],
                               rtol=1e-4)
        # tuned searches are still exact
        qs = synth.make_queries([150, 700, 33], 402)
        for q in qs:
            s, ts, ti, _ = sw.sw_search(db, q, synth.BLOSUM62, 1, 11, 10)
            es = oracle.scores(q, res, off, synth.BLOSUM62, 1, 11)
            assert np.array_equal(s, es)
        rows, _, _, _, _ = sw.sw_search_batch(db, qs, synth.BLOSUM62, 1, 11, 10, want_scores=True)
        for q, r in zip(qs, rows):
            assert np.array_equal(r, oracle.scores(q, res, off, synth.BLOSUM62, 1, 11))


def test_ring_short_last_pass_is_exact(tmp_path):
    """With a table that makes 24 rows per thread the cheapest, every query runs whole
    passes of 192 rows and one last pass of 8, 16 or 24 rows per thread; each way of
    ending the query (and none) must score exactly."""
    lengths = synth.gen_lengths(3000, synth.db_qtable(), 403, 1)
    res, off = synth.gen_residues(lengths, 403, 2)
    cache = str(tmp_path / "tune.json")
    with sw.sw_db_load(res, off) as db:
        sw.sw_db_autotune(db, synth.BLOSUM62, 1, 11, cache)
        table = json.load(open(cache))
        table["pair_ring"] = [1.0, 1.0, 1.0, 1.0, 1e-3]
        table["pair_db"] = [1.0] * 5
        with open(cache, "w") as f:
            json.dump(table, f)
        t = sw.sw_db_autotune(db, synth.BLOSUM62, 1, 11, cache)
        assert t["from_cache"] and t["ns_per_row_residue"]["pair_ring"][4] < 0.01
        # rows left after the whole passes: none, <= 64 (a last pass of 8 rows per thread),
        # <= 128 (16 rows), <= 191 (24 rows); below 192 rows a lone pass of 8 or 16 rows costs
        # the same in the 8- or 16-row kernel, which is then chosen
        qlens = [1, 64, 65, 128, 129, 191, 192, 193, 256, 257, 320, 321, 383, 384, 577, 705]
        qs = synth.make_queries(qlens, 404)
        for q in qs:
            s, ts, ti, _ = sw.sw_search(db, q, synth.BLOSUM62, 1, 11, 10)
            es = oracle.scores(q, res, off, synth.BLOSUM62, 1, 11)
            mism = np.nonzero(s != es)[0]
            assert mism.size == 0, (len(q), mism[:8], s[mism[:8]], es[mism[:8]])
            ets, eti = pins.ranked_top_k(es, 10)
            assert np.array_equal(ts, ets) and np.array_equal(ti, eti)
