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
