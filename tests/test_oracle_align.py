"""The oracle's traceback (one optimal local alignment), pinned by enumeration.

Brute force over every alignment of short sequences fixes the score, the end cell (the
first optimal end in query-then-database order), the start cell (the latest start of an
optimal alignment ending there) and that the op string is one of the optimal alignments
between them; on longer sequences the op string must reproduce the score of the
recurrence, whose linear-space form is pinned in test_oracle_pins.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

PENALTIES = [(1, 11), (2, 12), (0, 5), (5, 2), (0, 0), (3, 0), (2, 3)]


@pytest.mark.parametrize("ab", PENALTIES)
def test_align_matches_enumeration(ab):
    alpha, beta = ab
    rng = np.random.default_rng(7000 + 10 * alpha + beta)
    checked = 0
    for case in range(60):
        A = int(rng.integers(2, 6))
        M = rng.integers(-4, 6, size=(A, A)).astype(np.int8)
        q = rng.integers(0, A, size=int(rng.integers(1, 6))).astype(np.uint8)
        d = rng.integers(0, A, size=int(rng.integers(1, 6))).astype(np.uint8)
        r = oracle.align(q, d, M, alpha, beta)
        best, opt = pins.brute_force_optimal_alignments(q, d, M, alpha, beta)
        assert r["score"] == best, (case, q, d)
        if best == 0:
            assert r["ops"] == "" and r["q_end"] == r["q_begin"] == 0
            continue
        end = min((qe, de) for qb, qe, db, de, ops in opt)
        assert (r["q_end"], r["d_end"]) == end
        start = max((qb, db) for qb, qe, db, de, ops in opt if (qe, de) == end)
        assert (r["q_begin"], r["d_begin"]) == start
        paths = {ops for qb, qe, db, de, ops in opt if (qb, db, qe, de) == start + end}
        assert r["ops"] in paths
        checked += 1
    assert checked > 20


@pytest.mark.parametrize("ab", [(1, 11), (2, 12), (5, 2)])
def test_align_reproduces_the_score(ab):
    alpha, beta = ab
    rng = np.random.default_rng(7100 + alpha)
    for L in (40, 150, 400):
        q = synth.make_queries([L], 7100 + L)[0]
        d = synth.mutate(q, 7100, L, 0, 300) if L > 100 else synth.make_queries([L + 30], 7200 + L)[0]
        r = oracle.align(q, d, synth.BLOSUM62, alpha, beta)
        assert r["score"] == oracle.sw_score(q, d, synth.BLOSUM62, alpha, beta)
        ops = r["ops"]
        assert ops[0] == "M" and ops[-1] == "M"
        assert ops.count("M") + ops.count("I") == r["q_end"] - r["q_begin"]
        assert ops.count("M") + ops.count("D") == r["d_end"] - r["d_begin"]
        assert pins.score_of_ops(q, d, synth.BLOSUM62, alpha, beta, r["q_begin"], r["d_begin"],
                                 ops) == r["score"]
