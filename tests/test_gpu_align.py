"""GPU traceback (sw_align) vs the oracle's alignment: score, both cells and every letter."""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")


def _seq(res, off, i):
    return res[int(off[i]):int(off[i + 1])]


def _check(db, res, off, q, M, alpha, beta, idx):
    got = sw.sw_align(db, q, M, alpha, beta, idx)
    assert len(got) == len(idx)
    for g, i in zip(got, idx):
        d = _seq(res, off, int(i))
        e = oracle.align(q, d, M, alpha, beta)
        assert g["db_index"] == int(i)
        for k in ("score", "q_begin", "q_end", "d_begin", "d_end", "ops"):
            assert g[k] == e[k], (int(i), k, g[k] if k != "ops" else g[k][:80],
                                  e[k] if k != "ops" else e[k][:80])
        if g["score"]:
            assert pins.score_of_ops(q, d, M, alpha, beta, g["q_begin"], g["d_begin"],
                                     g["ops"]) == g["score"]
    return got


def test_top_hits_and_random_sequences():
    w = synth.small_search()
    q = w.queries[0]
    with sw.sw_db_load(w.residues, w.offsets) as db:
        _, ts, ti, _ = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, 20, want_scores=False)
        rng = np.random.default_rng(11)
        idx = np.concatenate([ti, rng.integers(0, w.n_seqs, size=60), ti[:3]]).astype(np.uint64)
        got = _check(db, w.residues, w.offsets, q, w.matrix, w.alpha, w.beta, idx)
        assert [g["score"] for g in got[:20]] == list(ts)


@pytest.mark.parametrize("ab", [(1, 11), (2, 12), (0, 5), (5, 2), (0, 0), (3, 0)])
def test_penalties_and_multipass(ab):
    """Queries and sequences longer than one 256-row band and one 64-column block."""
    alpha, beta = ab
    q = synth.make_queries([700], 21 + alpha)[0]
    seqs = [synth.mutate(q, 22, 10 * alpha + beta, k, 800) for k in range(6)]
    seqs += [synth.make_queries([L], 23 + L)[0] for L in (1, 5, 300, 1500)]
    seqs.append(np.concatenate([synth.make_queries([400], 24)[0], q[100:500],
                                synth.make_queries([300], 25)[0]]))
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    with sw.sw_db_load(res, off) as db:
        _check(db, res, off, q, synth.BLOSUM62, alpha, beta, np.arange(len(seqs), dtype=np.uint64))


@pytest.mark.parametrize("A", [4, 24, 32])
def test_alphabets_asymmetric(A):
    rng = np.random.default_rng(300 + A)
    M = rng.integers(-5, 7, size=(A, A)).astype(np.int8)
    lengths = (synth.gen_lengths(80, synth.db_qtable(), 301, 1) // 2 + 1).astype(np.uint64)
    res = rng.integers(0, A, size=int(lengths.sum())).astype(np.uint8)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    q = rng.integers(0, A, size=333).astype(np.uint8)
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check(db, res, off, q, M, 2, 9, np.arange(lengths.size, dtype=np.uint64))


def test_scores_beyond_16_bits_and_edge_cases():
    """Near-copies under 8x BLOSUM62 score above 32767 (int32 throughout); empty and
    unrelated sequences give score 0 and no letters; repeats and an empty request."""
    q = synth.make_queries([1200], 31)[0]
    seqs = [synth.mutate(q, 32, 0, k, 300) for k in range(3)]
    seqs += [np.zeros(0, np.uint8), synth.make_queries([50], 33)[0]]
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    M = (synth.BLOSUM62.astype(np.int32) * 8).astype(np.int8)
    with sw.sw_db_load(res, off) as db:
        got = _check(db, res, off, q, M, 8, 88, np.array([0, 1, 2, 3, 4, 0], np.uint64))
        assert got[0]["score"] > 32767 and got[3]["score"] == 0 and got[3]["ops"] == ""
        assert got[5] == got[0]
        assert sw.sw_align(db, q, M, 8, 88, np.zeros(0, np.uint64)) == []


def test_batch_of_queries_matches_single_calls():
    w = synth.small_search()
    qs = synth.make_queries([144, 700, 37, 1500], 41)
    with sw.sw_db_load(w.residues, w.offsets) as db:
        hits, singles = [], []
        for i, q in enumerate(qs):
            _, _, ti, _ = sw.sw_search(db, q, w.matrix, w.alpha, w.beta, 7, want_scores=False)
            hits += [(i, int(x)) for x in ti]
            singles += sw.sw_align(db, q, w.matrix, w.alpha, w.beta, ti)
        got = sw.sw_align_batch(db, qs, w.matrix, w.alpha, w.beta, hits)
    assert got == singles
    for (i, x), g in zip(hits[::5], got[::5]):
        e = oracle.align(qs[i], w.residues[int(w.offsets[x]):int(w.offsets[x + 1])], w.matrix,
                         w.alpha, w.beta)
        assert all(g[k] == e[k] for k in e)


@pytest.mark.parametrize("ab", [(1, 11), (5, 2), (0, 5)])
def test_long_hits_in_the_block_kernel(ab):
    """Hits of at least 2^20 cells take the score and start-cell programmes in the
    8-warp block kernel (bands of 256 rows, two rounds of warps for a 2,600-row query),
    beside short hits in the one-warp kernel; every alignment must match the oracle's
    letter for letter."""
    alpha, beta = ab
    rng = np.random.default_rng(31 + alpha)
    q = synth.make_queries([2600], 32 + alpha)[0]
    flank = lambda n: synth.make_queries([n], int(rng.integers(1, 1 << 30)))[0]
    seqs = [
        synth.mutate(q, 33, 1, 0, 500),                                  # 2600 x 2600
        np.concatenate([flank(700), synth.mutate(q[200:1900], 33, 2, 1, 700), flank(900)]),
        np.concatenate([flank(3000), q[2100:2600]]),                     # match at the ends
        q[::-1].copy(),                                                  # no long match
        synth.mutate(q[:1000], 33, 3, 2, 300),                           # 2.6 M cells
        flank(820),                                                      # 2.1 M: random
        flank(300),                                                      # 0.8 M: one warp
        synth.mutate(q[1200:1500], 33, 4, 3, 400),
    ]
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    with sw.sw_db_load(res, off) as db:
        got = _check(db, res, off, q, synth.BLOSUM62, alpha, beta,
                     np.arange(len(seqs), dtype=np.uint64))
    assert got[0]["score"] > 0 and len(got[0]["ops"]) > 2000


def test_batch_mixing_long_and_short_hits():
    """One sw_align_batch call whose hits of two queries fall on both kernels (the block
    kernel on the second stream and the one-warp kernel); every alignment must match the
    oracle's letter for letter."""
    rng = np.random.default_rng(51)
    qa = synth.make_queries([2600], 52)[0]
    qb = synth.make_queries([1800], 53)[0]
    flank = lambda n: synth.make_queries([n], int(rng.integers(1, 1 << 30)))[0]
    seqs = [synth.mutate(qa, 54, 1, 0, 600), flank(2000), synth.mutate(qb[100:1700], 54, 2, 1, 400),
            np.concatenate([flank(500), qa[:600], flank(500)]), flank(90), flank(400),
            synth.mutate(qb, 54, 3, 2, 900)]
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    hits = [(qi, d) for d in range(len(seqs)) for qi in (0, 1)]
    with sw.sw_db_load(res, off) as db:
        got = sw.sw_align_batch(db, [qa, qb], synth.BLOSUM62, 1, 11, hits)
    for (qi, d), g in zip(hits, got):
        e = oracle.align((qa, qb)[qi], seqs[d], synth.BLOSUM62, 1, 11)
        assert all(g[k] == e[k] for k in e), (qi, d, g["score"], e["score"])


@pytest.mark.parametrize("A", [3, 32])
def test_long_hits_other_alphabets(A):
    """The block kernel's score rings hold A + 1 code rows (the most shared memory at
    A = 32); long hits over other alphabets, with an asymmetric matrix, must still match
    the oracle letter for letter."""
    rng = np.random.default_rng(400 + A)
    M = rng.integers(-4, 5, size=(A, A)).astype(np.int8)
    np.fill_diagonal(M, 6)
    q = rng.integers(0, A, size=1500).astype(np.uint8)

    def mutated(x, rate):
        y = x.copy()
        hit = rng.random(y.size) < rate
        y[hit] = rng.integers(0, A, size=int(hit.sum()))
        return y

    seqs = [mutated(q, 0.1), np.concatenate([rng.integers(0, A, 400).astype(np.uint8),
                                              mutated(q[300:1200], 0.05)]),
            rng.integers(0, A, 1100).astype(np.uint8), rng.integers(0, A, 200).astype(np.uint8)]
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check(db, res, off, q, M, 1, 7, np.arange(len(seqs), dtype=np.uint64))
