"""Batched search (two queries per lane pair, one persistent launch) vs the CPU oracle.

Every query of a batch must get exactly the scores and top-k list the oracle
gives it alone; the batch must give the same result when its captured graph
is replayed.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")


def _db(n, seed, cap=None, long_lengths=()):
    lengths = synth.gen_lengths(n, synth.db_qtable(), seed, 1)
    if cap:
        lengths = np.minimum(lengths, cap)
    lengths = np.concatenate([lengths, np.asarray(long_lengths, dtype=np.uint32)]).astype(np.uint64)
    return synth.gen_residues(lengths, seed, 2)


def _check_batch(db, res, off, queries, M, alpha, beta, k):
    rows, ts, ti, nt, stats = sw.sw_search_batch(db, queries, M, alpha, beta, k, want_scores=True)
    for i, q in enumerate(queries):
        es = oracle.scores(q, res, off, M, alpha, beta)
        bad = np.nonzero(rows[i] != es)[0]
        assert bad.size == 0, (i, q.size, bad[:8], rows[i][bad[:8]], es[bad[:8]])
        ets, eti = pins.ranked_top_k(es, k)
        assert int(nt[i]) == ets.size
        assert np.array_equal(ts[i][: ets.size], ets) and np.array_equal(ti[i][: eti.size], eti)
    return stats


def test_batch_odd_count_mixed_lengths():
    res, off = _db(2500, 201)
    lens = [7, 1500, 144, 145, 600, 37, 999]
    qs = synth.make_queries(lens, 202)
    with sw.sw_db_load(res, off) as db:
        stats = _check_batch(db, res, off, qs, synth.BLOSUM62, 1, 11, 10)
    assert stats["recomputed"] == 0


def test_batch_single_query_and_large_k():
    res, off = _db(900, 203)
    qs = synth.make_queries([321], 204)
    with sw.sw_db_load(res, off) as db:
        _check_batch(db, res, off, qs, synth.BLOSUM62, 1, 11, 1024)


def test_batch_long_bin():
    res, off = _db(600, 205, long_lengths=[3100, 4000, 5200, 3001])
    qs = synth.make_queries([200, 777, 1300, 64], 206)
    with sw.sw_db_load(res, off, long_threshold=500) as db:
        assert db.info()["n_long"] > 4
        _check_batch(db, res, off, qs, synth.BLOSUM62, 1, 11, 10)


@pytest.mark.parametrize("ab", [(0, 5), (5, 2), (2, 12)])
def test_batch_penalties_and_asymmetric_matrix(ab):
    rng = np.random.default_rng(ab[0] * 7 + ab[1])
    A = 24
    M = rng.integers(-6, 9, size=(A, A)).astype(np.int8)
    lengths = synth.gen_lengths(700, synth.db_qtable(), 207, 1) // 3 + 1
    res = rng.integers(0, A, size=int(lengths.sum())).astype(np.uint8)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    qs = [rng.integers(0, A, size=n).astype(np.uint8) for n in (90, 91, 250, 3)]
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check_batch(db, res, off, qs, M, ab[0], ab[1], 15)


def test_batch_int32_penalties():
    res, off = _db(500, 208)
    qs = synth.make_queries([100, 300, 50], 209)
    with sw.sw_db_load(res, off) as db:
        _check_batch(db, res, off, qs, synth.BLOSUM62, 20000, 20000, 10)


def test_batch_saturation_is_rescored():
    q_long = synth.make_queries([900], 210)[0]
    res, off = _db(300, 211)
    seqs = [res[int(off[i]):int(off[i + 1])] for i in range(off.size - 1)]
    for p in (5, 77, 299):
        seqs[p] = synth.mutate(q_long, 211, 6, p, 300)
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    M = (synth.BLOSUM62.astype(np.int32) * 8).astype(np.int8)
    qs = [q_long, synth.make_queries([850], 212)[0], q_long[::-1].copy()]
    with sw.sw_db_load(res, off) as db:
        stats = _check_batch(db, res, off, qs, M, 8, 88, 10)
    assert stats["recomputed"] > 0


def test_batch_device_graph_replay():
    torch = pytest.importorskip("torch")
    res, off = _db(1500, 213)
    lens = [150, 400, 90, 1200]
    qs = synth.make_queries(lens, 214)
    qoff = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    dev = torch.device("cuda:0")
    d_q = torch.from_numpy(np.concatenate(qs)).to(dev)
    d_m = torch.from_numpy(synth.BLOSUM62.copy()).to(dev)
    n = off.size - 1
    d_s = torch.empty((len(qs), n), dtype=torch.int32, device=dev)
    d_ts = torch.empty((len(qs), 10), dtype=torch.int32, device=dev)
    d_ti = torch.empty((len(qs), 10), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    expect = [oracle.scores(q, res, off, synth.BLOSUM62, 1, 11) for q in qs]
    with sw.sw_db_load(res, off, flags=sw.SW_DB_FLAG_PROFILE) as db:
        for rep in range(3):  # capture, then two replays
            d_s.fill_(-5)
            torch.cuda.synchronize()
            sw.sw_search_batch_device(db, d_q, qoff, d_m, 1, 11, 10, d_s, d_ts, d_ti, stream)
            stream.synchronize()
            got = d_s.cpu().numpy()
            for i in range(len(qs)):
                assert np.array_equal(got[i], expect[i]), (rep, i)
                ets, eti = pins.ranked_top_k(expect[i], 10)
                assert np.array_equal(d_ts[i].cpu().numpy(), ets)
                assert np.array_equal(d_ti[i].cpu().numpy().astype(np.uint64), eti)
        prof = sw.sw_db_get_profile(db)
        assert prof["phases"]["batch"]["calls"] == 3


@pytest.mark.parametrize("A", [3, 32])
def test_batch_alphabets_and_rows_per_thread_groups(A):
    """Batches over alphabets of 3 and 32 codes (the query-pair profile holds A + 1 code
    rows), with lengths spread so the pairs fall into several rows-per-thread groups (one
    launch each); every score and top-k list must equal the oracle's."""
    rng = np.random.default_rng(220 + A)
    lengths = synth.gen_lengths(1200, synth.db_qtable(), 221, 1).astype(np.uint64)
    res = rng.integers(0, A, size=int(lengths.sum())).astype(np.uint8)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    M = rng.integers(-5, 6, size=(A, A)).astype(np.int8)
    lens = [40, 41, 60, 64, 100, 128, 129, 150, 160, 161, 250, 300, 383, 384, 700, 960]
    qs = [rng.integers(0, A, size=n).astype(np.uint8) for n in lens]
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check_batch(db, res, off, qs, M, 1, 6, 10)
