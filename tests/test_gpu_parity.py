"""GPU search vs the CPU oracle: every score and every top-k list must match bit for bit.

All calls go through the C ABI (ctypes binding). Inputs are seeded and
synthetic; sizes keep the oracle within seconds while spanning many tiles,
several query passes and ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")


def _db_from_lengths(lengths, seed, A=20):
    lengths = np.asarray(lengths, dtype=np.uint64)
    res, off = synth.gen_residues(lengths, seed, 2)
    if A != 20:
        rng = np.random.default_rng(seed)
        res = rng.integers(0, A, size=res.size).astype(np.uint8)
    return res, off


# single queries run in the score-profile ring kernel by default; the flag selects the
# int8 query-profile kernel, so every test below runs both
KERNELS = {"ring": 0, "qprof": sw.SW_DB_FLAG_QUERY_PROFILE}


@pytest.fixture(params=sorted(KERNELS))
def kflags(request):
    return KERNELS[request.param]


def _check(db, res, off, q, M, alpha, beta, k, *, expect_recompute=None):
    scores, ts, ti, stats = sw.sw_search(db, q, M, alpha, beta, k)
    es = oracle.scores(q, res, off, M, alpha, beta)
    mism = np.nonzero(scores != es)[0]
    assert mism.size == 0, (f"{mism.size} scores differ; first {mism[:8]}: gpu {scores[mism[:8]]} "
                            f"oracle {es[mism[:8]]}")
    ets, eti = pins.ranked_top_k(es, k)
    assert np.array_equal(ts, ets) and np.array_equal(ti, eti)
    if expect_recompute is not None:
        assert (stats["recomputed"] > 0) == expect_recompute, stats
    return scores, stats


def test_small_search_full(kflags):
    w = synth.small_search()
    with sw.sw_db_load(w.residues, w.offsets, flags=kflags) as db:
        _check(db, w.residues, w.offsets, w.queries[0], w.matrix, w.alpha, w.beta, w.top_k,
               expect_recompute=False)


@pytest.mark.parametrize("qlen", [1, 2, 7, 63, 64, 65, 96, 127, 128, 129, 160, 161, 192, 300, 513, 1100])
def test_query_lengths_across_pass_boundaries(qlen, kflags):
    lengths = synth.gen_lengths(1500, synth.db_qtable(), 31, 1)
    res, off = _db_from_lengths(lengths, 31)
    q = synth.make_queries([qlen], 1000 + qlen)[0]
    with sw.sw_db_load(res, off, flags=kflags) as db:
        _check(db, res, off, q, synth.BLOSUM62, 1, 11, 10)


def test_ragged_database_edges(kflags):
    # empty sequences, lengths around the 4-column blocks and tile boundaries,
    # a count that is not a multiple of 8, and a few long sequences
    lens = [0, 1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 0, 0, 100, 3000, 3001, 3004, 4100, 6, 1]
    res, off = _db_from_lengths(lens, 5)
    for qlen in (1, 50, 200):
        q = synth.make_queries([qlen], 77 + qlen)[0]
        with sw.sw_db_load(res, off, flags=kflags) as db:
            _check(db, res, off, q, synth.BLOSUM62, 1, 11, 30)


@pytest.mark.parametrize("threshold", [16, 64, 300])
def test_long_sequence_kernel(threshold, kflags):
    """Sequences above the threshold go to the warp-per-pair kernel (T = 32)."""
    lengths = synth.gen_lengths(700, synth.db_qtable(), 41, 1)
    res, off = _db_from_lengths(lengths, 41)
    q = synth.make_queries([700], 4242)[0]
    with sw.sw_db_load(res, off, long_threshold=threshold, flags=kflags) as db:
        info = db.info()
        assert info["n_long"] == int((lengths > threshold).sum())
        _check(db, res, off, q, synth.BLOSUM62, 1, 11, 10)


@pytest.mark.parametrize("A", [1, 2, 4, 20, 21, 24, 32])
@pytest.mark.parametrize("ab", [(1, 11), (0, 5), (5, 2), (0, 0), (3, 0), (2, 12)])
def test_alphabets_and_penalties(A, ab, kflags):
    rng = np.random.default_rng(A * 100 + ab[0] * 10 + ab[1])
    M = rng.integers(-6, 9, size=(A, A)).astype(np.int8)  # asymmetric
    lengths = synth.gen_lengths(400, synth.db_qtable(), 51, 1) // 3 + 1
    res, off = _db_from_lengths(lengths, 51, A)
    q = rng.integers(0, A, size=150).astype(np.uint8)
    with sw.sw_db_load(res, off, alphabet=A, flags=kflags) as db:
        _check(db, res, off, q, M, ab[0], ab[1], 15)


def test_int16_saturation_is_rescored_exactly(kflags):
    """Self-similar pairs under a scaled matrix exceed the 16-bit range and are rescored."""
    q = synth.make_queries([900], 9)[0]
    lengths = synth.gen_lengths(300, synth.db_qtable(), 61, 1)
    res, off = _db_from_lengths(lengths, 61)
    # plant copies of the query so their scores pass 32767 under 8x BLOSUM62
    seqs = [res[int(off[i]):int(off[i + 1])] for i in range(len(lengths))]
    for p in (3, 50, 151, 299):
        seqs[p] = synth.mutate(q, 61, 6, p, 300)
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    M = (synth.BLOSUM62.astype(np.int32) * 8).astype(np.int8)
    with sw.sw_db_load(res, off, flags=kflags) as db:
        scores, stats = _check(db, res, off, q, M, 8, 88, 10, expect_recompute=True)
    assert scores.max() > 32767


def test_large_penalties_use_int32():
    lengths = synth.gen_lengths(300, synth.db_qtable(), 71, 1)
    res, off = _db_from_lengths(lengths, 71)
    q = synth.make_queries([250], 71)[0]
    with sw.sw_db_load(res, off) as db:
        _check(db, res, off, q, synth.BLOSUM62, 20000, 20000, 10)
        _check(db, res, off, q, synth.BLOSUM62, 1, 32767, 10)


def test_force_int32_flag():
    lengths = synth.gen_lengths(900, synth.db_qtable(), 81, 1)
    res, off = _db_from_lengths(lengths, 81)
    q = synth.make_queries([333], 81)[0]
    with sw.sw_db_load(res, off, flags=sw.SW_DB_FLAG_FORCE_INT32, long_threshold=400) as db:
        _check(db, res, off, q, synth.BLOSUM62, 1, 11, 10)


@pytest.mark.parametrize("k", [0, 1, 10, 1024])
def test_top_k_sizes_and_ties(k):
    # a 2-letter alphabet and short sequences give many equal scores
    rng = np.random.default_rng(k + 5)
    A = 2
    M = np.array([[1, -1], [-1, 1]], np.int8)
    lengths = rng.integers(0, 12, size=3000).astype(np.uint64)
    res, off = _db_from_lengths(lengths, 91, A)
    q = rng.integers(0, A, size=20).astype(np.uint8)
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check(db, res, off, q, M, 1, 2, k)


@pytest.mark.parametrize("k", [10, 1024])
def test_top_k_ties_across_many_blocks(k):
    """200,000 short sequences over a 2-letter alphabet: scores take a handful of values,
    so the k-th score is tied thousands of times across the top-k kernel's blocks (each
    selects its slice's top k, the row's last block merges) and the list must take the
    lowest indices among the ties."""
    rng = np.random.default_rng(k + 17)
    A = 2
    M = np.array([[1, -1], [-1, 1]], np.int8)
    lengths = rng.integers(0, 12, size=200_000).astype(np.uint64)
    res, off = _db_from_lengths(lengths, 92, A)
    q = rng.integers(0, A, size=20).astype(np.uint8)
    with sw.sw_db_load(res, off, alphabet=A) as db:
        _check(db, res, off, q, M, 1, 2, k)
        # a batch: every row its own top-k in the same launch
        qs = [q, rng.integers(0, A, size=9).astype(np.uint8), rng.integers(0, A, size=31).astype(np.uint8)]
        rows, ts, ti, nt, _ = sw.sw_search_batch(db, qs, M, 1, 2, k, want_scores=True)
    for r, qq, a, b in zip(rows, qs, ts, ti):
        es = oracle.scores(qq, res, off, M, 1, 2)
        assert np.array_equal(r, es)
        ets, eti = pins.ranked_top_k(es, k)
        assert np.array_equal(a, ets) and np.array_equal(b, eti)


def test_top_k_larger_than_database():
    lengths = [5, 9, 0, 14]
    res, off = _db_from_lengths(lengths, 3)
    q = synth.make_queries([30], 3)[0]
    with sw.sw_db_load(res, off) as db:
        scores, ts, ti, _ = sw.sw_search(db, q, synth.BLOSUM62, 1, 11, 100)
    assert ts.size == 4 and ti.size == 4
    es = oracle.scores(q, res, off, synth.BLOSUM62, 1, 11)
    ets, eti = pins.ranked_top_k(es, 100)
    assert np.array_equal(ts, ets) and np.array_equal(ti, eti)


def test_repeated_searches_same_handle():
    w = synth.small_search()
    off = w.offsets[:3001].copy()
    res = w.residues[: int(off[-1])]
    qs = synth.make_queries([144, 600, 37, 2100], 12)
    with sw.sw_db_load(res, off) as db:
        for q in qs + qs[:1]:
            _check(db, res, off, q, w.matrix, w.alpha, w.beta, 10)


def test_device_api_with_torch_buffers():
    torch = pytest.importorskip("torch")
    w = synth.small_search()
    off = w.offsets[:2001].copy()
    res = w.residues[: int(off[-1])]
    q = w.queries[0]
    dev = torch.device("cuda:0")
    d_q = torch.from_numpy(q).to(dev)
    d_m = torch.from_numpy(w.matrix.copy()).to(dev)
    d_s = torch.empty(2000, dtype=torch.int32, device=dev)
    d_ts = torch.empty(10, dtype=torch.int32, device=dev)
    d_ti = torch.empty(10, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    with sw.sw_db_load(res, off) as db:
        sw.sw_search_device(db, d_q, q.size, d_m, 1, 11, 10, d_s, d_ts, d_ti, stream)
        stream.synchronize()
        es = oracle.scores(q, res, off, w.matrix, 1, 11)
        assert np.array_equal(d_s.cpu().numpy(), es)
        ets, eti = pins.ranked_top_k(es, 10)
        assert np.array_equal(d_ts.cpu().numpy(), ets)
        assert np.array_equal(d_ti.cpu().numpy().astype(np.uint64), eti)


def test_batch_matches_single():
    w = synth.small_search()
    off = w.offsets[:1500].copy()
    res = w.residues[: int(off[-1])]
    qs = synth.make_queries([80, 144, 500], 21)
    with sw.sw_db_load(res, off) as db:
        rows, ts, ti, nt, _ = sw.sw_search_batch(db, qs, w.matrix, 1, 11, 10, want_scores=True)
        for i, q in enumerate(qs):
            es = oracle.scores(q, res, off, w.matrix, 1, 11)
            assert np.array_equal(rows[i], es)
            ets, eti = pins.ranked_top_k(es, 10)
            assert np.array_equal(ts[i], ets) and np.array_equal(ti[i], eti)


def test_invalid_inputs_are_rejected():
    res, off = _db_from_lengths([5, 6], 1)
    with pytest.raises(sw.SwError) as e:
        sw.sw_db_load(np.array([0, 1, 25], np.uint8), np.array([0, 3], np.uint64), alphabet=20)
    assert e.value.status == "SW_ERR_INVALID_ARG"
    with sw.sw_db_load(res, off) as db:
        with pytest.raises(sw.SwError):
            sw.sw_search(db, np.array([1, 20], np.uint8), synth.BLOSUM62, 1, 11, 5)
        with pytest.raises(sw.SwError):
            sw.sw_search(db, np.array([1, 2], np.uint8), synth.BLOSUM62, -1, 11, 5)
        with pytest.raises(sw.SwError):
            sw.sw_search(db, np.array([1, 2], np.uint8), synth.BLOSUM62, 1, 11, 1025)
        with pytest.raises(sw.SwError):
            sw.sw_search(db, np.zeros(0, np.uint8), synth.BLOSUM62, 1, 11, 5)


def test_device_budget_gives_oom():
    res, off = _db_from_lengths([50] * 100, 1)
    with pytest.raises(sw.SwError) as e:
        sw.sw_db_load(res, off, device_budget=4096)
    assert e.value.status == "SW_ERR_OOM"


def test_two_handles_from_two_threads():
    """Different handles are independent: searched at the same time from two host threads
    they give the results each gives alone (the binding releases the GIL in C calls)."""
    import threading

    lens_a = synth.gen_lengths(3000, synth.db_qtable(), 101, 1)
    lens_b = synth.gen_lengths(2000, synth.db_qtable(), 102, 1)
    ra, oa = _db_from_lengths(lens_a, 101)
    rb, ob = _db_from_lengths(lens_b, 102)
    qs = synth.make_queries([90, 400, 1200], 103)
    with sw.sw_db_load(ra, oa) as da, sw.sw_db_load(rb, ob) as db_:
        alone = {(n, i): sw.sw_search(d, q, synth.BLOSUM62, 1, 11, 10)[0]
                 for n, d in (("a", da), ("b", db_)) for i, q in enumerate(qs)}
        got, errors = {}, []

        def work(name, d):
            try:
                for _ in range(3):
                    for i, q in enumerate(qs):
                        got[(name, i)] = sw.sw_search(d, q, synth.BLOSUM62, 1, 11, 10)[0]
            except Exception as e:  # reported below
                errors.append(e)

        ts = [threading.Thread(target=work, args=("a", da)), threading.Thread(target=work, args=("b", db_))]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    assert not errors, errors
    for key, v in alone.items():
        assert np.array_equal(got[key], v), key
    assert np.array_equal(alone[("a", 1)], oracle.scores(qs[1], ra, oa, synth.BLOSUM62, 1, 11))


@pytest.mark.parametrize("A", [20, 32])
def test_rescoring_bands_rounds_and_lengths(A, kflags):
    """Saturated pairs of many shapes go through the int32 rescoring kernel: a query of
    2,600 rows (11 bands of 256 rows, so two rounds of the 8 warps, handing rows on through
    the global scratch row), planted sequences shorter and longer than 16 column blocks of
    64, lengths that are not multiples of 64, a local match inside random flanks, one above
    the long-sequence threshold; every score must equal the oracle's."""
    rng = np.random.default_rng(71 + A)
    qlen = 2600
    q = rng.integers(0, A, size=qlen).astype(np.uint8)
    # a matrix with a strong diagonal: near-copies of the query pass the 16-bit range
    M = rng.integers(-6, 4, size=(A, A)).astype(np.int8)
    np.fill_diagonal(M, 60)
    lengths = synth.gen_lengths(300, synth.db_qtable(), 72, 1)
    res, off = _db_from_lengths(lengths, 72, A)
    seqs = [res[int(off[i]):int(off[i + 1])] for i in range(len(lengths))]

    def mutated(x, rate):
        y = x.copy()
        hit = rng.random(y.size) < rate
        y[hit] = rng.integers(0, A, size=int(hit.sum()))
        return y

    planted = {
        5: mutated(q, 0.05),                                   # whole query, L = 2600
        40: mutated(q[:700], 0.03),                            # 700 columns (< 16 blocks)
        41: mutated(q[1000:1999], 0.03),                       # 999 columns
        90: np.concatenate([rng.integers(0, A, 450).astype(np.uint8), mutated(q[300:1500], 0.04),
                            rng.integers(0, A, 777).astype(np.uint8)]),   # local, in flanks
        150: np.concatenate([mutated(q, 0.02), rng.integers(0, A, 900).astype(np.uint8)]),
        299: mutated(q[::-1][:1300], 0.0),                     # reversed: no long match
    }
    for p, s in planted.items():
        seqs[p] = s
    res = np.concatenate(seqs)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([s.size for s in seqs])
    with sw.sw_db_load(res, off, alphabet=A, long_threshold=3000, flags=kflags) as db:
        scores, stats = _check(db, res, off, q, M, 3, 20, 10, expect_recompute=True)
    assert stats["recomputed"] >= 4 and scores.max() > 32767
