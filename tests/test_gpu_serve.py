"""The continuous-batching server: exact results alone and in a mix, and its failure paths.

Failures are made on the host (a client that never waits, a cancelled ticket, a
full queue, a wait that times out); nothing here faults or stalls the GPU.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from tests import pins

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")

B62 = synth.BLOSUM62


@pytest.fixture(scope="module")
def database():
    lengths = synth.gen_lengths(4000, synth.db_qtable(), 301, 1)
    res, off = synth.gen_residues(lengths, 301, 2)
    return res, off


def _expect(res, off, q, alpha=1, beta=11, k=10, M=B62):
    es = oracle.scores(q, res, off, M, alpha, beta)
    return pins.ranked_top_k(es, k)


def test_results_alone_and_in_a_mix(database):
    res, off = database
    qs = synth.make_queries([144, 300, 51, 980, 210, 77, 1400, 333, 19], 302)
    with sw.sw_db_load(res, off) as db, sw.sw_server_create(db, max_active=4, slices=5) as srv:
        # alone
        t = srv.submit(qs[0], B62, 1, 11, 10)
        alone = srv.wait(t)
        # in a mix: three client threads submitting with staggered arrivals
        results = {}

        def client(idx):
            for i in idx:
                results[i] = srv.submit(qs[i], B62, 1, 11, 10)
                time.sleep(0.002)

        th = [threading.Thread(target=client, args=(list(range(j, len(qs), 3)),)) for j in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        got = {i: srv.wait(t) for i, t in results.items()}
        st = srv.stats()
    assert np.array_equal(alone[0], got[0][0]) and np.array_equal(alone[1], got[0][1])
    for i, q in enumerate(qs):
        ets, eti = _expect(res, off, q)
        assert np.array_equal(got[i][0], ets) and np.array_equal(got[i][1], eti), i
        lat = got[i][2]
        assert lat["submit_ms"] <= lat["admit_ms"] <= lat["done_ms"]
    assert st["completed"] == len(qs) + 1 and st["waves"] >= 5
    # the waves' device time is measured and lies within their wall time
    assert 0 < st["gpu_ms"] <= st["busy_ms"] * 1.01 + 0.5


def test_different_schemes_in_the_queue(database):
    res, off = database
    q1, q2 = synth.make_queries([200, 150], 303)
    with sw.sw_db_load(res, off) as db, sw.sw_server_create(db, slices=3) as srv:
        t1 = srv.submit(q1, B62, 1, 11, 5)
        t2 = srv.submit(q2, B62, 2, 12, 5)
        t3 = srv.submit(q1, B62, 20000, 20000, 5)  # int32 waves
        r1, r2, r3 = srv.wait(t1), srv.wait(t2), srv.wait(t3)
    for (q, a, b), r in zip([(q1, 1, 11), (q2, 2, 12), (q1, 20000, 20000)], [r1, r2, r3]):
        ets, eti = _expect(res, off, q, a, b, 5)
        assert np.array_equal(r[0], ets) and np.array_equal(r[1], eti)


def test_timeout_cancel_and_abandoned_client(database):
    res, off = database
    big = synth.make_queries([3000], 304)[0]
    small = synth.make_queries([120], 305)[0]
    with sw.sw_db_load(res, off) as db, sw.sw_server_create(db, max_active=2, slices=6) as srv:
        t_big = srv.submit(big, B62, 1, 11, 10)
        with pytest.raises(sw.SwError) as e:
            srv.wait(t_big, timeout_ms=0)
        assert e.value.status == "SW_ERR_TIMEOUT"
        # a client thread that submits and exits without waiting
        th = threading.Thread(target=lambda: srv.submit(small, B62, 1, 11, 10))
        th.start()
        th.join()
        t_c = srv.submit(small, B62, 1, 11, 10)
        srv.cancel(t_c)
        with pytest.raises(sw.SwError):
            srv.wait(t_c, timeout_ms=10)
        r = srv.wait(t_big)
        t_s = srv.submit(small, B62, 1, 11, 10)
        rs = srv.wait(t_s)
    ets, eti = _expect(res, off, big)
    assert np.array_equal(r[0], ets) and np.array_equal(r[1], eti)
    ets, eti = _expect(res, off, small)
    assert np.array_equal(rs[0], ets) and np.array_equal(rs[1], eti)


def test_queue_full_is_busy(database):
    res, off = database
    q = synth.make_queries([2500], 306)[0]
    with sw.sw_db_load(res, off) as db, sw.sw_server_create(db, max_queue=2, max_active=1,
                                                            slices=8) as srv:
        tickets, busy = [], 0
        for _ in range(12):
            try:
                tickets.append(srv.submit(q, B62, 1, 11, 3))
            except sw.SwError as e:
                assert e.status == "SW_ERR_BUSY"
                busy += 1
        assert busy > 0 and srv.stats()["rejected"] == busy
        for t in tickets:
            srv.wait(t)


def test_admission_by_device_budget(database):
    res, off = database
    with sw.sw_db_load(res, off) as db:
        n = off.size - 1
        slot = n * 4 + 8192 + 1024 * 12 + 64
        with sw.sw_server_create(db, max_active=64, device_budget=3 * slot) as srv:
            assert srv.stats()["max_active"] == 3
        with pytest.raises(sw.SwError) as e:
            sw.sw_server_create(db, device_budget=slot // 2)
        assert e.value.status == "SW_ERR_OOM"


def test_alphabet_32_alone_and_paired():
    """A 32-code alphabet (the single-query ring then runs with a one-column skew): queries
    of equal and of very different lengths through the server, paired or alone, must get
    the oracle's top-k."""
    rng = np.random.default_rng(331)
    lengths = synth.gen_lengths(2000, synth.db_qtable(), 332, 1).astype(np.uint64)
    res = rng.integers(0, 32, size=int(lengths.sum())).astype(np.uint8)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    M = rng.integers(-4, 6, size=(32, 32)).astype(np.int8)
    qs = [rng.integers(0, 32, size=n).astype(np.uint8) for n in (300, 300, 290, 40, 1200, 77)]
    with sw.sw_db_load(res, off, alphabet=32) as db, \
            sw.sw_server_create(db, max_active=6, slices=4) as srv:
        tickets = [srv.submit(q, M, 1, 9, 10) for q in qs]
        got = [srv.wait(t) for t in tickets]
    for q, g in zip(qs, got):
        ets, eti = _expect(res, off, q, 1, 9, 10, M)
        assert np.array_equal(g[0], ets) and np.array_equal(g[1], eti), q.size
