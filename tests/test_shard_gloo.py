"""The multi-GPU shard plan on CPU ranks: partition balance and the top-k exchange.

Two gloo processes each score their shard with the oracle (standing in for a
GPU) and exchange their local top-k with one all-gather; the merged list must
equal the single-process top-k of the whole database.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1404_4152_gb300 import shard
from tests import pins


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_balances_residues_and_covers_everything():
    lengths = synth.gen_lengths(5000, synth.db_qtable(), 501, 1)
    off = np.zeros(lengths.size + 1, np.uint64)
    off[1:] = np.cumsum(lengths)
    for world in (2, 3, 4, 8):
        parts = shard.partition(off, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(lengths.size))
        loads = [int(lengths[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(lengths.max())


def test_merge_matches_global_ranking_with_ties():
    rng = np.random.default_rng(5)
    scores = rng.integers(0, 6, size=300).astype(np.int32)  # heavy ties
    parts = shard.partition(np.concatenate([[0], np.cumsum(rng.integers(1, 9, size=300))]), 3)
    local = []
    for p in parts:
        ts, ti = pins.ranked_top_k(scores[p], 12)
        local.append((ts, p[ti.astype(np.int64)].astype(np.uint64)))
    ms, mi = shard.merge_top_k(local, 12)
    es, ei = pins.ranked_top_k(scores, 12)
    assert np.array_equal(ms, es) and np.array_equal(mi, ei)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.small_search()
    n = 1200
    off = w.offsets[: n + 1]
    res = w.residues[: int(off[-1])]
    gi = shard.partition(off, world)[rank]
    sres, soff = shard.shard_arrays(res, off, gi)
    local = oracle.scores(w.queries[0], sres, soff, w.matrix, w.alpha, w.beta)
    ts, ti = pins.ranked_top_k(local, 10)
    ms, mi = shard.allgather_top_k(ts, gi[ti.astype(np.int64)], 10)
    q.put((rank, ms.tolist(), mi.tolist()))
    dist.destroy_process_group()


def _sharded_worker(rank, world, port, q):
    """The sharded search entry point (shard.sharded_top_k), the oracle standing in for
    each rank's GPU search of its shard."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.small_search()
    n = 900
    off = w.offsets[: n + 1]
    res = w.residues[: int(off[-1])]
    queries = [w.queries[0], synth.make_queries([37], 9)[0]]

    def search_shard(sres, soff, qs, k):
        out = []
        for qq in qs:
            local = oracle.scores(qq, sres, soff, w.matrix, w.alpha, w.beta, nthreads=2)
            out.append(pins.ranked_top_k(local, k))
        return out

    merged = shard.sharded_top_k(res, off, queries, 10, search_shard, rank, world)
    q.put((rank, [(ms.tolist(), mi.tolist()) for ms, mi in merged]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_search_equals_single_database_top_k(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.small_search()
    off = w.offsets[:901]
    res = w.residues[: int(off[-1])]
    for qi, qq in enumerate([w.queries[0], synth.make_queries([37], 9)[0]]):
        full = oracle.scores(qq, res, off, w.matrix, w.alpha, w.beta)
        es, ei = pins.ranked_top_k(full, 10)
        for rank, lists in out:
            assert lists[qi][0] == es.tolist() and lists[qi][1] == ei.tolist(), (rank, qi)


def test_two_rank_allgather_top_k():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.small_search()
    off = w.offsets[:1201]
    full = oracle.scores(w.queries[0], w.residues[: int(off[-1])], off, w.matrix, w.alpha, w.beta)
    es, ei = pins.ranked_top_k(full, 10)
    for rank, ms, mi in out:
        assert ms == es.tolist() and mi == ei.tolist(), rank


def test_bench_strong_scaling_shards_partition_one_database():
    """bench.py's strong-scaling workload: every rank draws the same database and keeps
    its shard; the shards hold every sequence exactly once, residue for residue."""
    import argparse

    import bench

    args = argparse.Namespace(scaling="strong", n_seqs=3000, n_queries=3)
    world = 3
    full = None
    seen = []
    for rank in range(world):
        w, full, gi = bench.build_workload(args, rank, world)
        assert w.queries[0].tobytes() == full.queries[0].tobytes()
        for k, s in enumerate(gi):
            a = w.residues[int(w.offsets[k]):int(w.offsets[k + 1])]
            b = full.residues[int(full.offsets[s]):int(full.offsets[s + 1])]
            assert np.array_equal(a, b)
        seen.append(gi)
    allidx = np.sort(np.concatenate(seen))
    assert np.array_equal(allidx, np.arange(full.n_seqs))
    w1, f1, g1 = bench.build_workload(argparse.Namespace(scaling="weak", n_seqs=3000, n_queries=3), 1, world)
    assert f1 is None and g1 is None and w1.n_seqs == 3000
