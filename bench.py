#!/usr/bin/env python3
"""Benchmark: exact Smith-Waterman protein database search on GB300, in GCUPS.

Workload (default): 20 queries of 144..5,478 residues (geometrically spaced,
the paper's query-length range) searched one at a time against 2,000,000
synthetic database sequences (~700 M residues, log-normal lengths mean 350 /
sd 250, Robinson-Robinson composition), BLOSUM62, beta = 11, alpha = 1, top 10.
One step = all 20 searches (every DP cell of every pair, rescoring and top-k
included). GCUPS = sum(|query|) * sum(|db sequence|) / seconds.

  value      device-resident: queries, matrix and outputs in HBM, timed with
             CUDA events on the stream the library launches on.
  e2e        the same searches through the host-buffer call sw_search: query
             copied in from pinned memory, every score and the top-k copied
             back each call; wall-clock.
  roofline   the dominant kernel (wavefront over the shorter sequences):
             algorithmic ALU lane-operations / its mean launch time, against the
             ALU-pipe peak at the SM clock sampled during the run.
  cpu_baseline  the CPU oracle on a bounded sample of the same workload.
  batched    256 queries against 1,000,000 sequences in one graph-captured batch
             (a persistent launch per rows-per-thread group of query pairs, one more
             for the queries that run alone), against the config-1 loop (vs_plain)
             and against the same queries one at a time on the same database, with
             every score compared (vs_loop_same_db).
  served     the continuous-batching server over 20,000,000 resident sequences,
             Poisson arrivals at 10-500 q/s (200 each, bounded queue) and at the
             0.5-2 q/s knee (64 each): p50 / p99 latency, queueing and service
             time, sustained and busy GCUPS per rate.
  long_sequences  a 5,478-residue query against 100,000 long sequences (the
             warp-per-pair kernel), the same scaled x3 (int32 rescoring), and with
             a long tail of 20,000-35,000 residues with and without the block route.
  traceback  alignments of the top hits of every stream query.

The JSON line ends with compact "batched" and "served" summaries.
--impl reference times the CPU oracle itself as the reference arm.
Under torchrun the one database is partitioned over the ranks (strong scaling;
--scaling weak gives each rank its own database); the JSON line reports the
slowest rank's time and the merged top-k check, and the batched, served,
long-sequence and traceback legs (single-GPU measurements) are skipped.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# Minimal integer-ALU work per DP cell with this GPU's instruction set: H as one
# three-way max with the zero floor (the diagonal add runs on the FMA pipe), E and F
# as one fused add-max each, and half of a three-way running max.
ALU_OPS_PER_CELL = 3.5
ALU_LANES_PER_CLK_SM = 64     # 32-bit lanes per clock per SM on the integer ALU pipe (4 x 16)
S16X2_CELLS_PER_LANE = 2      # one 32-bit lane holds two 16-bit DP cells
PAPER_PHI_GCUPS_MAX = 58.8    # SWAPHI InterSP, one Xeon Phi 5110P, TrEMBL (Section IV.A)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant search kernel
# per launch: the mean over the 20 launches of one step of the 20-query stream against
# 2,000,000 sequences, every launch captured (ncu, one pass, full size). Valid for that
# workload and the kernel source whose sha256 starts with TRAFFIC_SOURCE.
TRAFFIC_BYTES_PER_LAUNCH = 18.60e9
TRAFFIC_SOURCE = "6984e149683534ad"
# ALU-pipe work per row update of that kernel (sm__pipe_alu_cycles_active over row updates,
# 7.83 cycles, in two-cycle instruction equivalents; an 807-residue query's launch): the mix
# the kernel executes, against the 3.5 minimum
ALU_OPS_PER_CELL_MEASURED = 3.92


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-seqs", type=int, default=2_000_000)
    p.add_argument("--n-queries", type=int, default=20)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--batch-steps", type=int, default=1,
                   help="timed steps of the batched workload (0 skips it)")
    p.add_argument("--batch-loop", action=argparse.BooleanOptionalAction, default=True,
                   help="also time the batch's queries one at a time on the same database")
    p.add_argument("--batch-seqs", type=int, default=1_000_000)
    p.add_argument("--batch-queries", type=int, default=256)
    p.add_argument("--serve-seqs", type=int, default=20_000_000)
    p.add_argument("--serve-rates", default="10,50,100,500",
                   help="comma-separated Poisson arrival rates (queries/s), all past one GPU's "
                        "capacity of about 1.8 q/s; empty skips them")
    p.add_argument("--serve-arrivals", type=int, default=200, help="arrivals per overload rate")
    p.add_argument("--serve-knee", default="0.5,1,2",
                   help="arrival rates around one GPU's capacity (the latency knee); empty skips")
    p.add_argument("--serve-knee-arrivals", type=int, default=64)
    p.add_argument("--serve-slots", type=int, default=8,
                   help="queries on the GPU at once (device-memory slots)")
    p.add_argument("--serve-queue", type=int, default=16,
                   help="waiting queries before arrivals are rejected")
    p.add_argument("--long-steps", type=int, default=2,
                   help="timed searches of the long-sequence workloads (scores x1 and x3; 0 skips)")
    p.add_argument("--align-top", type=int, default=10,
                   help="alignments (traceback) of this many top hits per query of the 20-query stream "
                        "(0 skips)")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                   help="N > 1: one database partitioned over the GPUs (strong) or one database "
                        "per GPU (weak)")
    return p.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def cpu_oracle_sample(w, seconds: float, threads: int):
    """Time the oracle on all queries x the first S database sequences (~`seconds` of work)."""
    import oracle

    # calibrate on a small slice with a mid-length query
    q0 = w.queries[len(w.queries) // 2]
    n_cal = 300
    t = time.perf_counter()
    oracle.scores(q0, w.residues, w.offsets[: n_cal + 1], w.matrix, w.alpha, w.beta, nthreads=threads)
    dt = time.perf_counter() - t
    rate = q0.size * int(w.offsets[n_cal]) / max(dt, 1e-6)  # cells/s
    qsum = sum(int(q.size) for q in w.queries)
    per_seq = float(w.offsets[-1]) / w.n_seqs
    S = int(max(64, min(w.n_seqs, seconds * rate / (qsum * per_seq))))
    for _ in range(3):  # grow the sample until it takes about `seconds`
        off = w.offsets[: S + 1]
        t = time.perf_counter()
        for q in w.queries:
            oracle.scores(q, w.residues, off, w.matrix, w.alpha, w.beta, nthreads=threads)
        dt = time.perf_counter() - t
        if dt >= 0.6 * seconds or S >= w.n_seqs:
            break
        S = int(min(w.n_seqs, S * seconds / max(dt, 1e-3)))
    cells = qsum * int(off[-1])
    return cells / dt / 1e9, {"sequences": S, "residues": int(off[-1]), "cells": cells, "seconds": dt}


def build_workload(args, rank, world):
    """The 20-query stream. Strong scaling (N > 1, the default): every rank generates the
    same 2,000,000-sequence database and keeps its shard (shard.partition: residues dealt
    longest first to the least-loaded rank). Weak scaling: each rank its own database."""
    if world > 1 and args.scaling == "strong":
        import dataclasses

        from paper_1404_4152_gb300 import shard

        full = synth.query_stream(seed=1405, n_seqs=args.n_seqs, n_queries=args.n_queries)
        gi = shard.partition(full.offsets, world)[rank]
        sres, soff = shard.shard_arrays(full.residues, full.offsets, gi)
        return dataclasses.replace(full, residues=sres, offsets=soff), full, gi
    w = synth.query_stream(seed=1405 + 1000 * rank, n_seqs=args.n_seqs, n_queries=args.n_queries)
    return w, None, None


def workload_config(w, args, world, full=None):
    db = full if full is not None else w
    per_gpu = "" if full is not None else " per GPU"
    return {
        "workload": (f"query_stream: {len(w.queries)} queries of {min(q.size for q in w.queries)}.."
                     f"{max(q.size for q in w.queries)} aa, one at a time, vs {db.n_seqs:,} "
                     f"sequences ({db.db_residues / 1e6:.0f} M aa){per_gpu}"
                     + (f", sharded over {world} GPUs" if full is not None else "")
                     + f"; BLOSUM62, beta={w.beta}, alpha={w.alpha}; every score + top-{w.top_k}"),
        "global_batch": len(w.queries) * (1 if full is not None else world),
        "db_sequences_per_gpu": w.n_seqs,
        "db_residues_per_gpu": w.db_residues,
        "query_lengths": [int(q.size) for q in w.queries],
        "parallelism": (f"db-shard x{world} (one database partitioned)" if full is not None
                        else f"db x{world} (one database per GPU)" if world > 1 else "single GPU"),
        "l2": "inputs larger than L2 (database resident in HBM, ~0.7 GB > 129 MB L2)",
    }


def compact_batched(b):
    if not b:
        return None
    return {"gcups": round(b["value"], 1), "vs_plain": round(b.get("vs_plain", 0.0), 4),
            "vs_loop_same_db": (round(b["vs_loop_same_db"], 4) if b.get("vs_loop_same_db")
                                else None),
            "padded_frac": b.get("padded_frac"), "launches_per_batch": b.get("launches_per_batch"),
            "ms_per_step": round(b["ms_per_step"], 1)}


def compact_served(s):
    if not s:
        return None
    cols = ["rate_qps", "arrivals", "completed", "rejected", "p50_s", "p99_s", "sustained_gcups",
            "busy_gcups"]
    rows = [[r[c] if not isinstance(r[c], float) else round(r[c], 3 if c.endswith("_s") else 1)
             for c in cols] for r in s["rates"]]
    return {"columns": cols, "rates": rows}


def check_sharded_top_k(sw, w, full, shard_index, db, d_ts, d_ti, rank, world):
    """After the timed region of a sharded run: every query's shard-local top-k mapped to
    global indices and merged over the ranks (one all-gather each, the only exchange), and
    on rank 0 compared with the single-GPU search of the whole database."""
    from paper_1404_4152_gb300 import shard

    k = w.top_k
    ts_all, ti_all = d_ts.cpu().numpy(), d_ti.cpu().numpy()
    merged = [shard.allgather_top_k(ts_all[i], shard.local_to_global(ti_all[i], shard_index), k)
              for i in range(len(w.queries))]
    if rank != 0:
        return None
    equal = 0
    with sw.sw_db_load(full.residues, full.offsets, alphabet=20) as whole:
        for i, q in enumerate(full.queries):
            _, ts, ti, _ = sw.sw_search(whole, q, full.matrix, full.alpha, full.beta, k,
                                        want_scores=False)
            equal += int(np.array_equal(ts, merged[i][0]) and np.array_equal(ti, merged[i][1]))
    return {"queries": len(full.queries), "merged_equal_to_single_gpu": equal,
            "exchange": f"one all-gather of {k} (score, index) pairs per rank per query"}


def batch_padding(qlens, tuning):
    """Padded query rows of a batch under the library's plan rule (queries sorted by length
    and paired, the pair running the longer query's rows for both; each pair on the rows per
    thread of least measured cost, whole passes of 8 x R rows; a pair that costs more than
    its two queries alone in the score-profile ring, and a query without a partner, run
    there: 24 rows per lane and a short last pass of 8, 16 or 24): computed rows / real
    rows - 1, the number of rows-per-thread groups (one persistent launch each) and the
    number of queries run alone (one more launch when any)."""
    Rs = [8, 12, 16, 20, 24]
    ns_tab = (tuning or {}).get("ns_per_row_residue", {})
    ns = ns_tab.get("query_pair") or [0.0] * 5
    ns_ring = ns_tab.get("pair_ring") or [0.0] * 5

    def pass_cost(tab, j, alu):
        return tab[j] * 8 * Rs[j] if tab[j] > 0 else alu * Rs[j] + 8.0

    def qp_cost(la, j):
        c = -(-la // (8 * Rs[j])) * pass_cost(ns, j, 3.5)
        return c * (0.97 if ns[j] <= 0 and Rs[j] == 16 else 1.0)

    def ring_rows(m):  # rows the ring computes for an m-row query, and their cost
        rem = m % 192
        last = 0 if rem == 0 else 8 if rem <= 64 else 16 if rem <= 128 else 24
        cost = (m // 192) * pass_cost(ns_ring, 4, 3.9) + (
            pass_cost(ns_ring, Rs.index(last), 3.9) if last else 0.0)
        return (m // 192) * 192 + 8 * last, cost

    order = sorted(qlens, reverse=True)
    computed, groups, singles = 0, set(), 0
    for i in range(0, len(order), 2):
        la = order[i]
        lb = order[i + 1] if i + 1 < len(order) else 0
        j = min(range(5), key=lambda j: qp_cost(la, j))
        alone = [ring_rows(m) for m in (la, lb) if m]
        pair = 2 * -(-la // (8 * Rs[j])) * pass_cost(ns, j, 3.5)
        if lb == 0 or pair > sum(c for _, c in alone):
            computed += sum(r for r, _ in alone)
            singles += len(alone)
            continue
        groups.add(Rs[j])
        computed += 2 * (-(-la // (8 * Rs[j]))) * 8 * Rs[j]
    return computed / max(1, sum(qlens)) - 1.0, len(groups), singles


def run_batched(args, sw, torch, dev, rank):
    """256 queries (lengths uniform in [50, 2000]) vs 1,000,000 sequences in one
    graph-captured batch per step (a persistent launch per rows-per-thread group of query
    pairs, one more for the queries that run alone in the ring); GCUPS and the kernel-phase
    time."""
    w = synth.query_batch(seed=1406 + 1000 * rank, n_seqs=args.batch_seqs, n_queries=args.batch_queries)
    db = sw.sw_db_load(w.residues, w.offsets, alphabet=20, flags=sw.SW_DB_FLAG_PROFILE)
    tuning = None if args.no_tune else sw.sw_db_autotune(db, w.matrix, w.alpha, w.beta)
    qlens = [int(q.size) for q in w.queries]
    qoff = np.concatenate([[0], np.cumsum(qlens)]).astype(np.uint64)
    nq, n, k = len(qlens), w.n_seqs, w.top_k
    padded_frac, groups, singles = batch_padding(qlens, tuning)
    d_q = torch.from_numpy(np.concatenate(w.queries)).to(dev)
    d_m = torch.from_numpy(w.matrix.copy()).to(dev)
    d_s = torch.empty((nq, n), dtype=torch.int32, device=dev)
    d_ts = torch.empty((nq, k), dtype=torch.int32, device=dev)
    d_ti = torch.empty((nq, k), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        sw.sw_search_batch_device(db, d_q, qoff, d_m, w.alpha, w.beta, k, d_s, d_ts, d_ti, stream)

    step()  # captures the graph
    stream.synchronize()
    sw.sw_db_reset_profile(db)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_steps):
        step()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    prof = sw.sw_db_get_profile(db)
    cells = sum(qlens) * w.db_residues * args.batch_steps
    loop = None
    if args.batch_loop:
        # the same queries one at a time on the same database and buffers (one pass), and
        # whether every score equals the batch's
        batch_scores = d_s.clone()
        e0.record(stream)
        for i in range(nq):
            sw.sw_search_device(db, d_q[int(qoff[i]):int(qoff[i + 1])], qlens[i], d_m, w.alpha,
                                w.beta, k, d_s[i], d_ts[i], d_ti[i], stream)
        e1.record(stream)
        stream.synchronize()
        lms = e0.elapsed_time(e1)
        loop = {"gcups": sum(qlens) * w.db_residues / (lms / 1e3) / 1e9, "ms": lms,
                "scores_identical": bool(torch.equal(batch_scores, d_s))}
        del batch_scores
    db.free()
    return {"workload": f"query_batch: {nq} queries, lengths uniform [50, 2000] (sum {sum(qlens)}), "
                        f"vs {n:,} sequences ({w.db_residues / 1e6:.0f} M aa), one graph-captured "
                        f"batch per step (a persistent launch per rows-per-thread group)",
            "value": cells / (ms / 1e3) / 1e9, "unit": "GCUPS", "steps": args.batch_steps,
            "ms_per_step": ms / args.batch_steps, "gpu_launches": int(prof["launches"]),
            "launches_per_batch": int(prof["launches"]) // max(1, args.batch_steps),
            "wavefront_launches_per_batch": groups + (1 if singles else 0),
            "queries_alone": singles, "padded_frac": round(padded_frac, 4),
            "loop_same_db": loop,
            "vs_loop_same_db": (cells / (ms / 1e3) / 1e9) / loop["gcups"] if loop else None}


def run_long(args, sw, torch, dev, rank):
    """Long sequences: a 5,478-residue query vs 100,000 sequences (mean 2,000, up to 35,000;
    17 % above 3,000 residues go to the warp-per-pair kernel), with 1,000 planted
    near-duplicates; the second run scales matrix and penalties by 3 so the planted pairs pass the
    16-bit range and are rescored in int32. GCUPS and the per-phase device time."""
    out = []
    # (scale, long tail, sequences, block threshold): the workload, the same x3, and the
    # variant with 64 sequences of 20,000-35,000 residues, with the block route and without,
    # at 100,000 sequences (where no pair unit outgrows a warp's share: the automatic
    # threshold routes nothing, so the route is forced at 20,000) and at 10,000 (where the
    # automatic threshold routes the tail)
    off = sw.SW_BLOCK_ROUTE_OFF
    for scale, tail, n, bt in ((1, 0, 100_000, 0), (3, 0, 100_000, 0), (1, 64, 100_000, 20_000),
                               (1, 64, 100_000, off), (1, 64, 10_000, 0), (1, 64, 10_000, off)):
        w = synth.long_sequences(seed=1408 + 1000 * rank, scale=scale, long_tail=tail, n_seqs=n,
                                 n_planted=1000 * n // 100_000)
        db = sw.sw_db_load(w.residues, w.offsets, alphabet=20, long_threshold=3000,
                           flags=sw.SW_DB_FLAG_PROFILE, block_threshold=bt)
        q = w.queries[0]
        n, k = w.n_seqs, w.top_k
        d_q = torch.from_numpy(q).to(dev)
        d_m = torch.from_numpy(w.matrix.copy()).to(dev)
        d_s = torch.empty(n, dtype=torch.int32, device=dev)
        d_ts = torch.empty(k, dtype=torch.int32, device=dev)
        d_ti = torch.empty(k, dtype=torch.int64, device=dev)
        stream = torch.cuda.Stream(device=dev)

        def step():
            sw.sw_search_device(db, d_q, q.size, d_m, w.alpha, w.beta, k, d_s, d_ts, d_ti, stream)

        step()
        stream.synchronize()
        sw.sw_db_reset_profile(db)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.long_steps):
            step()
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        prof = sw.sw_db_get_profile(db)
        info = db.info()
        planted = w.notes["planted"]
        saturated = int((d_s.cpu().numpy()[planted] > 32767).sum())
        db.free()
        cells = q.size * w.db_residues * args.long_steps
        out.append({"workload": f"{w.name}: one {q.size}-residue query vs {w.n_seqs:,} sequences "
                                f"({w.db_residues / 1e6:.0f} M aa, {info['n_long']:,} above 3,000), "
                                f"{len(planted)} planted near-duplicates"
                                + (", matrix and penalties x3" if scale > 1 else "")
                                + (f", {tail} sequences of 20,000-35,000 aa" if tail else ""),
                    "block_route": ({"threshold": info["block_threshold"],
                                     "sequences": info["n_block"]} if info["n_block"] else None),
                    "value": cells / (ms / 1e3) / 1e9, "unit": "GCUPS", "steps": args.long_steps,
                    "ms_per_step": ms / args.long_steps,
                    "phases_ms": {p: v["ms"] / args.long_steps for p, v in prof["phases"].items()},
                    "gpu_launches": int(prof["launches"]),
                    "planted_above_16_bit": saturated})
    return out


def run_traceback(args, sw, w, db, top_index, qlens):
    """Alignments of the top hits of every query of the 20-query stream through sw_align
    (host buffers, wall clock; the second of two rounds is timed), with the dynamic-programming cells of
    its three passes, and the oracle's traceback of a few of them on the host for scale."""
    import oracle

    k = min(args.align_top, top_index.shape[1])
    idx = [np.ascontiguousarray(top_index[i, :k], dtype=np.uint64) for i in range(len(qlens))]
    off = w.offsets
    for rnd in range(2):
        t0 = time.perf_counter()
        res = [sw.sw_align(db, w.queries[i], w.matrix, w.alpha, w.beta, idx[i])
               for i in range(len(qlens))]
        secs_each = time.perf_counter() - t0
    hits = [(i, int(x)) for i in range(len(qlens)) for x in idx[i]]
    for rnd in range(2):
        t0 = time.perf_counter()
        flat = sw.sw_align_batch(db, w.queries, w.matrix, w.alpha, w.beta, hits)
        secs = time.perf_counter() - t0
    assert flat == [a for r in res for a in r]
    n_al = sum(len(r) for r in res)
    cells = 0
    for i, r in enumerate(res):
        for a in r:
            n = int(off[a["db_index"] + 1] - off[a["db_index"]])
            cells += qlens[i] * n
            if a["score"] > 0:
                cells += a["q_end"] * a["d_end"]  # the anchored pass behind the end cell
                cells += (a["q_end"] - a["q_begin"]) * (a["d_end"] - a["d_begin"])
    # the oracle on the top hit of every query (one core)
    t0 = time.perf_counter()
    for i, r in enumerate(res):
        a = r[0]
        oracle.align(w.queries[i], w.residues[int(off[a["db_index"]]):int(off[a["db_index"] + 1])],
                     w.matrix, w.alpha, w.beta)
    cpu_secs = time.perf_counter() - t0
    gpu_top = None  # the same 20 alignments on the GPU, one call each
    t0 = time.perf_counter()
    for i in range(len(qlens)):
        sw.sw_align(db, w.queries[i], w.matrix, w.alpha, w.beta, idx[i][:1])
    gpu_top = time.perf_counter() - t0
    return {"workload": f"top {k} hits of each of the {len(qlens)} stream queries: one optimal "
                        f"alignment each (score, end and start cells, op string), all in one "
                        f"sw_align_batch call",
            "alignments": n_al, "ms": secs * 1e3, "alignments_per_s": n_al / secs,
            "ms_one_call_per_query": secs_each * 1e3,
            "dp_cells": cells, "gcups": cells / secs / 1e9,
            "mean_ops_len": float(np.mean([len(a["ops"]) for r in res for a in r])),
            "top1_per_query_ms": {"gpu": gpu_top * 1e3, "cpu_oracle_1_core": cpu_secs * 1e3}}


def _serve_rate(sw, db, n_res, rate, n_arrivals, seed, slots, queue):
    """One Poisson stream of n_arrivals queries at `rate` q/s through a fresh server."""
    import threading

    lens = synth.served_query_lengths(n_arrivals, seed)
    qs = synth.make_queries(lens, seed)
    arrive = synth.arrival_times(len(qs), rate, seed)
    srv = sw.sw_server_create(db, max_active=slots, max_queue=queue, slices=8)
    tickets = [None] * len(qs)
    t0 = time.perf_counter()

    def submitter():
        for i, q in enumerate(qs):
            d = arrive[i] - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            try:
                tickets[i] = srv.submit(q, synth.BLOSUM62, 1, 11, 10)
            except sw.SwError as e:
                if e.status != "SW_ERR_BUSY":
                    raise

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, queued, service = [], [], []
    cells = 0
    for i, tk in enumerate(tickets):
        if tk is None:
            continue
        _, _, l = srv.wait(tk)
        lat.append(l["done_ms"] - l["submit_ms"])
        queued.append(l["admit_ms"] - l["submit_ms"])
        service.append(l["done_ms"] - l["admit_ms"])
        cells += int(qs[i].size) * n_res
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.destroy()
    lat = np.array(lat) if lat else np.zeros(1)
    return {"rate_qps": rate, "arrivals": len(qs), "completed": int(st["completed"]),
            "rejected": int(st["rejected"]),
            "p50_s": float(np.percentile(lat, 50)) / 1e3, "p99_s": float(np.percentile(lat, 99)) / 1e3,
            "mean_queue_s": float(np.mean(queued)) / 1e3 if queued else None,
            "mean_service_s": float(np.mean(service)) / 1e3 if service else None,
            "sustained_gcups": cells / wall / 1e9,
            "busy_gcups": cells / (st["busy_ms"] / 1e3) / 1e9 if st["busy_ms"] else None,
            "waves": int(st["waves"]), "wave_ms_mean": st["busy_ms"] / max(1, st["waves"]),
            "wave_host_ms_mean": (st["busy_ms"] - st["gpu_ms"]) / max(1, st["waves"]),
            "wall_s": wall}


def run_served(args, sw, rank):
    """Serving: a resident database of 20,000,000 sequences; Poisson arrivals of queries
    (log-normal lengths, median 300) at the overload rates (10-500 q/s, a fixed number of
    arrivals each, bounded admission with rejections counted) and at the knee rates below one
    GPU's capacity; p50/p99 latency (queueing and service), sustained and busy GCUPS per rate,
    and the host's share of each wave (launches and the wave-end synchronisation)."""
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    knee = [float(r) for r in args.serve_knee.split(",") if r.strip()]
    if not rates and not knee:
        return None
    res, off = synth.make_db(args.serve_seqs, 1407 + 1000 * rank)
    db = sw.sw_db_load(res, off, alphabet=20)
    if not args.no_tune:
        sw.sw_db_autotune(db, synth.BLOSUM62, 1, 11)
    n_res = int(off[-1])
    del res
    out = []
    runs = [(r, args.serve_arrivals) for r in rates] + [(r, args.serve_knee_arrivals) for r in knee]
    for rate, n_arr in runs:
        # each rate's arrival stream and queries depend on the rate alone
        out.append(_serve_rate(sw, db, n_res, rate, n_arr, 1407 + int(round(rate * 100)),
                               args.serve_slots, args.serve_queue))
    db.free()
    return {"workload": f"served_stream: {args.serve_seqs:,} resident sequences "
                        f"({n_res / 1e9:.2f} G aa); Poisson arrivals, query lengths log-normal "
                        f"median 300 [20, 5000]; {args.serve_slots} query slots, queue bound "
                        f"{args.serve_queue} (arrivals beyond it rejected), 8 slices per query",
            "rates": out}


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    w, _, _ = build_workload(args, 0, 1)
    threads = os.cpu_count() or 1
    budget = max(2.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        g, info = cpu_oracle_sample(w, budget, threads)
        if i >= args.warmup:
            vals.append(g)
    v = statistics.median(vals) if vals else 0.0
    line = {
        "impl": "reference", "metric": "GCUPS", "value": v, "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": info["seconds"] * 1e3 if info else None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(w, args, 1),
        "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                         "sample": f"all {len(w.queries)} queries x the first {info['sequences']} "
                                   f"database sequences ({info['residues']} residues) per step"},
        "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1404_4152_gb300 import build as swbuild

    # one rank builds (or finds the build current); the others wait for it
    if rank == 0:
        swbuild.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1404_4152_gb300 as sw

    if world > 1:
        # the scaling runs time the headline search (and its e2e) only; the batched,
        # served, long-sequence and traceback legs are single-GPU measurements
        args.batch_steps, args.serve_rates, args.long_steps, args.align_top = 0, "", 0, 0
        args.serve_knee = ""

    w, full, shard_index = build_workload(args, rank, world)
    db = sw.sw_db_load(w.residues, w.offsets, alphabet=20, device=local, flags=sw.SW_DB_FLAG_PROFILE)
    tuning = None if args.no_tune else sw.sw_db_autotune(db, w.matrix, w.alpha, w.beta)
    n = w.n_seqs
    qlens = [int(q.size) for q in w.queries]
    qoff = np.concatenate([[0], np.cumsum(qlens)]).astype(np.int64)
    d_q = torch.from_numpy(np.concatenate(w.queries)).to(dev)
    d_m = torch.from_numpy(w.matrix.copy()).to(dev)
    d_s = torch.empty(n, dtype=torch.int32, device=dev)
    k = w.top_k
    d_ts = torch.empty((len(qlens), k), dtype=torch.int32, device=dev)
    d_ti = torch.empty((len(qlens), k), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        for i, L in enumerate(qlens):
            sw.sw_search_device(db, d_q.data_ptr() + int(qoff[i]), L, d_m, w.alpha, w.beta, k, d_s,
                                d_ts[i], d_ti[i], stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()

    props = torch.cuda.get_device_properties(dev)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    sw.sw_db_reset_profile(db)
    sampler.start()
    time.sleep(0.4)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = sw.sw_db_get_profile(db)

    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    res_all = torch.tensor([float(w.db_residues)], dtype=torch.float64, device=dev)
    merged = None
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(res_all, op=torch.distributed.ReduceOp.SUM)
    ms_max = float(t.item())
    cells_all = sum(qlens) * int(res_all.item()) * args.steps
    value = cells_all / (ms_max / 1e3) / 1e9
    if full is not None:
        merged = check_sharded_top_k(sw, w, full, shard_index, db, d_ts, d_ti, rank, world)
    # per-query GCUPS (outside the timed region)
    per_query = []
    for i, L in enumerate(qlens):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sw.sw_search_device(db, d_q.data_ptr() + int(qoff[i]), L, d_m, w.alpha, w.beta, k, d_s,
                            d_ts[i], d_ti[i], stream)
        b.record(stream)
        stream.synchronize()
        per_query.append({"qlen": L, "gcups": L * w.db_residues / (a.elapsed_time(b) / 1e3) / 1e9})

    # roofline of the dominant kernel
    ph = prof["phases"]
    dom = "wavefront"  # the search kernel: every DP cell of both length bins
    d = ph[dom]
    mean_ms = d["ms"] / max(1, d["calls"])
    cells_per_launch = d["cells"] / max(1, d["calls"])
    achieved = ALU_OPS_PER_CELL * cells_per_launch / (mean_ms / 1e3) / 1e9  # Gop/s
    nsm = props.multi_processor_count
    sm_mhz = clocks["sm_mhz"] if clocks else 2070.0
    peak = nsm * sm_mhz * 1e6 * ALU_LANES_PER_CLK_SM * S16X2_CELLS_PER_LANE / 1e9
    import hashlib

    src = os.path.join(ROOT, "paper_1404_4152_gb300", "csrc", "sw_wavefront.cu")
    same_kernel = hashlib.sha256(open(src, "rb").read()).hexdigest().startswith(TRAFFIC_SOURCE)
    default_workload = (args.n_seqs == 2_000_000 and args.n_queries == 20 and full is None
                        and world == 1)
    traffic = TRAFFIC_BYTES_PER_LAUNCH if same_kernel and default_workload else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Gop/s",
                "frac": achieved / peak, "traffic": traffic,
                "dram_gbs": traffic / (mean_ms / 1e3) / 1e9 if traffic else None,
                "measured_mix": ({"alu_ops_per_cell": ALU_OPS_PER_CELL_MEASURED,
                                  "frac": achieved / ALU_OPS_PER_CELL * ALU_OPS_PER_CELL_MEASURED / peak}
                                 if same_kernel else None),
                "per_unit": f"{ALU_OPS_PER_CELL} integer ALU lane-ops per DP cell (minimum); "
                            f"{cells_per_launch:.4g} cells per launch, mean launch {mean_ms:.2f} ms",
                "peak_basis": f"{nsm} SMs x {sm_mhz:.0f} MHz (sampled) x {ALU_LANES_PER_CLK_SM} ALU "
                              f"lanes/clk/SM x {S16X2_CELLS_PER_LANE} (s16x2)"}

    # end to end through the host-buffer call
    e2e = None
    if not args.no_e2e:
        pinned_q = [torch.from_numpy(q.copy()).pin_memory() for q in w.queries]
        pinned_s = torch.empty(n, dtype=torch.int32).pin_memory()
        import ctypes

        lib = sw.load_library()
        mat = np.ascontiguousarray(w.matrix, dtype=np.int8)
        ts = np.empty(k, np.int32)
        ti = np.empty(k, np.uint64)
        ntop = ctypes.c_uint32()

        def e2e_step():
            for q in pinned_q:
                rc = lib.sw_search(db.handle, q.data_ptr(), q.numel(), mat.ctypes.data, w.alpha,
                                   w.beta, k, pinned_s.data_ptr(), ts.ctypes.data, ti.ctypes.data,
                                   ctypes.byref(ntop), None)
                if rc != 0:
                    raise sw.SwError(rc, sw.sw_last_error())

        e2e_step()
        barrier()
        e2e_steps = max(1, min(args.steps, 5))  # the same metric; a few steps keep the run short
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        t1 = time.perf_counter()
        tt = torch.tensor([t1 - t0], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": cells_all / args.steps * e2e_steps / float(tt.item()) / 1e9, "unit": "GCUPS",
               "steps": e2e_steps,
               "h2d_bytes_per_step": int(sum(qlens) + len(qlens) * w.matrix.size),
               "d2h_bytes_per_step": int(len(qlens) * (4 * n + 12 * k + 4))}

    served = run_served(args, sw, rank)

    batched = None
    if args.batch_steps > 0:
        batched = run_batched(args, sw, torch, dev, rank)
        batched["vs_plain"] = batched["value"] / (value / world)

    long_seqs = run_long(args, sw, torch, dev, rank) if args.long_steps > 0 else None

    traceback = None
    if args.align_top > 0:
        traceback = run_traceback(args, sw, w, db, d_ti.cpu().numpy(), qlens)

    cpu = None
    if not args.no_cpu and world == 1 and rank == 0:
        threads = os.cpu_count() or 1
        g, info = cpu_oracle_sample(w, args.cpu_seconds, threads)
        cpu = {"value": g, "unit": "GCUPS", "cores": threads, "kind": "oracle",
               "sample": f"all {len(w.queries)} queries x the first {info['sequences']} database "
                         f"sequences ({info['residues']} residues), {info['seconds']:.1f} s"}
        g1, info1 = cpu_oracle_sample(w, max(2.0, args.cpu_seconds / 3), 1)
        cpu["one_thread"] = {"value": g1, "unit": "GCUPS", "cores": 1,
                             "sample": f"all {len(w.queries)} queries x the first "
                                       f"{info1['sequences']} database sequences, "
                                       f"{info1['seconds']:.1f} s"}

    line = {
        "metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if full is not None else "weak", "vs_baseline": None, "dtype": "s16x2",
        "data": "synthetic",
        "config": workload_config(w, args, world, full),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(prof["launches"]),
        "phases_ms": {p: ph[p]["ms"] for p in ph},
        "tuning": tuning,
        "per_query": per_query,
        "context": {"paper_xeon_phi_gcups_max": PAPER_PHI_GCUPS_MAX},
        "traceback": traceback,
        "long_sequences": long_seqs,
        "sharded_top_k": merged,
        "batched_detail": batched,
        "served_detail": served,
        # the headline comparison last, compact, so the end of the line carries it
        "batched": compact_batched(batched),
        "served": compact_served(served),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    db.free()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
