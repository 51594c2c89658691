"""The bounds-checked build (-DSW_DEBUG_BOUNDS) over every kernel path: results still match
the oracle and no kernel recorded an out-of-bounds access.

The checked library is loaded in a child process (SWGB_DEBUG_BOUNDS=1) so this process
keeps the normal one.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import oracle, synth
import paper_1404_4152_gb300 as sw
from paper_1404_4152_gb300 import build
assert build.lib_path(debug=True) == sw.load_library()._name

def check(db, what):
    site = sw.sw_db_debug_check(db)
    assert site == 0, f"{what}: out-of-bounds access at site {site}"

lens = synth.gen_lengths(2500, synth.db_qtable(), 91, 1)
lens[:6] = [0, 1, 3001, 4100, 7, 3500]
res, off = synth.gen_residues(lens, 91, 2)
M = synth.BLOSUM62
for flags in (0, sw.SW_DB_FLAG_QUERY_PROFILE, sw.SW_DB_FLAG_FORCE_INT32):
    with sw.sw_db_load(res, off, long_threshold=3000, flags=flags) as db:
        for L in (1, 63, 200, 700):
            q = synth.make_queries([L], 92 + L)[0]
            s, ts, ti, _ = sw.sw_search(db, q, M, 1, 11, 10)
            assert np.array_equal(s, oracle.scores(q, res, off, M, 1, 11)), (flags, L)
            check(db, f"search flags={flags} qlen={L}")
        qs = synth.make_queries([120, 333, 50], 93)
        rows, _, _, _, _ = sw.sw_search_batch(db, qs, M, 1, 11, 5, want_scores=True)
        for q, r in zip(qs, rows):
            assert np.array_equal(r, oracle.scores(q, res, off, M, 1, 11))
        check(db, f"batch flags={flags}")
# alphabet above 20: the one-column ring
rng = np.random.default_rng(94)
A = 28
MA = rng.integers(-5, 7, size=(A, A)).astype(np.int8)
resA = rng.integers(0, A, size=res.size).astype(np.uint8)
qA = rng.integers(0, A, size=300).astype(np.uint8)
with sw.sw_db_load(resA, off, alphabet=A) as db:
    s, _, _, _ = sw.sw_search(db, qA, MA, 2, 9, 10)
    assert np.array_equal(s, oracle.scores(qA, resA, off, MA, 2, 9))
    check(db, "alphabet 28")
# saturation: int32 rescoring; then alignments
q = synth.make_queries([900], 95)[0]
seqs = [synth.mutate(q, 95, 0, k, 300) for k in range(3)] + [synth.make_queries([400], 96)[0]]
resS = np.concatenate(seqs)
offS = np.zeros(len(seqs) + 1, np.uint64)
offS[1:] = np.cumsum([x.size for x in seqs])
M8 = (M.astype(np.int32) * 8).astype(np.int8)
with sw.sw_db_load(resS, offS) as db:
    s, _, _, st = sw.sw_search(db, q, M8, 8, 88, 4)
    assert st["recomputed"] > 0 and np.array_equal(s, oracle.scores(q, resS, offS, M8, 8, 88))
    check(db, "rescoring")
    al = sw.sw_align(db, q, M8, 8, 88, np.arange(4, dtype=np.uint64))
    for a, d in zip(al, seqs):
        e = oracle.align(q, d, M8, 8, 88)
        assert all(a[k] == e[k] for k in e)
    check(db, "alignment")
print("debug-bounds ok")
'''


def test_bounds_checked_build_runs_clean():
    from paper_1404_4152_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, SWGB_DEBUG_BOUNDS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug-bounds ok" in r.stdout
