"""The seeded input generator: determinism, table digests and distribution shape."""
import numpy as np

import synth

# sha256 of the standard database length table (log-normal mean 350, sd 250,
# clipped [10, 5000]); both hosts must build the same table to draw the same data.
DB_QTABLE_SHA256 = "fabc0140d75b4427"


def test_length_table_digest():
    assert synth.qtable_digest(synth.db_qtable()).startswith(DB_QTABLE_SHA256)


def test_blosum62_and_background():
    B = synth.BLOSUM62.astype(int)
    assert B.shape == (20, 20) and (B == B.T).all()
    assert B.min() == -4 and B.max() == 11
    assert (np.diag(B) == B.max(axis=1)).all()  # each residue scores best against itself
    assert int(synth.ROBINSON_WEIGHTS.sum()) == 100000


def test_determinism_and_thread_independence():
    lens = synth.gen_lengths(500, synth.db_qtable(), 7, 1)
    a, oa = synth.gen_residues(lens, 7, 2, nthreads=1)
    b, ob = synth.gen_residues(lens, 7, 2, nthreads=5)
    assert np.array_equal(a, b) and np.array_equal(oa, ob)
    assert a.max() < 20


def test_database_shape():
    lens = synth.gen_lengths(200_000, synth.db_qtable(), 3, 1).astype(np.float64)
    assert lens.min() >= 10 and lens.max() <= 5000
    assert abs(lens.mean() - 350) < 10 and abs(lens.std() - 250) < 20
    res, _ = synth.gen_residues(lens[:20000].astype(np.uint64), 3, 2)
    freq = np.bincount(res, minlength=20) / res.size
    assert np.allclose(freq, synth.ROBINSON_WEIGHTS / 1e5, atol=2e-3)


def test_config_shapes():
    assert synth.stream_query_lengths()[0] == 144 and synth.stream_query_lengths()[-1] == 5478
    w = synth.long_sequences(n_seqs=2000, n_planted=20)
    assert w.queries[0].size == 5478
    pos = w.notes["planted"]
    for p in pos:
        d = w.residues[int(w.offsets[p]):int(w.offsets[p + 1])]
        frac = (d != w.queries[0]).mean()
        assert d.size == 5478 and 0.02 < frac < 0.08
