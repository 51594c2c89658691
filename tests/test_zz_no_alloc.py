"""sw_search_noalloc: scoring for callers that may not allocate device memory.

Some callers cannot call cudaMalloc: their application hands all device memory
to its own allocator up front, or they cannot afford the device-wide
synchronisation an allocation can cause. They pass their own device buffers
to sw_search_noalloc, which works in the library's fixed scratch array. This
file checks, through the C ABI, that calls in a row give exactly the CPU
oracle's scores and the regular entry point sw_search's, across one, two and
four query passes and sequences longer than the fixed rows hold; that the
inputs the kernel cannot score are marked (-1: a sequence longer than the
caller promised; -2: a code outside the alphabet); and that inputs too large
for the fixed array are refused with a clear error.

The file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")
torch = pytest.importorskip("torch")

M = synth.BLOSUM62


def _database(n, seed, cap, floor=0, every=0, long_len=0):
    lengths = synth.gen_lengths(n, synth.db_qtable(), seed, 1).astype(np.uint64)
    lengths = np.clip(lengths, floor, cap)
    if floor == 0:
        lengths[::97] = 0  # a few empty sequences
    if every:
        lengths[3::every] = long_len  # planted long sequences
    return synth.gen_residues(lengths, seed, 2), int(lengths.max())


def _run(q, res, off, max_len, stream=None, alphabet=20):
    dev = torch.device("cuda:0")
    n = off.size - 1
    d_q = torch.from_numpy(q).to(dev)
    d_res = torch.from_numpy(res).to(dev)
    d_off = torch.from_numpy(off.astype(np.int64)).to(dev)
    d_m = torch.from_numpy(M.copy()).to(dev)
    d_scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    stream = stream or torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    sw.sw_search_noalloc(d_q, q.size, d_m, alphabet, 1, 11, d_res, d_off, n, max_len, d_scores,
                         stream)
    stream.synchronize()
    return d_scores.cpu().numpy()


def test_noalloc_matches_oracle_and_sw_search_on_two_calls_in_a_row():
    (res, off), max_len = _database(3000, 123, 2048)
    # a query over 512 residues (the kernel carries rows between passes in the
    # fixed array) and a short one (a single pass), each called twice
    queries = [synth.make_queries([777], 124)[0], synth.make_queries([144], 125)[0]]
    with sw.sw_db_load(res, off) as db:
        regular = [sw.sw_search(db, q, M, 1, 11, 0)[0] for q in queries]
    stream = torch.cuda.Stream(device=torch.device("cuda:0"))
    for q, reg in zip(queries, regular):
        exp = oracle.scores(q, res, off, M, 1, 11)
        assert np.array_equal(reg, exp)
        for _ in range(2):
            got = _run(q, res, off, max_len, stream)
            assert np.array_equal(got, exp), np.nonzero(got != exp)[0][:10]


def test_noalloc_four_passes():
    """A 1,600-residue query: four passes of 512 rows through both halves of the row slots."""
    (res, off), max_len = _database(2000, 130, 2048)
    q = synth.make_queries([1600], 131)[0]
    got = _run(q, res, off, max_len)
    exp = oracle.scores(q, res, off, M, 1, 11)
    assert np.array_equal(got, exp), np.nonzero(got != exp)[0][:10]


def test_noalloc_one_pass_query_against_long_sequences():
    """A query of at most 512 residues takes sequences of any length (no rows are kept)."""
    (res, off), max_len = _database(300, 132, 6000, floor=3000)
    assert max_len > 2048
    q = synth.make_queries([400], 133)[0]
    got = _run(q, res, off, max_len)
    exp = oracle.scores(q, res, off, M, 1, 11)
    assert np.array_equal(got, exp), np.nonzero(got != exp)[0][:10]


def test_noalloc_marks_sequences_longer_than_promised():
    """A two-pass query with max_len understated: the sequences past 2,048 residues get -1,
    every other score is exact."""
    (res, off), true_max = _database(800, 134, 2048, every=40, long_len=2600)
    lengths = np.diff(off)
    assert true_max > 2048 and (lengths <= 2048).sum() > 100
    q = synth.make_queries([700], 135)[0]
    got = _run(q, res, off, 2048)
    long_ = lengths > 2048
    assert np.all(got[long_] == -1)
    exp = oracle.scores(q, res, off, M, 1, 11, which=np.nonzero(~long_)[0])
    assert np.array_equal(got[~long_], exp)


def test_noalloc_marks_codes_outside_the_alphabet():
    """A database code >= alphabet marks its sequence -2; a query code >= alphabet marks
    every score -2 (sw_search rejects such codes when the database is loaded)."""
    (res, off), max_len = _database(400, 136, 2048)
    res = res.copy()
    bad = [5, 17, 200]
    for i in bad:
        if off[i + 1] > off[i]:
            res[int(off[i])] = 20 + i % 12
    q = synth.make_queries([300], 137)[0]
    got = _run(q, res, off, max_len)
    marked = [i for i in bad if off[i + 1] > off[i]]
    assert np.all(got[marked] == -2)
    rest = np.setdiff1d(np.arange(off.size - 1), marked)
    exp = oracle.scores(q, res, off, M, 1, 11, which=rest)
    assert np.array_equal(got[rest], exp)
    qb = q.copy()
    qb[123] = 31
    assert np.all(_run(qb, res, off, max_len) == -2)


def test_noalloc_rejects_sequences_beyond_its_fixed_scratch():
    (res, off), _ = _database(50, 126, 4000)
    dev = torch.device("cuda:0")
    q = synth.make_queries([600], 127)[0]
    d_q = torch.from_numpy(q).to(dev)
    d_res = torch.from_numpy(res).to(dev)
    d_off = torch.from_numpy(off.astype(np.int64)).to(dev)
    d_m = torch.from_numpy(M.copy()).to(dev)
    d_scores = torch.zeros(off.size - 1, dtype=torch.int32, device=dev)
    with pytest.raises(sw.SwError) as e:
        sw.sw_search_noalloc(d_q, q.size, d_m, 20, 1, 11, d_res, d_off, off.size - 1, 4000,
                             d_scores)
    assert e.value.status == "SW_ERR_INVALID_ARG"
    assert "2048" in str(e.value)
