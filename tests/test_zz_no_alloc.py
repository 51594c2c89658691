"""sw_search_noalloc: scoring for callers that may not allocate device memory.

Some callers cannot call cudaMalloc: their application hands all device memory
to its own allocator up front, or they cannot afford the device-wide
synchronisation an allocation can cause. They pass their own device buffers
to sw_search_noalloc, which works in the library's fixed scratch array. This
file checks, through the C ABI, that two calls in a row give exactly the
scores of the regular entry point sw_search, and that inputs too large for the
fixed array are refused with a clear error.

The file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

sw = pytest.importorskip("paper_1404_4152_gb300")
torch = pytest.importorskip("torch")


def _database(n, seed, cap):
    lengths = np.minimum(synth.gen_lengths(n, synth.db_qtable(), seed, 1), cap).astype(np.uint64)
    lengths[::97] = 0  # a few empty sequences
    return synth.gen_residues(lengths, seed, 2), int(lengths.max())


def test_noalloc_matches_sw_search_on_two_calls_in_a_row():
    (res, off), max_len = _database(3000, 123, 2048)
    n = off.size - 1
    # a query over 512 residues (the kernel carries rows between passes in the
    # fixed array) and a short one (a single pass)
    queries = [synth.make_queries([777], 124)[0], synth.make_queries([144], 125)[0]]
    M = synth.BLOSUM62
    with sw.sw_db_load(res, off) as db:
        expected = [sw.sw_search(db, q, M, 1, 11, 0)[0] for q in queries]
    dev = torch.device("cuda:0")
    d_res = torch.from_numpy(res).to(dev)
    d_off = torch.from_numpy(off.astype(np.int64)).to(dev)
    d_m = torch.from_numpy(M.copy()).to(dev)
    d_scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for q, exp in zip(queries, expected):
        d_q = torch.from_numpy(q).to(dev)
        torch.cuda.synchronize()
        sw.sw_search_noalloc(d_q, q.size, d_m, 20, 1, 11, d_res, d_off, n, max_len, d_scores,
                             stream)
        stream.synchronize()
        got = d_scores.cpu().numpy()
        assert np.array_equal(got, exp), np.nonzero(got != exp)[0][:10]


def test_noalloc_rejects_sequences_beyond_its_fixed_scratch():
    (res, off), _ = _database(50, 126, 4000)
    dev = torch.device("cuda:0")
    q = synth.make_queries([600], 127)[0]
    d_q = torch.from_numpy(q).to(dev)
    d_res = torch.from_numpy(res).to(dev)
    d_off = torch.from_numpy(off.astype(np.int64)).to(dev)
    d_m = torch.from_numpy(synth.BLOSUM62.copy()).to(dev)
    d_scores = torch.zeros(off.size - 1, dtype=torch.int32, device=dev)
    with pytest.raises(sw.SwError) as e:
        sw.sw_search_noalloc(d_q, q.size, d_m, 20, 1, 11, d_res, d_off, off.size - 1, 4000,
                             d_scores)
    assert e.value.status == "SW_ERR_INVALID_ARG"
    assert "2048" in str(e.value)
