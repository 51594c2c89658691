"""Saved database files: sw_db_open rejects what is not a consistent file of this library
before it touches the GPU (CPU tests), and an opened database searches exactly like the
original (GPU test)."""
import os
import struct

import numpy as np
import pytest

import synth

sw = pytest.importorskip("paper_1404_4152_gb300")

HDR = struct.Struct("<8sII QQ II QQQQQQ II")


def _header(**kw):
    f = dict(magic=b"SWGBDB01", version=1, alphabet=20, n_seqs=1, total=5, max_len=5, thr=3000,
             n_tiles=1, n_long_tiles=0, n_long=0, tile_bytes=64, rs=5, rl=0, mll=0, mls=8)
    f.update(kw)
    return HDR.pack(f["magic"], f["version"], f["alphabet"], f["n_seqs"], f["total"], f["max_len"],
                    f["thr"], f["n_tiles"], f["n_long_tiles"], f["n_long"], f["tile_bytes"],
                    f["rs"], f["rl"], f["mll"], f["mls"])


def _open_error(path):
    with pytest.raises(sw.SwError) as ei:
        sw.sw_db_open(path)
    return str(ei.value)


def test_rejects_bad_files_without_gpu(tmp_path):
    assert HDR.size == 96
    assert "cannot open" in _open_error(tmp_path / "missing.db")
    p = tmp_path / "magic.db"
    p.write_bytes(_header(magic=b"NOTADB01") + b"\0" * 200)
    assert "not a database file" in _open_error(p)
    p = tmp_path / "short.db"
    p.write_bytes(b"SWGB")
    assert "not a database file" in _open_error(p)
    p = tmp_path / "tiles.db"
    p.write_bytes(_header(n_tiles=3))
    assert "inconsistent header" in _open_error(p)
    p = tmp_path / "size.db"
    p.write_bytes(_header() + b"\0" * 10)
    assert "size does not match" in _open_error(p)
    # right size, but the sorted ids name sequence 7 of 1
    body = (struct.pack("<I", 5) + struct.pack("<8I", 7, *([0xFFFFFFFF] * 7)) + struct.pack("<I", 8)
            + bytes(64))
    p = tmp_path / "ids.db"
    p.write_bytes(_header() + body)
    assert "bad sorted ids" in _open_error(p)
    # consistent arrays, but lengths that disagree with the header's residue count
    body = (struct.pack("<I", 4) + struct.pack("<8I", 0, *([0xFFFFFFFF] * 7)) + struct.pack("<I", 8)
            + bytes(64))
    p = tmp_path / "sums.db"
    p.write_bytes(_header() + body)
    assert "disagree" in _open_error(p)


@pytest.mark.gpu
def test_saved_database_searches_like_the_original(tmp_path):
    lens = synth.gen_lengths(3000, synth.db_qtable(), 81, 1)
    lens[:5] = [0, 3500, 4000, 1, 3001]
    res, off = synth.gen_residues(lens, 81, 2)
    q = synth.make_queries([260], 82)[0]
    path = str(tmp_path / "db.swgb")
    with sw.sw_db_load(res, off, long_threshold=3000) as db:
        s1, ts1, ti1, _ = sw.sw_search(db, q, synth.BLOSUM62, 1, 11, 10)
        a1 = sw.sw_align(db, q, synth.BLOSUM62, 1, 11, ti1[:3])
        info1 = db.info()
        sw.sw_db_save(db, path)
    assert os.path.getsize(path) > int(off[-1])
    with sw.sw_db_open(path) as db2:
        info2 = db2.info()
        s2, ts2, ti2, _ = sw.sw_search(db2, q, synth.BLOSUM62, 1, 11, 10)
        a2 = sw.sw_align(db2, q, synth.BLOSUM62, 1, 11, ti1[:3])
        rows, _, _, _, _ = sw.sw_search_batch(db2, [q, q[:100]], synth.BLOSUM62, 1, 11, 5,
                                              want_scores=True)
    for k in ("n_seqs", "total_residues", "alphabet", "max_length", "n_long"):
        assert info1[k] == info2[k]
    assert np.array_equal(s1, s2) and np.array_equal(ts1, ts2) and np.array_equal(ti1, ti2)
    assert a1 == a2
    assert np.array_equal(rows[0], s1)
