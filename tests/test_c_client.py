"""The C ABI from C: tests/c/search_client.c, built with gcc against include/sw.h and the
library, searches, aligns, saves and reopens a database; its output must agree with the
oracle (GPU test). Building the client needs no GPU and is checked on the CPU."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "search_client.c")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")


def _build(tmp_path):
    from paper_1404_4152_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "search_client")
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return exe


def _inputs():
    # the same database and query the client builds
    N, A = 64, 20
    offsets, res = [0], []
    for s in range(N):
        L = 20 + (s * 37) % 260
        res += [(s * 7 + i * 13 + i // 5) % A for i in range(L)]
        offsets.append(len(res))
    res = np.array(res, np.uint8)
    offsets = np.array(offsets, np.uint64)
    q = res[int(offsets[3]) + 5:int(offsets[3]) + 65].copy()
    M = np.array([[5 if a == b else -(1 + (a + b) % 3) for b in range(A)] for a in range(A)], np.int8)
    return res, offsets, q, M


def test_client_builds(tmp_path):
    assert os.access(_build(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_client_agrees_with_the_oracle(tmp_path):
    exe = _build(tmp_path)
    out = subprocess.run([exe, str(tmp_path / "db.swgb")], capture_output=True, text=True,
                         check=True).stdout
    kv = dict(re.findall(r"(\w+)=(\S+)", out))
    res, off, q, M = _inputs()
    es, ets, eti = oracle.search(q, res, off, M, 1, 11, 5)
    assert int(kv["n_top"]) == 5 and int(kv["top_index"]) == int(eti[0])
    assert int(kv["top_score"]) == int(ets[0]) and int(kv["sum"]) == int(es.sum())
    assert kv["reopened_same"] == "1" and kv["rejected"] == "1"
    e = oracle.align(q, res[int(off[eti[0]]):int(off[eti[0] + 1])], M, 1, 11)
    assert int(kv["align_score"]) == e["score"] and kv["ops"] == e["ops"]
    assert kv["q"] == f"{e['q_begin']}-{e['q_end']}" and kv["d"] == f"{e['d_begin']}-{e['d_end']}"
    assert int(kv["cells"]) == 60 * int(off[-1])
    # every score and every top-k entry, element by element
    assert [int(v) for v in kv["scores"].split(",")] == es.tolist()
    top = [tuple(int(x) for x in e.split(":")) for e in kv["top"].split(",")]
    assert top == list(zip(ets.tolist(), eti.tolist()))
