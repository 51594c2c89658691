"""Pins for the CPU oracle: it must agree with references that do not run recurrence (1).

Every check here compares the oracle (``oracle/sw_oracle.c``) with something
other than itself: brute-force enumeration of local alignments, an explicit
gap-length DP, Kadane's algorithm, invariants of the local-alignment score,
and a plain sort for the top-k order. ``test_mutants_are_caught`` plants
plausible mistakes in a copy of the oracle source and checks that these pins
reject each one.
"""
import os
import re
import shutil
import tempfile

import numpy as np
import pytest

import oracle
import synth
from tests import pins

B62 = synth.BLOSUM62


def _rand_seq(rng, n, A):
    return rng.integers(0, A, size=n, dtype=np.uint8)


def _rand_matrix(rng, A, lo=-5, hi=8):
    return rng.integers(lo, hi + 1, size=(A, A)).astype(np.int8)


SCHEMES = [(1, 11), (2, 12), (1, 12), (0, 5), (3, 3), (4, 2), (5, 0), (0, 0), (2, 1)]


def test_linear_space_equals_full_matrix():
    rng = np.random.default_rng(11)
    for _ in range(200):
        A = int(rng.integers(2, 21))
        M = _rand_matrix(rng, A)
        q, d = _rand_seq(rng, int(rng.integers(1, 40)), A), _rand_seq(rng, int(rng.integers(1, 40)), A)
        a, b = SCHEMES[int(rng.integers(len(SCHEMES)))]
        assert oracle.sw_score(q, d, M, a, b) == oracle.sw_score(q, d, M, a, b, full=True)


def _brute_cases(rng, count, max_len, schemes, max_cells=None):
    for _ in range(count):
        A = int(rng.integers(2, 7))
        M = _rand_matrix(rng, A, -4, 6)
        m = int(rng.integers(1, max_len + 1))
        n = int(rng.integers(1, max_len + 1))
        if max_cells and m * n > max_cells:
            n = max(1, max_cells // m)
        a, b = schemes[int(rng.integers(len(schemes)))]
        yield _rand_seq(rng, m, A), _rand_seq(rng, n, A), M, a, b


def test_brute_force_maximal_gap_runs():
    """alpha <= beta: the affine cost of maximal runs is what recurrence (1) optimises."""
    rng = np.random.default_rng(12)
    schemes = [(a, b) for a, b in SCHEMES if a <= b]
    for q, d, M, a, b in _brute_cases(rng, 300, 6, schemes):
        assert oracle.sw_score(q, d, M, a, b) == pins.brute_force_maximal_runs(q, d, M, a, b)


def test_brute_force_eight_residues():
    rng = np.random.default_rng(13)
    for k in range(3):
        q, d = _rand_seq(rng, 8, 4), _rand_seq(rng, 8 if k == 0 else 6, 4)
        M = _rand_matrix(rng, 4, -3, 5)
        assert oracle.sw_score(q, d, M, 1, 3) == pins.brute_force_maximal_runs(q, d, M, 1, 3)
    q = np.array([synth.ALPHABET.index(c) for c in "HEAGAWGH"], dtype=np.uint8)
    d = np.array([synth.ALPHABET.index(c) for c in "PAWHEAE"], dtype=np.uint8)
    assert oracle.sw_score(q, d, B62, 1, 11) == pins.brute_force_maximal_runs(q, d, B62, 1, 11)


def test_brute_force_all_paths_any_penalties():
    """Every path of the recurrence's move set, including alpha > beta, alpha = 0, beta = 0."""
    rng = np.random.default_rng(14)
    for q, d, M, a, b in _brute_cases(rng, 250, 5, SCHEMES):
        assert oracle.sw_score(q, d, M, a, b) == pins.brute_force_paths(q, d, M, a, b)


def test_explicit_gap_length_dp():
    rng = np.random.default_rng(15)
    for i in range(60):
        A = 20 if i % 2 else int(rng.integers(2, 8))
        M = B62 if (i % 4 == 1) else _rand_matrix(rng, A)
        q, d = _rand_seq(rng, int(rng.integers(1, 36)), A), _rand_seq(rng, int(rng.integers(1, 36)), A)
        a, b = SCHEMES[i % len(SCHEMES)]
        assert oracle.sw_score(q, d, M, a, b) == pins.explicit_gap_dp(q, d, M, a, b), (i, a, b)


def test_no_gap_case_is_kadane_per_diagonal():
    rng = np.random.default_rng(16)
    for _ in range(60):
        A = int(rng.integers(2, 21))
        M = _rand_matrix(rng, A, -6, 6)
        q, d = _rand_seq(rng, int(rng.integers(1, 30)), A), _rand_seq(rng, int(rng.integers(1, 30)), A)
        # any gap costs >= 1000 > 30 * 6, so no gapped alignment can win
        assert oracle.sw_score(q, d, M, 1000, 1000) == pins.kadane_no_gaps(q, d, M)


def test_invariants_on_blosum62():
    rng = np.random.default_rng(17)
    B = B62.astype(np.int64)
    # the self-alignment is optimal when every off-diagonal entry is at most the
    # mean of the two diagonal entries and the diagonal is positive
    assert (np.diag(B) > 0).all()
    assert (B <= (np.diag(B)[:, None] + np.diag(B)[None, :]) / 2).all()
    for _ in range(40):
        q = _rand_seq(rng, int(rng.integers(1, 120)), 20)
        d = _rand_seq(rng, int(rng.integers(1, 120)), 20)
        s = oracle.sw_score(q, d, B62, 1, 11)
        assert s >= 0
        assert oracle.sw_score(q, q, B62, 1, 11) == int(B[q, q].sum())
        # swap symmetry (symmetric matrix), reversal, integer scaling
        assert oracle.sw_score(d, q, B62, 1, 11) == s
        assert oracle.sw_score(q[::-1].copy(), d[::-1].copy(), B62, 1, 11) == s
        for c in (2, 3):
            Mc = (B * c).astype(np.int8)
            assert oracle.sw_score(q, d, Mc, c, 11 * c) == c * s
        # appending sequence can only help; the score never exceeds min(B(q), B(d))
        d2 = np.concatenate([d, _rand_seq(rng, int(rng.integers(1, 50)), 20)])
        assert oracle.sw_score(q, d2, B62, 1, 11) >= s
        assert s <= pins.upper_bound(q, d, B62)


def test_swap_symmetry_asymmetric_matrix():
    rng = np.random.default_rng(18)
    for _ in range(80):
        A = int(rng.integers(2, 25))
        M = _rand_matrix(rng, A)
        q, d = _rand_seq(rng, int(rng.integers(1, 60)), A), _rand_seq(rng, int(rng.integers(1, 60)), A)
        a, b = SCHEMES[int(rng.integers(len(SCHEMES)))]
        assert oracle.sw_score(q, d, M, a, b) == oracle.sw_score(d, q, M.T.copy(), a, b)


def test_zero_score_padding_is_invisible():
    """Dummy residues that score zero against everything (Section III.B.1) change nothing."""
    rng = np.random.default_rng(19)
    for _ in range(80):
        A = int(rng.integers(2, 21))
        M = _rand_matrix(rng, A)
        Mp = np.zeros((A + 1, A + 1), dtype=np.int8)
        Mp[:A, :A] = M
        q, d = _rand_seq(rng, int(rng.integers(1, 50)), A), _rand_seq(rng, int(rng.integers(1, 50)), A)
        a, b = SCHEMES[int(rng.integers(len(SCHEMES)))]
        s = oracle.sw_score(q, d, M, a, b)
        pad = lambda x, k, front: np.concatenate([np.full(k, A, np.uint8), x] if front else [x, np.full(k, A, np.uint8)])
        for kq, kd in ((0, 7), (5, 0), (3, 9)):
            assert oracle.sw_score(pad(q, kq, False), pad(d, kd, False), Mp, a, b) == s
            assert oracle.sw_score(pad(q, kq, True), pad(d, kd, True), Mp, a, b) == s


def test_borders_and_empty():
    M = B62
    q = np.array([0, 1, 2], np.uint8)
    assert oracle.sw_score(q, np.zeros(0, np.uint8), M, 1, 11) == 0
    assert oracle.sw_score(np.zeros(0, np.uint8), q, M, 1, 11) == 0
    # one residue: max(0, fsbt)
    for a in range(20):
        for b in range(20):
            assert oracle.sw_score(np.array([a], np.uint8), np.array([b], np.uint8), M, 1, 11) == max(0, int(M[a, b]))


def test_top_k_order_and_ties():
    rng = np.random.default_rng(20)
    for n, k in ((0, 5), (1, 1), (7, 10), (100, 0), (1000, 10), (5000, 1024), (3000, 3000)):
        s = rng.integers(0, 12, size=n).astype(np.int32)  # many ties
        ts, ti = oracle.top_k(s, k)
        es, ei = pins.ranked_top_k(s, k)
        assert np.array_equal(ts, es) and np.array_equal(ti, ei)


def test_search_matches_pairwise():
    w = synth.small_search()
    q = w.queries[0]
    sub = 300
    off = w.offsets[: sub + 1]
    s, ts, ti = oracle.search(q, w.residues, off, w.matrix, w.alpha, w.beta, w.top_k)
    for i in range(0, sub, 17):
        d = w.residues[int(off[i]):int(off[i + 1])]
        assert s[i] == oracle.sw_score(q, d, w.matrix, w.alpha, w.beta, full=True)
    for i in (0, 1, 2):
        d = w.residues[int(off[i]):int(off[i + 1])]
        assert s[i] == pins.explicit_gap_dp(q, d, w.matrix, w.alpha, w.beta)
    es, ei = pins.ranked_top_k(s, w.top_k)
    assert np.array_equal(ts, es) and np.array_equal(ti, ei)


# ---------------------------------------------------------------------------
# Mutation check: every plausible slip in the recurrence must fail some pin.
# ---------------------------------------------------------------------------

MUTANTS = {
    "transposed_fsbt": ("row[S2[j - 1]]", "fsbt[(size_t)S2[j - 1] * A + S1[i - 1]]"),
    "alpha_beta_swapped_in_E": ("max2(E[j] - alpha, H[j] - beta)", "max2(E[j] - beta, H[j] - alpha)"),
    "alpha_beta_swapped_in_F": ("max2(F - alpha, Hleft - beta)", "max2(F - beta, Hleft - alpha)"),
    "no_zero_floor": ("int32_t h = max2(0, diag + (int32_t)row[S2[j - 1]]);",
                      "int32_t h = diag + (int32_t)row[S2[j - 1]];"),
    "E_reads_left": ("max2(E[j] - alpha, H[j] - beta)", "max2(E[j] - alpha, Hleft - beta)"),
    "F_reads_up": ("max2(F - alpha, Hleft - beta)", "max2(F - alpha, H[j] - beta)"),
    "F_dropped": ("h = max2(h, max2(e, f));", "h = max2(h, e);"),
    "E_dropped": ("h = max2(h, max2(e, f));", "h = max2(h, f);"),
    "diag_off_by_one": ("diag = H[j];", "diag = H[j - 1];"),
    "last_column_skipped": ("for (uint32_t j = 1; j <= n; ++j) {\n            const int32_t e",
                            "for (uint32_t j = 1; j < n; ++j) {\n            const int32_t e"),
    "extension_not_charged": ("max2(E[j] - alpha, H[j] - beta)", "max2(E[j], H[j] - beta)"),
}


def _pin_suite(lib) -> bool:
    """True when every pin agrees with the oracle build ``lib``."""
    rng = np.random.default_rng(99)
    sc = lambda q, d, M, a, b: oracle.sw_score(q, d, M, a, b, lib=lib)
    schemes = [(1, 3), (2, 5), (1, 11), (3, 2)]
    for q, d, M, a, b in _brute_cases(rng, 60, 5, schemes):
        if a <= b and sc(q, d, M, a, b) != pins.brute_force_maximal_runs(q, d, M, a, b):
            return False
        if sc(q, d, M, a, b) != pins.brute_force_paths(q, d, M, a, b):
            return False
    for _ in range(15):
        A = int(rng.integers(2, 8))
        M = _rand_matrix(rng, A)
        q, d = _rand_seq(rng, int(rng.integers(1, 25)), A), _rand_seq(rng, int(rng.integers(1, 25)), A)
        if sc(q, d, M, 1, 4) != pins.explicit_gap_dp(q, d, M, 1, 4):
            return False
        if sc(q, d, M, 1, 4) != sc(d, q, M.T.copy(), 1, 4):
            return False
    return True


def test_unmodified_oracle_passes_pin_suite():
    assert _pin_suite(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name):
    src = os.path.join(os.path.dirname(oracle.__file__), "sw_oracle.c")
    text = open(src).read()
    old, new = MUTANTS[name]
    body_start = text.index("int32_t oracle_sw_score(")
    body_end = text.index("int32_t oracle_sw_score_full(")
    body = text[body_start:body_end]
    assert old in body, f"mutation anchor for {name} not found"
    mutated = text[:body_start] + body.replace(old, new, 1) + text[body_end:]
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        p = os.path.join(tmp, "m.c")
        open(p, "w").write(mutated)
        lib = oracle.load(oracle.build(src=p, out=os.path.join(tmp, "libm.so")))
        assert not _pin_suite(lib), f"mutant {name} survived the pins"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
