"""Independent references that pin the oracle (none of them calls it).

Each function restates what recurrence (1) of Section II.A scores, by a route
that does not run the recurrence:

- ``brute_force_maximal_runs``: enumerate every local alignment (an op string
  of matches and gap runs) and charge a maximal gap run of length k the affine
  cost beta + (k - 1) * alpha. This is the textbook meaning of the penalties
  named below recurrence (1); it agrees with the recurrence when alpha <= beta.
- ``brute_force_paths``: enumerate every path of recurrence (1)'s own move
  set: a gap may be opened (cost beta) after any move, extended (cost alpha)
  only right after a gap of the same kind. With alpha > beta re-opening is
  cheaper than extending, and the recurrence allows it because E and F read
  H, which already includes E and F.
- ``explicit_gap_dp``: the O(m n (m + n)) formulation that charges a gap of
  length k through the gap-length function w(k) = beta + (k - 1) * alpha
  directly (no E/F state).
- ``kadane_no_gaps``: with gaps too expensive to ever pay, the local score is
  the best maximum-subarray sum over the diagonals of the score grid.
"""
from __future__ import annotations

import numpy as np


def _sub(M, a, b):
    return int(M[int(a)][int(b)])


def brute_force_maximal_runs(q, d, M, alpha, beta) -> int:
    """Best score over every local alignment, gap run of length k costing beta+(k-1)alpha."""
    m, n = len(q), len(d)
    best = 0

    def walk(i, j, last, score):
        # (i, j): residues consumed so far (next match uses q[i], d[j]); last in 'MDI'
        nonlocal best
        if score > best:
            best = score
        if i < m and j < n:
            walk(i + 1, j + 1, "M", score + _sub(M, q[i], d[j]))
        if i < m:  # S1[i] against a gap (vertical move, E)
            walk(i + 1, j, "D", score - (alpha if last == "D" else beta))
        if j < n:  # S2[j] against a gap (horizontal move, F)
            walk(i, j + 1, "I", score - (alpha if last == "I" else beta))

    for i0 in range(m):
        for j0 in range(n):
            walk(i0 + 1, j0 + 1, "M", _sub(M, q[i0], d[j0]))
    return best


def brute_force_paths(q, d, M, alpha, beta) -> int:
    """Best score over every path of recurrence (1)'s move set (open after any move)."""
    m, n = len(q), len(d)
    best = 0

    def walk(i, j, last, score):
        nonlocal best
        if score > best:
            best = score
        if i < m and j < n:
            walk(i + 1, j + 1, "M", score + _sub(M, q[i], d[j]))
        if i < m:
            walk(i + 1, j, "D", score - beta)
            if last == "D":
                walk(i + 1, j, "D", score - alpha)
        if j < n:
            walk(i, j + 1, "I", score - beta)
            if last == "I":
                walk(i, j + 1, "I", score - alpha)

    for i0 in range(m):
        for j0 in range(n):
            walk(i0 + 1, j0 + 1, "M", _sub(M, q[i0], d[j0]))
    return best


def explicit_gap_dp(q, d, M, alpha, beta) -> int:
    """O(m n (m+n)): H[i][j] = max(0, diag + s, max_k H[i-k][j] - w(k), max_k H[i][j-k] - w(k))."""
    m, n = len(q), len(d)
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    w = beta + alpha * np.arange(0, max(m, n) + 1, dtype=np.int64)  # w[k-1] = beta + (k-1)alpha
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            v = max(0, int(H[i - 1, j - 1]) + _sub(M, q[i - 1], d[j - 1]))
            # vertical gaps ending at (i, j): from H[i-k][j], k = 1..i
            col = H[i - 1::-1, j] - w[:i]
            row = H[i, j - 1::-1] - w[:j]
            v = max(v, int(col.max()), int(row.max()))
            H[i, j] = v
    return int(H.max())


def kadane_no_gaps(q, d, M) -> int:
    """max(0, best maximum-subarray sum along any diagonal i - j = const of M[q_i][d_j])."""
    m, n = len(q), len(d)
    best = 0
    for off in range(-(n - 1), m):
        run = 0
        for i in range(m):
            j = i - off
            if 0 <= j < n:
                run = max(0, run + _sub(M, q[i], d[j]))
                best = max(best, run)
    return best


def upper_bound(q, d, M) -> int:
    """min(B(q), B(d)) with B(q) = sum_i max(0, max_r M[q_i][r]), B(d) by columns."""
    Mi = np.asarray(M, dtype=np.int64)
    bq = int(np.maximum(Mi.max(axis=1), 0)[np.asarray(q, dtype=np.int64)].sum()) if len(q) else 0
    bd = int(np.maximum(Mi.max(axis=0), 0)[np.asarray(d, dtype=np.int64)].sum()) if len(d) else 0
    return min(bq, bd)


def ranked_top_k(scores, k):
    """Plain sort: score descending, then index ascending; the first min(k, n)."""
    s = np.asarray(scores, dtype=np.int64)
    order = np.lexsort((np.arange(s.size), -s))
    kk = min(k, s.size)
    return s[order[:kk]].astype(np.int32), order[:kk].astype(np.uint64)


def score_of_ops(q, d, M, alpha, beta, q_begin, d_begin, ops) -> int:
    """Score of one alignment under recurrence (1)'s move set: 'M' adds fsbt, a gap step
    costs beta when it opens a run and min(alpha, beta) when it continues a run of the
    same kind ('I': a query residue against a gap, 'D': a database residue)."""
    i, j, s, prev = q_begin, d_begin, 0, ""
    for op in ops:
        if op == "M":
            s += _sub(M, q[i], d[j])
            i += 1
            j += 1
        elif op == "I":
            s -= min(alpha, beta) if prev == "I" else beta
            i += 1
        else:
            s -= min(alpha, beta) if prev == "D" else beta
            j += 1
        prev = op
    return s


def brute_force_optimal_alignments(q, d, M, alpha, beta):
    """(best score, every optimal alignment as (q_begin, q_end, d_begin, d_end, ops)) over
    all local alignments that begin and end with an aligned pair, enumerated path by path
    with recurrence (1)'s move set (0-based half-open ranges)."""
    m, n = len(q), len(d)
    found = []

    def walk(i0, j0, i, j, ops, last, score):
        if last == "M":
            found.append((score, i0, i, j0, j, ops))
        if i < m and j < n:
            walk(i0, j0, i + 1, j + 1, ops + "M", "M", score + _sub(M, q[i], d[j]))
        if i < m:
            walk(i0, j0, i + 1, j, ops + "I", "I",
                 score - (min(alpha, beta) if last == "I" else beta))
        if j < n:
            walk(i0, j0, i, j + 1, ops + "D", "D",
                 score - (min(alpha, beta) if last == "D" else beta))

    for i0 in range(m):
        for j0 in range(n):
            walk(i0, j0, i0 + 1, j0 + 1, "M", "M", _sub(M, q[i0], d[j0]))
    best = max([0] + [f[0] for f in found])
    return best, [f[1:] for f in found if f[0] == best and best > 0]
