"""Pins for the oracle's global affine-gap alignment score.

The paper leaves the per-bucket aligner open (Section 2.3.3: any sequential
method); the score here is the global alignment score with affine gaps, a gap
run of length g costing go + g*ge, end gaps included. These tests do not reuse
the oracle's recursion: they enumerate every alignment by brute force, and use
closed forms and theorems.
"""
import itertools
import random

import numpy as np
import pytest

from paper_0901_2742_gb300 import synth


def all_alignments(m, n):
    """Every alignment of lengths m, n as a column string over M (x_i~y_j),
    X (x_i against a gap) and Y (a gap against y_j)."""
    out = []

    def rec(i, j, cols):
        if i == m and j == n:
            out.append("".join(cols))
            return
        if i < m and j < n:
            cols.append("M"); rec(i + 1, j + 1, cols); cols.pop()
        if i < m:
            cols.append("X"); rec(i + 1, j, cols); cols.pop()
        if j < n:
            cols.append("Y"); rec(i, j + 1, cols); cols.pop()

    rec(0, 0, [])
    return out


def score_alignment(cols, x, y, S, go, ge):
    total, i, j = 0, 0, 0
    for c in cols:
        if c == "M":
            total += int(S[x[i]][y[j]]); i += 1; j += 1
        elif c == "X":
            i += 1
        else:
            j += 1
    for kind, run in itertools.groupby(cols):
        if kind in "XY":
            total += go + ge * len(list(run))
    return total


def brute_force(x, y, S, go, ge):
    return max(score_alignment(a, x, y, S, go, ge) for a in all_alignments(len(x), len(y)))


def delannoy(m, n):
    return sum(__import__("math").comb(m, k) * __import__("math").comb(n, k) * 2 ** k
               for k in range(min(m, n) + 1))


def test_enumerator_counts_delannoy():
    # the enumeration covers every monotone path: the Delannoy numbers
    for m in range(5):
        for n in range(5):
            assert len(all_alignments(m, n)) == delannoy(m, n)
    assert delannoy(6, 6) == 8989


def random_symmetric(rng, A, lo, hi):
    S = np.zeros((A, A), dtype=np.int8)
    for a in range(A):
        for b in range(a, A):
            S[a, b] = S[b, a] = rng.randint(lo, hi)
    return S


@pytest.mark.parametrize("seed", range(4))
def test_gotoh_equals_brute_force(orc, seed):
    rng = random.Random(seed)
    for _ in range(60):
        A = rng.choice([2, 3, 4, 20])
        S = random_symmetric(rng, A, -6, 9)
        go = rng.choice([0, -1, -3, -11])
        ge = rng.choice([0, -1, -2])
        m = rng.randint(0, 5 if seed < 3 else 6)
        n = rng.randint(0, 5 if seed < 3 else 6)
        x = [rng.randrange(A) for _ in range(m)]
        y = [rng.randrange(A) for _ in range(n)]
        assert orc.gotoh(x, y, S, go, ge) == brute_force(x, y, S, go, ge), (x, y, go, ge)


def test_gotoh_adversarial_small(orc):
    # homopolymers and alternating strings, both gap regimes
    S = np.array([[5, -4], [-4, 5]], dtype=np.int8)
    cases = [([0] * 6, [0] * 3), ([0, 1] * 3, [1, 0] * 3), ([0] * 6, [1] * 6), ([1], [0] * 6),
             ([], [1, 1]), ([0, 1, 1, 0, 0, 1], [0, 1])]
    for go, ge in [(-11, -1), (0, -1), (-1, 0), (0, 0)]:
        for x, y in cases:
            assert orc.gotoh(x, y, S, go, ge) == brute_force(x, y, S, go, ge)


def test_empty_closed_forms(orc):
    S = synth.subst_matrix(3)
    assert orc.gotoh([], [], S, -11, -1) == 0
    for n in range(1, 40):
        y = list(synth.uniform_residues(n, n))
        assert orc.gotoh([], y, S, -11, -1) == -11 - n
        assert orc.gotoh(y, [], S, -7, -2) == -7 - 2 * n


def test_single_residue_closed_form(orc):
    # x = (a): either a is matched to some y_j, leaving at most two gap runs
    # (left of j and right of j), or a and y are both gapped (two runs).
    rng = random.Random(5)
    for _ in range(50):
        S = random_symmetric(rng, 20, -4, 11)
        go, ge = rng.choice([-11, -3, 0]), rng.choice([-1, -2])
        n = rng.randint(1, 30)
        y = [rng.randrange(20) for _ in range(n)]
        a = rng.randrange(20)
        run = lambda g: 0 if g == 0 else go + g * ge
        best = (go + ge) + run(n)
        for j in range(n):
            best = max(best, int(S[a][y[j]]) + run(j) + run(n - 1 - j))
        assert orc.gotoh([a], y, S, go, ge) == best


def test_prohibitive_gaps_give_ungapped_score(orc):
    # equal lengths and gap costs larger than any gain: the diagonal alignment wins
    rng = random.Random(6)
    S = synth.subst_matrix(11)
    for _ in range(20):
        m = rng.randint(1, 60)
        x = [rng.randrange(20) for _ in range(m)]
        y = [rng.randrange(20) for _ in range(m)]
        want = sum(int(S[a][b]) for a, b in zip(x, y))
        assert orc.gotoh(x, y, S, -10000, -1) == want


def test_symmetry_and_self_score(orc):
    # Config matrices have every off-diagonal entry <= 3 < 4 <= every diagonal
    # entry, so s(a,b) <= (s(a,a)+s(b,b))/2; with non-positive gap costs the
    # identity alignment is optimal: S(x,x) = sum_i s(x_i,x_i).
    S = synth.subst_matrix(2024)
    rng = random.Random(7)
    for _ in range(12):
        m, n = rng.randint(1, 250), rng.randint(1, 250)
        x = synth.uniform_residues(rng.randrange(1 << 30), m)
        y = synth.uniform_residues(rng.randrange(1 << 30), n)
        assert orc.gotoh(x, y, S, -11, -1) == orc.gotoh(y, x, S, -11, -1)
        assert orc.gotoh(x, x, S, -11, -1) == sum(int(S[a, a]) for a in x)


# ---- alignments (traceback) -------------------------------------------------------

def test_alignment_scorer_matches_the_enumeration(orc):
    """The oracle's column scorer agrees with this file's scorer on every alignment of small pairs."""
    rng = random.Random(11)
    for _ in range(12):
        m, n = rng.randint(0, 4), rng.randint(0, 4)
        x = [rng.randrange(4) for _ in range(m)]
        y = [rng.randrange(4) for _ in range(n)]
        S = random_symmetric(rng, 4, -4, 6)
        go, ge = -rng.randint(0, 6), -rng.randint(0, 3)
        for cols in all_alignments(m, n):
            assert orc.alignment_score(x, y, cols, S, go, ge) == score_alignment(cols, x, y, S, go, ge)


def test_alignment_scorer_rejects_non_alignments(orc):
    S = np.eye(4, dtype=np.int8) * 5
    x, y = [0, 1, 2], [0, 2]
    assert orc.alignment_score(x, y, "MXM", S, -3, -1) == 5 + (-3 - 1) + 5
    for bad in ("MM", "MXMY", "MMMX", "MZM", "XXXYY" + "M"):
        assert orc.alignment_score(x, y, bad, S, -3, -1) is None


@pytest.mark.parametrize("seed", range(3))
def test_traceback_is_optimal_and_valid(orc, seed):
    """The traced alignment consumes both sequences and scores exactly the optimum (brute force for small pairs)."""
    rng = random.Random(100 + seed)
    for _ in range(40):
        m, n = rng.randint(0, 6), rng.randint(0, 6)
        x = [rng.randrange(5) for _ in range(m)]
        y = [rng.randrange(5) for _ in range(n)]
        S = random_symmetric(rng, 5, -4, 8)
        go, ge = -rng.randint(0, 8), -rng.randint(0, 3)
        sc, cols = orc.align(x, y, S, go, ge)
        assert sc == brute_force(x, y, S, go, ge)
        assert score_alignment(cols, x, y, S, go, ge) == sc
        assert cols.count("M") + cols.count("X") == m and cols.count("M") + cols.count("Y") == n


def test_traceback_long_family_pairs(orc):
    w = synth.workload(1)
    res, offs = w.residues, w.offsets
    for a, b in ((0, 1), (2, 40), (5, 5), (63, 7)):
        x, y = res[offs[a]:offs[a + 1]], res[offs[b]:offs[b + 1]]
        sc, cols = orc.align(x, y, w.subst, w.gap_open, w.gap_extend)
        assert sc == orc.gotoh(x, y, w.subst, w.gap_open, w.gap_extend)
        assert orc.alignment_score(x, y, cols, w.subst, w.gap_open, w.gap_extend) == sc
