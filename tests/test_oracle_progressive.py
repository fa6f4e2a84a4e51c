"""Pins of the oracle's progressive alignment (each bucket aligned along its
guide tree, profile against profile; the per-processor aligner of Section
2.3.3), none of which re-types its recursion:
  - a hand-derived example (tests/golden/progressive_tiny.json), with a tie,
    an empty sequence, a one-member and an empty bucket;
  - brute force: every merge of random tiny buckets on random trees is read
    back from the final alignment (a cluster's alignment is the final one
    restricted to its members), re-scored member by member, and compared with
    the best of ALL alignments of its two children, enumerated;
  - a two-member bucket is a pairwise global alignment: its score is the
    Gotoh score, which is itself pinned by brute force;
  - invariants on the synthetic families: every member's residues sit in
    increasing columns, no column is empty, and the root merge re-scores to
    the reported value.
"""
import functools
import json
import os
import random

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth
from test_oracle_gotoh import random_symmetric

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rows_of(seqs, bucket_offsets, order, colmap):
    """Per bucket: {position u: list of final columns of its residues}."""
    out, t = [], 0
    for b in range(len(bucket_offsets) - 1):
        rows = {}
        for u in range(bucket_offsets[b + 1] - bucket_offsets[b]):
            L = len(seqs[order[bucket_offsets[b] + u]])
            rows[u] = [int(x) for x in colmap[t:t + L]]
            t += L
        out.append(rows)
    return out


def restrict(rows, members):
    """The alignment of a member subset: its used columns, renumbered."""
    used = sorted({c for u in members for c in rows[u]})
    idx = {c: i for i, c in enumerate(used)}
    return used, {u: [idx[c] for c in rows[u]] for u in members}


def path_score(letters, P, Q, cols_p, cols_q, wp, wq, path, S, go, ge):
    """Score of aligning alignment P (members -> columns, width wp) with Q by
    the op string path, member pair by member pair: a column pair adds S of
    every residue pair across it; a run of g gap columns costs the member
    count product times (go + g ge)."""
    at_p = [dict() for _ in range(wp)]
    at_q = [dict() for _ in range(wq)]
    for u in P:
        for r, c in enumerate(cols_p[u]):
            at_p[c][u] = letters[u][r]
    for u in Q:
        for r, c in enumerate(cols_q[u]):
            at_q[c][u] = letters[u][r]
    total, i, j, prev = 0, 0, 0, None
    for op in path:
        if op == "M":
            total += sum(S[a][b] for a in at_p[i].values() for b in at_q[j].values())
            i, j = i + 1, j + 1
        else:
            if op != prev:
                total += len(P) * len(Q) * go
            total += len(P) * len(Q) * ge
            if op == "X":
                i += 1
            else:
                j += 1
        prev = op
    assert i == wp and j == wq
    return total


def all_paths(m, n):
    @functools.lru_cache(None)
    def go(i, j):
        if i == 0 and j == 0:
            return [""]
        out = []
        if i > 0 and j > 0:
            out += [p + "M" for p in go(i - 1, j - 1)]
        if i > 0:
            out += [p + "X" for p in go(i - 1, j)]
        if j > 0:
            out += [p + "Y" for p in go(i, j - 1)]
        return out
    return go(m, n)


def check_merges(letters, nb, left, right, scores, widths, rows, S, go, ge, brute=True):
    """Every merge read back from the final alignment `rows` of one bucket."""
    members = {u: [u] for u in range(nb)}
    for k in range(nb - 1):
        a, c = int(left[k]), int(right[k])
        P, Q = members.pop(a), members.pop(c)
        used, merged = restrict(rows, P + Q)
        assert widths[k] == len(used)
        _, cols_p = restrict(rows, P)
        _, cols_q = restrict(rows, Q)
        wp = len({x for u in P for x in rows[u]})
        wq = len({x for u in Q for x in rows[u]})
        in_p = {x for u in P for x in rows[u]}
        in_q = {x for u in Q for x in rows[u]}
        path = "".join("M" if x in in_p and x in in_q else ("X" if x in in_p else "Y") for x in used)
        got = path_score(letters, P, Q, cols_p, cols_q, wp, wq, path, S, go, ge)
        assert got == scores[k], (k, path, got, scores[k])
        if brute:
            best = max(path_score(letters, P, Q, cols_p, cols_q, wp, wq, q, S, go, ge) for q in all_paths(wp, wq))
            assert best == scores[k], (k, best, scores[k])
        members[nb + k] = P + Q


def check_rows(rows, width):
    used = set()
    for cols in rows.values():
        assert all(x < y for x, y in zip(cols, cols[1:]))
        used |= set(cols)
    assert used == set(range(width))


@pytest.mark.parametrize("name", ["progressive_tiny.json", "progressive_tree3.json"])
def test_golden_example(name):
    with open(os.path.join(GOLD, name)) as f:
        c = json.load(f)
    res, offs = synth.pack(c["seqs"])
    r = oracle.progressive(res, offs, c["bucket_offsets"], c["order"], c["merge_offsets"], c["left"], c["right"],
                           np.array(c["subst"]).ravel(), c["gap_open"], c["gap_extend"])
    for f in ("widths", "merge_scores", "merge_widths", "colmap"):
        assert r[f].tolist() == c[f], (name, f)


def random_tree(rng, nb):
    live, left, right = list(range(nb)), [], []
    for k in range(nb - 1):
        a, c = sorted(rng.sample(live, 2))
        live.remove(a)
        live.remove(c)
        live.append(nb + k)
        left.append(a)
        right.append(c)
    return left, right


@pytest.mark.parametrize("seed", range(12))
def test_every_merge_optimal_by_brute_force(seed):
    rng = random.Random(seed)
    A = rng.choice([2, 3, 4])
    S = random_symmetric(rng, A, -4, 6).astype(np.int64).tolist()
    go, ge = rng.choice([(0, -1), (-3, -1), (-2, -2)])
    sizes = [rng.randint(0, 4) for _ in range(3)]
    maxlen = {0: 0, 1: 5, 2: 5, 3: 3, 4: 2}
    seqs, bo, left, right, mo = [], [0], [], [], [0]
    for nb in sizes:
        seqs += [[rng.randrange(A) for _ in range(rng.randint(0, maxlen[nb]))] for _ in range(nb)]
        bo.append(bo[-1] + nb)
        lt, rt = random_tree(rng, nb) if nb > 1 else ([], [])
        left += lt
        right += rt
        mo.append(mo[-1] + max(nb - 1, 0))
    order = list(range(len(seqs)))
    res, offs = synth.pack(seqs)
    flat = np.array(S, np.int8).ravel()
    r = oracle.progressive(res, offs, bo, order, mo, left, right, flat, go, ge)
    all_rows = rows_of(seqs, bo, order, r["colmap"])
    for b, nb in enumerate(sizes):
        rows = all_rows[b]
        check_rows(rows, int(r["widths"][b]))
        letters = {u: seqs[order[bo[b] + u]] for u in range(nb)}
        k0, k1 = mo[b], mo[b + 1]
        check_merges(letters, nb, left[k0:k1], right[k0:k1], r["merge_scores"][k0:k1].tolist(),
                     r["merge_widths"][k0:k1].tolist(), rows, S, go, ge)


@pytest.mark.parametrize("seed", range(4))
def test_two_members_is_the_pairwise_score(seed):
    rng = random.Random(100 + seed)
    S = random_symmetric(rng, 20, -4, 11)
    seqs = [[rng.randrange(20) for _ in range(rng.randint(0, 60))] for _ in range(8)]
    res, offs = synth.pack(seqs)
    bo = [0, 2, 4, 6, 8]
    r = oracle.progressive(res, offs, bo, list(range(8)), [0, 1, 2, 3, 4], [0] * 4, [1] * 4,
                           np.array(S, np.int8).ravel(), -11, -1)
    for b in range(4):
        x, y = seqs[2 * b], seqs[2 * b + 1]
        assert r["merge_scores"][b] == oracle.gotoh(x, y, S, -11, -1)


def test_invariants_on_synthetic_families():
    w = synth.workload(1)
    rk = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p)
    pt = oracle.partition(rk["key_a"], rk["key_b"], w.p)
    bo, order = pt["bucket_offsets"], pt["order"]
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, bo, order, w.subst, w.gap_open, w.gap_extend)
    t = oracle.guide_trees(bo, so, sc)
    r = oracle.progressive(w.residues, w.offsets, bo, order, t["merge_offsets"], t["left"], t["right"], w.subst,
                           w.gap_open, w.gap_extend)
    seqs = [w.residues[w.offsets[i]:w.offsets[i + 1]].tolist() for i in range(w.n)]
    all_rows = rows_of(seqs, bo, order, r["colmap"])
    S = np.array(w.subst, np.int64).reshape(w.alphabet, w.alphabet).tolist()
    for b in range(w.p):
        nb = int(bo[b + 1] - bo[b])
        rows = all_rows[b]
        check_rows(rows, int(r["widths"][b]))
        assert r["widths"][b] >= max(len(v) for v in rows.values())
        letters = {u: seqs[order[bo[b] + u]] for u in range(nb)}
        k0, k1 = int(t["merge_offsets"][b]), int(t["merge_offsets"][b + 1])
        check_merges(letters, nb, t["left"][k0:k1], t["right"][k0:k1], r["merge_scores"][k0:k1].tolist(),
                     r["merge_widths"][k0:k1].tolist(), rows, S, w.gap_open, w.gap_extend, brute=False)
        assert r["merge_widths"][k1 - 1] == r["widths"][b]
