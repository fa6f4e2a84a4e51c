"""Pins of the oracle's per-bucket guide tree (average linkage on the pair
scores; the first step of the progressive aligner run on each bucket,
Section 2.3.3), none of which re-types its formula:
  - hand-derived examples (tests/golden/guide_tree_tiny.json), one with a tie;
  - scipy's average linkage (an independent library routine) on tie-free
    random distance matrices: same merges, same distances, same sizes;
  - invariants on the synthetic families: merge distances never decrease,
    every cluster but the root is a child exactly once, and each merge
    distance is the mean of d over the two clusters' member pairs, recounted
    from explicit membership lists.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tri(nb):
    return [(u, v) for u in range(nb) for v in range(u, nb)]


def test_golden_examples():
    with open(os.path.join(GOLD, "guide_tree_tiny.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases[:2]:
        nb = int(round((np.sqrt(8 * len(c["scores"]) + 1) - 1) / 2))
        t = oracle.guide_trees(np.array([0, nb], np.int32), np.array([0, len(c["scores"])]),
                               np.array(c["scores"], np.int32))
        for f in ("left", "right", "num", "den"):
            assert t[f].tolist() == c[f], (c["name"], f)
    # one member, and an empty bucket, have no merges
    t = oracle.guide_trees(np.array([0, 1, 1], np.int32), np.array([0, 1, 1]), np.array([7], np.int32))
    assert t["merge_offsets"].tolist() == [0, 0, 0] and len(t["left"]) == 0


@pytest.mark.parametrize("seed", range(6))
def test_matches_scipy_average_linkage(seed):
    hierarchy = pytest.importorskip("scipy.cluster.hierarchy")
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(2, 40))
    # self scores 0 and distinct pair scores: d_uv = -2 S_uv, all different
    vals = rng.choice(10 ** 6, size=nb * (nb - 1) // 2, replace=False) + 1
    scores, k = [], 0
    cond = []
    for u, v in tri(nb):
        if u == v:
            scores.append(0)
        else:
            scores.append(-int(vals[k]))
            cond.append(2.0 * vals[k])
            k += 1
    t = oracle.guide_trees(np.array([0, nb], np.int32), np.array([0, len(scores)]), np.array(scores, np.int32))
    Z = hierarchy.linkage(np.array(cond), method="average")
    sizes = {i: 1 for i in range(nb)}
    for m in range(nb - 1):
        a, b, dist, cnt = Z[m]
        assert sorted((int(a), int(b))) == [t["left"][m], t["right"][m]], m
        assert t["num"][m] / t["den"][m] == pytest.approx(dist, rel=1e-12)
        sizes[nb + m] = sizes[int(a)] + sizes[int(b)]
        assert sizes[nb + m] == int(cnt)
        assert t["den"][m] == sizes[int(a)] * sizes[int(b)]


def test_invariants_on_families():
    w = synth.workload(1)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    bo = pt["bucket_offsets"]
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, bo, pt["order"], w.subst, w.gap_open,
                                       w.gap_extend)
    t = oracle.guide_trees(bo, so, sc)
    for b in range(w.p):
        nb = int(bo[b + 1] - bo[b])
        m0, m1 = int(t["merge_offsets"][b]), int(t["merge_offsets"][b + 1])
        assert m1 - m0 == max(nb - 1, 0)
        S = {}
        for (u, v), s in zip(tri(nb), sc[so[b]:so[b + 1]]):
            S[u, v] = S[v, u] = int(s)
        d = lambda u, v: S[u, u] + S[v, v] - 2 * S[u, v]
        members = {i: [i] for i in range(nb)}
        used = set()
        last = None
        for m in range(m0, m1):
            a, c = int(t["left"][m]), int(t["right"][m])
            assert a < c and a not in used and c not in used and a in members and c in members
            used.update((a, c))
            pairs = [(u, v) for u in members[a] for v in members[c]]
            assert t["num"][m] == sum(d(u, v) for u, v in pairs) and t["den"][m] == len(pairs)
            h = Fraction(int(t["num"][m]), int(t["den"][m]))
            assert last is None or h >= last  # average linkage never merges closer later
            last = h
            members[nb + m - m0] = members.pop(a) + members.pop(c)
        assert len(members) == min(nb, 1)
