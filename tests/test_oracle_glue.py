"""Pins of the oracle's realignment against the global ancestor and the glue
(the last steps of Algorithm Sample-Align-D, Section 2.3.3), none of which
re-types its recursion:
  - hand-derived examples (tests/golden/ancestor_glue_tiny.json): a tie, an
    insertion before the first anchor, an anchor no bucket matches;
  - brute force: each bucket's alignment with the ancestor, read back from the
    anchors, is re-scored member pair by member pair and compared with the best
    of all alignments of the bucket's profile with the ancestor, enumerated;
  - invariants of the joined alignment: restricted to one bucket's members it
    is that bucket's alignment; every column holds a residue; all residues
    anchored at one ancestor position share one column, and those columns rise
    with the position; an insertion of slot s lies between anchors s - 1 and s.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth
from test_oracle_gotoh import random_symmetric
from test_oracle_progressive import all_paths, path_score, random_tree, restrict, rows_of

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_examples():
    with open(os.path.join(GOLD, "ancestor_glue_tiny.json")) as f:
        g = json.load(f)
    S = np.array(g["subst"], np.int8).ravel()
    for c in g["cases"]:
        res, offs = synth.pack(c["seqs"])
        r = oracle.ancestor_glue(res, offs, c["bucket_offsets"], c["order"], c["widths"], c["colmap"], c["ga"], S,
                                 g["gap_open"], g["gap_extend"])
        assert r["ga_scores"].tolist() == c["ga_scores"], c["name"]
        assert r["anchors"].tolist() == c["anchors"], c["name"]
        assert r["width"] == c["width"], c["name"]
        assert r["colmap"].tolist() == c["global_colmap"], c["name"]


def path_from_anchors(anchors, lg):
    """The bucket-vs-ancestor columns the anchors imply (M, X = bucket column
    against a gap, Y = ancestor position against a gap)."""
    out, g = [], 0
    for a in anchors:
        if a >= 0:
            out += ["Y"] * (a - g) + ["M"]
            g = a + 1
        else:
            out += ["Y"] * (-a - 1 - g) + ["X"]
            g = -a - 1
    return "".join(out + ["Y"] * (lg - g))


def check_glue(seqs, bo, order, widths, colmap, ga, S, go, ge, r, brute=True):
    p = len(bo) - 1
    rows = rows_of(seqs, bo, order, colmap)          # per bucket: the bucket's alignment
    grows = rows_of(seqs, bo, order, r["colmap"])    # per bucket: the joined columns
    lg = len(seqs[ga])
    col_off = np.concatenate([[0], np.cumsum(widths)]).astype(int)
    used, at_anchor = set(), {}
    for b in range(p):
        nb = bo[b + 1] - bo[b]
        anchors = [int(x) for x in r["anchors"][col_off[b]:col_off[b + 1]]]
        if nb == 0:
            assert r["ga_scores"][b] == 0
            continue
        letters = {u: seqs[order[bo[b] + u]] for u in range(nb)}
        letters["ga"] = seqs[ga]
        P = list(range(nb))
        path = path_from_anchors(anchors, lg)
        assert path.count("M") + path.count("X") == widths[b]
        cols_q = {"ga": list(range(lg))}
        got = path_score(letters, P, ["ga"], rows[b], cols_q, widths[b], lg, path, S, go, ge)
        assert got == r["ga_scores"][b]
        if brute:
            best = max(path_score(letters, P, ["ga"], rows[b], cols_q, widths[b], lg, q, S, go, ge)
                       for q in all_paths(widths[b], lg))
            assert best == r["ga_scores"][b]
        # restricted to the bucket, the joined alignment is the bucket's alignment
        _, mine = restrict(grows[b], P)
        assert mine == {u: rows[b][u] for u in P}
        for u in P:
            for bc, gc in zip(rows[b][u], grows[b][u]):
                used.add(gc)
                a = anchors[bc]
                if a >= 0:
                    assert at_anchor.setdefault(a, gc) == gc
    assert used == set(range(r["width"]))
    keys = sorted(at_anchor)
    assert all(at_anchor[x] < at_anchor[y] for x, y in zip(keys, keys[1:]))
    # an insertion of slot s lies after anchor s - 1 and before anchor s
    for b in range(p):
        anchors = [int(x) for x in r["anchors"][col_off[b]:col_off[b + 1]]]
        for u in range(bo[b + 1] - bo[b]):
            for bc, gc in zip(rows[b][u], grows[b][u]):
                a = anchors[bc]
                if a < 0:
                    s = -a - 1
                    if s - 1 in at_anchor:
                        assert gc > at_anchor[s - 1]
                    if s in at_anchor:
                        assert gc < at_anchor[s]


@pytest.mark.parametrize("seed", range(10))
def test_random_buckets_brute_force(seed):
    rng = random.Random(300 + seed)
    A = rng.choice([2, 3])
    S = random_symmetric(rng, A, -4, 6).astype(np.int64).tolist()
    go, ge = rng.choice([(0, -1), (-3, -1), (-2, -2)])
    sizes = [rng.randint(0, 3) for _ in range(rng.randint(1, 4))]
    seqs, bo, left, right, mo = [], [0], [], [], [0]
    for nb in sizes:
        seqs += [[rng.randrange(A) for _ in range(rng.randint(0, 3))] for _ in range(nb)]
        bo.append(bo[-1] + nb)
        lt, rt = random_tree(rng, nb) if nb > 1 else ([], [])
        left += lt
        right += rt
        mo.append(mo[-1] + max(nb - 1, 0))
    seqs.append([rng.randrange(A) for _ in range(rng.randint(0, 4))])   # an ancestor outside the buckets
    order = list(range(len(seqs) - 1))
    res, offs = synth.pack(seqs)
    flat = np.array(S, np.int8).ravel()
    pr = oracle.progressive(res, offs, bo, order, mo, left, right, flat, go, ge)
    for ga in {len(seqs) - 1, rng.randrange(len(seqs))}:
        r = oracle.ancestor_glue(res, offs, bo, order, pr["widths"], pr["colmap"], ga, flat, go, ge)
        check_glue(seqs, bo, order, pr["widths"].tolist(), pr["colmap"], ga, S, go, ge, r)


def test_invariants_on_synthetic_families():
    w = synth.workload(1)
    rk = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p)
    pt = oracle.partition(rk["key_a"], rk["key_b"], w.p)
    bo, order = pt["bucket_offsets"], pt["order"]
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, bo, order, w.subst, w.gap_open, w.gap_extend)
    t = oracle.guide_trees(bo, so, sc)
    pr = oracle.progressive(w.residues, w.offsets, bo, order, t["merge_offsets"], t["left"], t["right"], w.subst,
                            w.gap_open, w.gap_extend)
    r = oracle.ancestor_glue(w.residues, w.offsets, bo, order, pr["widths"], pr["colmap"], rk["ga"], w.subst,
                             w.gap_open, w.gap_extend)
    seqs = [w.residues[w.offsets[i]:w.offsets[i + 1]].tolist() for i in range(w.n)]
    S = np.array(w.subst, np.int64).reshape(w.alphabet, w.alphabet).tolist()
    check_glue(seqs, bo.tolist(), order.tolist(), pr["widths"].tolist(), pr["colmap"], int(rk["ga"]), S,
               w.gap_open, w.gap_extend, r, brute=False)
    assert r["width"] >= max(pr["widths"])


def test_invariants_at_paper_scale():
    """N = 2000 families, p = 16: the oracle's trees, bucket alignments and the
    joined alignment satisfy the same invariants (each realignment re-scored
    member pair by member pair from its anchors)."""
    w = synth.workload(2)
    rk = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(rk["key_a"], rk["key_b"], w.p)
    bo, order = pt["bucket_offsets"], pt["order"]
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, bo, order, w.subst, w.gap_open, w.gap_extend)
    t = oracle.guide_trees(bo, so, sc)
    pr = oracle.progressive(w.residues, w.offsets, bo, order, t["merge_offsets"], t["left"], t["right"], w.subst,
                            w.gap_open, w.gap_extend)
    r = oracle.ancestor_glue(w.residues, w.offsets, bo, order, pr["widths"], pr["colmap"], rk["ga"], w.subst,
                             w.gap_open, w.gap_extend)
    seqs = [w.residues[w.offsets[i]:w.offsets[i + 1]].tolist() for i in range(w.n)]
    S = np.array(w.subst, np.int64).reshape(w.alphabet, w.alphabet).tolist()
    check_glue(seqs, bo.tolist(), order.tolist(), pr["widths"].tolist(), pr["colmap"], int(rk["ga"]), S,
               w.gap_open, w.gap_extend, r, brute=False)
    assert r["width"] >= max(pr["widths"])
