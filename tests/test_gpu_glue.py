"""GPU realignment against the global ancestor and glue (sad_ancestor_glue,
through the C ABI) against the oracle.

Every output is an integer (each bucket's optimum against the ancestor, the
anchor of every bucket column, the joined width and the joined column of
every residue), both sides take the same tie order, so the bar is bit-exact.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth
from test_oracle_gotoh import random_symmetric
from test_oracle_progressive import random_tree

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


@pytest.fixture(params=[1, 2], ids=["one-column steps", "two-column steps"])
def columns(request, sad):
    """Force the profile DP form for one test (results must not depend on it)."""
    sad.progressive_columns(request.param)
    yield request.param
    sad.progressive_columns(0)


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def assert_same(got, want):
    np.testing.assert_array_equal(to_np(got["ga_scores"]), want["ga_scores"], err_msg="ga_scores")
    np.testing.assert_array_equal(to_np(got["anchors"]), want["anchors"], err_msg="anchors")
    assert got["width"] == want["width"]
    np.testing.assert_array_equal(to_np(got["colmap"]), want["colmap"], err_msg="colmap")


def test_golden_examples(sad):
    with open(os.path.join(GOLD, "ancestor_glue_tiny.json")) as f:
        g = json.load(f)
    S = np.array(g["subst"], np.int8)
    for c in g["cases"]:
        res, offs = synth.pack(c["seqs"])
        r = sad.ancestor_glue(res, offs, g["alphabet"], np.array(c["bucket_offsets"], np.int32),
                              np.array(c["order"], np.int32), np.array(c["widths"], np.int32),
                              np.array(c["colmap"], np.int32), c["ga"], S, g["gap_open"], g["gap_extend"])
        assert to_np(r["ga_scores"]).tolist() == c["ga_scores"], c["name"]
        assert to_np(r["anchors"]).tolist() == c["anchors"], c["name"]
        assert r["width"] == c["width"], c["name"]
        assert to_np(r["colmap"]).tolist() == c["global_colmap"], c["name"]


def random_case(rng, A, nbuckets, max_nb, max_len, ga_len):
    seqs, bo, left, right, mo = [], [0], [], [], [0]
    for _ in range(nbuckets):
        nb = rng.randint(0, max_nb)
        seqs += [[rng.randrange(A) for _ in range(rng.randint(0, max_len))] for _ in range(nb)]
        bo.append(bo[-1] + nb)
        lt, rt = random_tree(rng, nb) if nb > 1 else ([], [])
        left += lt
        right += rt
        mo.append(mo[-1] + max(nb - 1, 0))
    seqs.append([rng.randrange(A) for _ in range(ga_len)])   # an ancestor outside the buckets
    return seqs, bo, left, right, mo


@pytest.mark.parametrize("seed", range(6))
def test_random_buckets(sad, seed, columns):
    """Short sequences over small alphabets (many ties), the ancestor inside or outside the buckets."""
    rng = random.Random(900 + seed)
    A = rng.choice([2, 3, 4])
    S = random_symmetric(rng, A, -4, 6)
    go, ge = rng.choice([(0, -1), (-3, -1), (-2, -2)])
    seqs, bo, left, right, mo = random_case(rng, A, rng.randint(1, 5), 6, 7, rng.randint(0, 8))
    res, offs = synth.pack(seqs)
    order = np.arange(len(seqs) - 1, dtype=np.int32)
    pr = oracle.progressive(res, offs, bo, order, mo, left, right, S.ravel(), go, ge)
    for ga in sorted({len(seqs) - 1, rng.randrange(len(seqs))}):
        want = oracle.ancestor_glue(res, offs, bo, order, pr["widths"], pr["colmap"], ga, S.ravel(), go, ge)
        got = sad.ancestor_glue(res, offs, A, np.array(bo, np.int32), order, pr["widths"], pr["colmap"], ga, S,
                                go, ge)
        assert_same(got, want)


@pytest.mark.parametrize("mem", ["host", "device"])
def test_several_strips(sad, mem, columns):
    """Bucket alignments wider than one 64-row strip against a long ancestor."""
    rng = random.Random(41)
    S = random_symmetric(rng, 20, -4, 11)
    seqs, bo, left, right, mo = random_case(rng, 20, 5, 7, 400, 350)
    res, offs = synth.pack(seqs)
    order = np.arange(len(seqs) - 1, dtype=np.int32)
    pr = oracle.progressive(res, offs, bo, order, mo, left, right, S.ravel(), -11, -1)
    ga = len(seqs) - 1
    want = oracle.ancestor_glue(res, offs, bo, order, pr["widths"], pr["colmap"], ga, S.ravel(), -11, -1)
    args = [res, offs, np.array(bo, np.int32), order, pr["widths"], pr["colmap"]]
    if mem == "device":
        import torch
        args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args]
    got = sad.ancestor_glue(args[0], args[1], 20, args[2], args[3], args[4], args[5], ga, S, -11, -1)
    assert_same(got, want)


def test_paper_scale_after_the_device_pipeline(sad):
    """N = 2000, p = 16: pipeline, guide trees, progressive alignment and the glue
    on the GPU (the pipeline's own global ancestor); the oracle runs the same
    chain on its own layout."""
    import torch
    w = synth.workload(2)
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    o = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1)
    total = int(o["score_offsets"][-1].item())
    t = sad.guide_trees(o["bucket_offsets"], o["score_offsets"], o["scores"][:max(total, 1)])
    pa = sad.progressive_align(res, offs, w.alphabet, o["bucket_offsets"], o["order"][:w.n], t["merge_offsets"],
                               t["left"], t["right"], w.subst, w.gap_open, w.gap_extend)
    ga = int(o["ga"][0].item())
    got = sad.ancestor_glue(res, offs, w.alphabet, o["bucket_offsets"], o["order"][:w.n], pa["widths"],
                            pa["colmap"], ga, w.subst, w.gap_open, w.gap_extend)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    assert int(r["ga"]) == ga
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    tr = oracle.guide_trees(pt["bucket_offsets"], so, sc)
    pr = oracle.progressive(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], tr["merge_offsets"],
                            tr["left"], tr["right"], w.subst, w.gap_open, w.gap_extend)
    want = oracle.ancestor_glue(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], pr["widths"],
                                pr["colmap"], ga, w.subst, w.gap_open, w.gap_extend)
    assert_same(got, want)


def test_column_outside_the_bucket_is_reported(sad):
    res, offs = synth.pack([[0, 1], [1]])
    S = np.eye(2, dtype=np.int8)
    with pytest.raises(sad.SadError):   # a column index beyond the bucket's width of 2
        sad.ancestor_glue(res, offs, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32),
                          np.array([2], np.int32), np.array([0, 1, 5], np.int32), 0, S, -3, -1)
