"""GPU guide trees (sad_guide_trees, through the C ABI) against the oracle.

Every output is an integer (cluster ids and the exact pair-sum / size-product
distance of every merge), so the bar is bit-exact, including the order of
tied merges.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def assert_trees_equal(got, want):
    for f in ("merge_offsets", "left", "right", "num", "den"):
        np.testing.assert_array_equal(to_np(got[f]), want[f], err_msg=f)


def test_golden_examples(sad):
    with open(os.path.join(GOLD, "guide_tree_tiny.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases[:2]:
        nb = int(round((np.sqrt(8 * len(c["scores"]) + 1) - 1) / 2))
        t = sad.guide_trees(np.array([0, nb], np.int32), np.array([0, len(c["scores"])], np.int64),
                            np.array(c["scores"], np.int32))
        for f in ("left", "right", "num", "den"):
            assert to_np(t[f]).tolist() == c[f], (c["name"], f)


def random_layout(rng, sizes, lo, hi):
    bo = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    so = np.concatenate([[0], np.cumsum([n * (n + 1) // 2 for n in sizes])]).astype(np.int64)
    sc = rng.integers(lo, hi, int(so[-1])).astype(np.int32)
    return bo, so, sc


@pytest.mark.parametrize("mem", ["host", "device"])
def test_random_buckets_with_many_ties(sad, mem):
    """Scores from a small range: many equal cluster distances, so the tie rule decides."""
    rng = np.random.default_rng(4)
    sizes = [0, 1, 2, 3, 17, 64, 5, 200, 0, 33]
    bo, so, sc = random_layout(rng, sizes, -3, 4)
    want = oracle.guide_trees(bo, so, sc)
    args = (bo, so, sc)
    if mem == "device":
        import torch
        args = tuple(torch.from_numpy(a).cuda() for a in args)
    assert_trees_equal(sad.guide_trees(*args), want)


def test_wide_score_range(sad):
    rng = np.random.default_rng(9)
    bo, so, sc = random_layout(rng, [150, 90, 1, 120], -200000, 200000)
    assert_trees_equal(sad.guide_trees(bo, so, sc), oracle.guide_trees(bo, so, sc))


@pytest.mark.parametrize("lo,hi", [(-20, 21), (-300000, 300000)], ids=["32-bit", "64-bit"])
def test_large_bucket_in_global_memory(sad, lo, hi):
    """A 420-member bucket: its cluster matrix does not fit in shared memory."""
    rng = np.random.default_rng(21)
    bo, so, sc = random_layout(rng, [420, 3], lo, hi)
    assert_trees_equal(sad.guide_trees(bo, so, sc), oracle.guide_trees(bo, so, sc))


def test_paper_scale_buckets(sad):
    """N = 2000 families, p = 16: the trees of the real bucket layout and scores."""
    w = synth.workload(2)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    want = oracle.guide_trees(pt["bucket_offsets"], so, sc)
    assert_trees_equal(sad.guide_trees(pt["bucket_offsets"], so, sc), want)


def test_after_the_device_pipeline(sad):
    """The trees of the pipeline's own device outputs equal the oracle's trees."""
    import torch
    w = synth.workload(1)
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    o = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1)
    total = int(o["score_offsets"][-1].item())
    t = sad.guide_trees(o["bucket_offsets"], o["score_offsets"], o["scores"][:max(total, 1)])
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    assert_trees_equal(t, oracle.guide_trees(pt["bucket_offsets"], so, sc))


def test_bad_layout_is_reported(sad):
    bo = np.array([0, 4], np.int32)
    with pytest.raises(sad.SadError):
        sad.guide_trees(bo, np.array([0, 9], np.int64), np.zeros(9, np.int32))  # 4 members need 10 pairs
