"""GPU progressive alignment (sad_progressive_align, through the C ABI)
against the oracle.

Every output is an integer (the optimum of every merge, the width of every
merged cluster and the column of every residue), and both sides take the
same fixed tie order, so the bar is bit-exact: one different tie at any merge
would change every later profile and show up in the columns.
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
    for f in ("widths", "merge_scores", "merge_widths", "colmap"):
        np.testing.assert_array_equal(to_np(got[f]), want[f], err_msg=f)


def layout(rng, seqs_per_bucket, tree):
    """Concatenate buckets of sequences; tree(nb) gives (left, right)."""
    seqs, bo, left, right, mo = [], [0], [], [], [0]
    for bucket in seqs_per_bucket:
        nb = len(bucket)
        seqs += bucket
        bo.append(bo[-1] + nb)
        lt, rt = tree(nb) if nb > 1 else ([], [])
        left += lt
        right += rt
        mo.append(mo[-1] + max(nb - 1, 0))
    res, offs = synth.pack(seqs)
    order = np.arange(len(seqs), dtype=np.int32)
    return (res, offs, np.array(bo, np.int32), order, np.array(mo, np.int64), np.array(left, np.int32),
            np.array(right, np.int32))


def run_both(sad, alphabet, args, subst, go, ge, mem="host"):
    res, offs, bo, order, mo, left, right = args
    want = oracle.progressive(res, offs, bo, order, mo, left, right, np.asarray(subst, np.int8).ravel(), go, ge)
    if mem == "device":
        import torch
        args = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args)
    got = sad.progressive_align(*args[:2], alphabet, *args[2:], subst, go, ge)
    return got, want


@pytest.mark.parametrize("name", ["progressive_tiny.json", "progressive_tree3.json"])
def test_golden_example(sad, name):
    with open(os.path.join(GOLD, name)) as f:
        c = json.load(f)
    res, offs = synth.pack(c["seqs"])
    S = np.array(c["subst"], np.int8)
    got = sad.progressive_align(res, offs, c["alphabet"], np.array(c["bucket_offsets"], np.int32),
                                np.array(c["order"], np.int32), np.array(c["merge_offsets"], np.int64),
                                np.array(c["left"], np.int32), np.array(c["right"], np.int32), S, c["gap_open"],
                                c["gap_extend"])
    for f in ("widths", "merge_scores", "merge_widths", "colmap"):
        assert to_np(got[f]).tolist() == c[f], (name, f)


@pytest.mark.parametrize("seed", range(6))
def test_tiny_buckets_on_random_trees(sad, seed, columns):
    """Small alphabets and short sequences: many equal alternatives, so the tie order decides."""
    rng = random.Random(seed)
    A = rng.choice([2, 3, 4])
    S = random_symmetric(rng, A, -4, 6)
    go, ge = rng.choice([(0, -1), (-3, -1), (-2, -2)])
    buckets = [[[rng.randrange(A) for _ in range(rng.randint(0, 6))] for _ in range(rng.randint(0, 9))]
               for _ in range(5)]
    args = layout(rng, buckets, lambda nb: random_tree(rng, nb))
    got, want = run_both(sad, A, args, S, go, ge)
    assert_same(got, want)


@pytest.mark.parametrize("mem", ["host", "device"])
def test_several_strips_and_ragged_tails(sad, mem, columns):
    """Profiles wider than one 128-row strip, widths not multiples of 4 or 128."""
    rng = random.Random(77)
    S = random_symmetric(rng, 20, -4, 11)
    buckets = [[[rng.randrange(20) for _ in range(rng.randint(1, 700))] for _ in range(nb)]
               for nb in (2, 5, 1, 0, 9, 3)]
    buckets[0][0] = []                                      # an empty sequence against a long one
    args = layout(rng, buckets, lambda nb: random_tree(rng, nb))
    got, want = run_both(sad, 20, args, S, -11, -1, mem)
    assert_same(got, want)


def test_strip_wait_that_runs_out_reports_a_timeout_and_the_context_recovers(sad):
    """The strip hand-off wait of the profile DP is the kernel's one device-side
    wait. With a bound of one poll, every strip that has to wait for the strip
    above gives up: the call must return SAD_ETIMEOUT (not hang, not fault, not
    report success), and the same context must then give the exact result once
    the default bound is back."""
    rng = random.Random(5)
    S = random_symmetric(rng, 20, -4, 11)
    buckets = [[[rng.randrange(20) for _ in range(600)] for _ in range(2)] for _ in range(3)]
    args = layout(rng, buckets, lambda nb: random_tree(rng, nb))
    sad.progressive_wait_limit(1)
    try:
        with pytest.raises(sad.SadError) as e:
            sad.progressive_align(*args[:2], 20, *args[2:], S, -11, -1)
        assert e.value.code == sad.SAD_ETIMEOUT, e.value
    finally:
        sad.progressive_wait_limit(0)
    got, want = run_both(sad, 20, args, S, -11, -1)
    assert_same(got, want)


def test_wait_limit_setting_is_checked(sad):
    with pytest.raises(sad.SadError):
        sad.progressive_wait_limit(-1)


def balanced_tree(nb):
    """Pairs neighbours level by level: the last merges join clusters of about nb/2 members."""
    live, left, right, k = list(range(nb)), [], [], 0
    while len(live) > 1:
        nxt = []
        for t in range(0, len(live) - 1, 2):
            a, c = sorted((live[t], live[t + 1]))
            left.append(a)
            right.append(c)
            nxt.append(nb + k)
            k += 1
        if len(live) % 2:
            nxt.append(live[-1])
        live = nxt
    return left, right


def test_large_member_products_take_64_bit_values(sad):
    """A 4096-member bucket on a balanced tree: the root merge pairs 2048 x 2048
    members, whose optimum is beyond 2^31 (the DP runs in 64 bits)."""
    rng = random.Random(5)
    S = random_symmetric(rng, 20, -4, 11)
    fam = [rng.randrange(20) for _ in range(200)]
    bucket = [[x if rng.random() > 0.1 else rng.randrange(20) for x in fam] for _ in range(4096)]
    args = layout(rng, [bucket, bucket[:3]], balanced_tree)
    got, want = run_both(sad, 20, args, S, -11, -1)
    assert_same(got, want)
    assert want["merge_scores"].max() > 2 ** 31


def test_paper_scale_buckets_after_the_device_pipeline(sad):
    """N = 2000 families, p = 16: the pipeline's buckets, the GPU guide trees,
    then every bucket aligned; the oracle runs on the oracle's own layout."""
    import torch
    w = synth.workload(2)
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    o = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, cap=w.cap,
                     kmer_alphabet=w.kmer_alphabet, class_map=w.class_map, mode=1)
    total = int(o["score_offsets"][-1].item())
    t = sad.guide_trees(o["bucket_offsets"], o["score_offsets"], o["scores"][:max(total, 1)])
    got = sad.progressive_align(res, offs, w.alphabet, o["bucket_offsets"], o["order"][:w.n], t["merge_offsets"],
                                t["left"], t["right"], w.subst, w.gap_open, w.gap_extend)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    tr = oracle.guide_trees(pt["bucket_offsets"], so, sc)
    want = oracle.progressive(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], tr["merge_offsets"],
                              tr["left"], tr["right"], w.subst, w.gap_open, w.gap_extend)
    assert_same(got, want)


def test_bad_tree_is_reported(sad):
    res, offs = synth.pack([[0, 1], [1], [0]])
    S = np.eye(2, dtype=np.int8)
    bo, od, mo = np.array([0, 3], np.int32), np.arange(3, dtype=np.int32), np.array([0, 2], np.int64)
    with pytest.raises(sad.SadError):   # merge 1 joins cluster 0 again
        sad.progressive_align(res, offs, 2, bo, od, mo, np.array([0, 0], np.int32), np.array([1, 2], np.int32),
                              S, -3, -1)


def test_columns_setting_is_checked(sad):
    with pytest.raises(sad.SadError):
        sad.progressive_columns(3)
    sad.progressive_columns(0)
