"""Globalized rank (Section 2.3.1: every block sends a sample set to all
blocks and each sequence is ranked against all of them) and the partition on
64-bit integer keys, GPU through the C ABI against the CPU oracle, bit-exact.

The samples, the sums G and the bucket layout are integers; both sides use
the same definition (samples at floor((2j+1) w / (2s)) of the block ordered by
(dloc, index); G_i the sum of floor(a 2^32 / b) over the sample slots).
"""
import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def make_workload(seqs, p, k=3, alphabet=20):
    res, offs = synth.pack(seqs)
    return synth.Workload("adhoc", res, offs, alphabet, synth.subst_matrix(99, alphabet), -11, -1, k, p, 0,
                          alphabet, None)


def check_global(sad, w, s, cap=0, device=False):
    res, offs = w.residues, w.offsets
    if device:
        import torch
        res, offs = torch.from_numpy(res).cuda(), torch.from_numpy(offs).cuda()
    got = sad.kmer_rank(res, offs, w.alphabet, w.k, w.p, cap=cap, kmer_alphabet=w.kmer_alphabet,
                        class_map=w.class_map, global_samples=s)
    want = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, class_map=w.class_map,
                            kmer_alphabet=w.kmer_alphabet, want_A=False)
    np.testing.assert_array_equal(to_np(got["dloc"]), want["dloc"])
    G, smp = oracle.global_rank(w.residues, w.offsets, w.k, w.p, s, want["dloc"], class_map=w.class_map,
                                kmer_alphabet=w.kmer_alphabet)
    np.testing.assert_array_equal(to_np(got["sample_idx"]), smp, err_msg="sample slots")
    np.testing.assert_array_equal(to_np(got["G"]), G, err_msg="G")
    return got, G


@pytest.mark.parametrize("s", [1, 3, 15])
def test_global_rank_small_family(sad, s):
    w = synth.workload(1)
    check_global(sad, w, s)


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_global_rank_paper_scale(sad, device):
    """N = 2000, p = 16, s = p - 1 samples per block (240 sample slots)."""
    w = synth.workload(2)
    check_global(sad, w, w.p - 1, device=device)


@pytest.mark.parametrize("cap", [1, 4])
def test_global_rank_on_the_plane_path(sad, cap):
    """cap > 0: the byte sums are clamped to the cap and the residual adds the rest."""
    rng = np.random.default_rng(10 + cap)
    seqs = [list(rng.integers(0, 4, L)) for L in rng.integers(3, 300, 150)]
    seqs += [[4] * 400, [4, 5] * 200, [1] * 3, []]
    w = make_workload(seqs, p=5, k=2)
    check_global(sad, w, 4, cap=cap)


def test_global_rank_compressed_alphabet(sad):
    w = synth.workload(4, n_override=500)
    check_global(sad, w, 7, cap=4)


def test_global_rank_more_samples_than_members(sad):
    """w_b < s: members are taken more than once and count once per slot."""
    rng = np.random.default_rng(11)
    seqs = [list(rng.integers(0, 20, rng.integers(20, 120))) for _ in range(13)]
    w = make_workload(seqs, p=4)
    check_global(sad, w, 9)


def test_global_rank_empty_blocks_and_short_sequences(sad):
    rng = np.random.default_rng(12)
    seqs = [[], [3], list(rng.integers(0, 20, 40)), [1, 2]]
    w = make_workload(seqs, p=7)   # three empty blocks
    got, _ = check_global(sad, w, 2)
    assert (to_np(got["sample_idx"]).reshape(7, 2)[[0, 2, 4]] == -1).all()


def test_global_rank_every_member_sampled_equals_centralized(sad):
    """s = block size with equal blocks samples every sequence once: G = dcen."""
    w = synth.workload(1)          # N = 64, p = 4: blocks of 16
    got = sad.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, global_samples=16)
    np.testing.assert_array_equal(got["G"], got["dcen"])
    assert sorted(got["sample_idx"].tolist()) == list(range(64))


def test_partition_keys64_random_with_ties(sad):
    rng = np.random.default_rng(13)
    for n, p in ((500, 7), (64, 4), (3, 5), (2000, 16), (1000, 1), (4096, 64), (0, 3)):
        keys = rng.integers(0, 1 << 52, n, dtype=np.uint64)
        keys[rng.random(n) < 0.3] = np.uint64(12345)        # many equal keys
        want = oracle.partition_keys64(keys, p)
        got = sad.partition_keys64(keys, p)
        np.testing.assert_array_equal(got["bucket_offsets"], want["bucket_offsets"])
        np.testing.assert_array_equal(got["order"][:n], want["order"])
        np.testing.assert_array_equal(got["pivot_idx"], want["pivot_idx"])


def test_partition_keys64_extreme_keys(sad):
    keys = np.array([0, (1 << 64) - 1, 1 << 63, 5, (1 << 64) - 1, 0, 1 << 32, (1 << 32) - 1], np.uint64)
    for p in (2, 3, 8):
        want = oracle.partition_keys64(keys, p)
        got = sad.partition_keys64(keys, p)
        np.testing.assert_array_equal(got["bucket_offsets"], want["bucket_offsets"])
        np.testing.assert_array_equal(got["order"], want["order"])


@pytest.mark.parametrize("mem", ["host", "device"])
def test_pipeline_globalized_matches_oracle(sad, mem):
    """The pipeline with global_samples partitions by G and scores those buckets
    (with device arrays the stages write G and the sample slots in place)."""
    w = synth.workload(2)
    s = w.p - 1
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    G, smp = oracle.global_rank(w.residues, w.offsets, w.k, w.p, s, r["dloc"])
    pt = oracle.partition_keys64(G, w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    res, offs = w.residues, w.offsets
    if mem == "device":
        import torch
        res, offs = torch.from_numpy(res).cuda(), torch.from_numpy(offs).cuda()
    o = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1,
                     global_samples=s)
    o = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in o.items()}
    np.testing.assert_array_equal(o["G"][:w.n], G)
    np.testing.assert_array_equal(o["sample_idx"], smp)
    np.testing.assert_array_equal(o["bucket_offsets"], pt["bucket_offsets"])
    np.testing.assert_array_equal(o["order"][:w.n], pt["order"])
    np.testing.assert_array_equal(o["score_offsets"], so)
    np.testing.assert_array_equal(o["scores"][:int(so[-1])], sc)
