"""Sorted-list (sparse) k-mer path against the CPU oracle, bit-exact.

The path serves k-mer spaces beyond the dense count rows (k = 4, 5 over the
20-letter alphabet) and must give the same numerators, D sums, ancestors, keys,
globalized sums and buckets as the definition, whatever the table sizing
(rows per CTA), the counts above 255 (residual) or degenerate inputs.
"""
import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth

pytestmark = pytest.mark.gpu

SPARSE = -1


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def make_workload(seqs, p, k=3, alphabet=20, seed=99):
    res, offs = synth.pack(seqs)
    return synth.Workload("adhoc", res, offs, alphabet, synth.subst_matrix(seed, alphabet), -11, -1, k, p, 0,
                          alphabet, None)


def check_rank(sad, w, cap=SPARSE, want_A=True, device=False, global_samples=0):
    res, offs = w.residues, w.offsets
    if device:
        import torch
        res, offs = torch.from_numpy(res).cuda(), torch.from_numpy(offs).cuda()
    got = sad.kmer_rank(res, offs, w.alphabet, w.k, w.p, cap=cap, kmer_alphabet=w.kmer_alphabet,
                        class_map=w.class_map, want_A=want_A, global_samples=global_samples)
    want = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, class_map=w.class_map,
                            kmer_alphabet=w.kmer_alphabet, want_A=want_A)
    for f in ("dloc", "dcen", "la", "key_a", "key_b"):
        np.testing.assert_array_equal(to_np(got[f]), want[f], err_msg=f)
    assert int(np.asarray(to_np(got["ga"])).reshape(-1)[0]) == want["ga"]
    if want_A:
        np.testing.assert_array_equal(to_np(got["A"]), want["A"])
    if global_samples:
        G, smp = oracle.global_rank(w.residues, w.offsets, w.k, w.p, global_samples, want["dloc"],
                                    class_map=w.class_map, kmer_alphabet=w.kmer_alphabet)
        np.testing.assert_array_equal(to_np(got["sample_idx"]), smp)
        np.testing.assert_array_equal(to_np(got["G"]), G)
    return got, want


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_sparse_small_family_k3(sad, device):
    check_rank(sad, synth.workload(1), device=device)


def test_sparse_paper_scale_k3(sad):
    """N = 2000, k = 3: the same results as the dense paths (and the oracle)."""
    check_rank(sad, synth.workload(2))


@pytest.mark.parametrize("k", [4, 5])
def test_sparse_large_kmer_space(sad, k):
    """20^4 = 160000 and 20^5 = 3.2e6 k-mers: beyond the dense rows, chosen automatically with cap = 0."""
    w = synth.workload(2, n_override=300)
    w.k, w.p = k, 8
    check_rank(sad, w, cap=0)


def test_sparse_counts_above_255_use_the_residual(sad):
    rng = np.random.default_rng(3)
    seqs = [[4] * 700, [4] * 300 + [5] * 300, [4, 5] * 350, [4] * 260, list(rng.integers(0, 20, 300)),
            [4] * 1000 + list(rng.integers(0, 20, 50)), [5] * 600]
    check_rank(sad, make_workload(seqs, p=2))


def test_sparse_short_empty_and_fewer_than_p(sad):
    rng = np.random.default_rng(1)
    seqs = [[], [3], [1, 2], [1, 2, 3], list(rng.integers(0, 20, 40)), [], list(rng.integers(0, 20, 5)),
            [7, 7, 7]]
    check_rank(sad, make_workload(seqs, p=3))
    check_rank(sad, make_workload(seqs[:3], p=8))


def test_sparse_long_sequences_fewer_rows_per_table(sad):
    """Sequences of several thousand k-mers: the hash table holds fewer than 8 rows per CTA."""
    rng = np.random.default_rng(4)
    lens = [8000, 6000, 5000, 4000, 3000, 7000, 2500, 100, 8194, 1]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    for i in range(1, 4):  # related pairs so the numerators are not all tiny
        seqs[i][:2000] = seqs[0][:2000]
    w = make_workload(seqs, p=3, k=4)
    check_rank(sad, w)


def test_sparse_compressed_alphabet(sad):
    w = synth.workload(4, n_override=400)
    check_rank(sad, w, cap=SPARSE)


def test_sparse_globalized_rank(sad):
    check_rank(sad, synth.workload(1), global_samples=3)
    w = synth.workload(2, n_override=500)
    w.k, w.p = 4, 10
    check_rank(sad, w, cap=0, want_A=False, global_samples=9)


def test_sparse_pipeline_matches_oracle(sad):
    w = synth.workload(2, n_override=600)
    w.k = 4
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    o = sad.pipeline(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, cap=0,
                     mode=1)
    np.testing.assert_array_equal(o["bucket_offsets"], pt["bucket_offsets"])
    np.testing.assert_array_equal(o["order"][:w.n], pt["order"])
    np.testing.assert_array_equal(o["scores"][:int(so[-1])], sc)


def test_sparse_rejects_sequences_beyond_the_limit(sad):
    seqs = [[1] * 20000, [2] * 30]
    w = make_workload(seqs, p=1)
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank(w.residues, w.offsets, 20, 3, 1, cap=SPARSE)
    assert e.value.code == sad.SAD_EINVAL
