"""The whole method in one binding call (sad.msa: pipeline, guide trees,
progressive alignment, glue, all through the C ABI) against the oracle's
chain of the same steps: bit-exact."""
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


@pytest.mark.parametrize("cfg", [1, 2])
def test_msa_matches_the_oracle_chain(sad, cfg):
    import torch
    w = synth.workload(cfg)
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    got = sad.msa(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, cap=w.cap,
                  kmer_alphabet=w.kmer_alphabet, class_map=w.class_map)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    tr = oracle.guide_trees(pt["bucket_offsets"], so, sc)
    pr = oracle.progressive(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], tr["merge_offsets"],
                            tr["left"], tr["right"], w.subst, w.gap_open, w.gap_extend)
    gl = oracle.ancestor_glue(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], pr["widths"], pr["colmap"],
                              r["ga"], w.subst, w.gap_open, w.gap_extend)
    assert got["ga"] == int(r["ga"])
    np.testing.assert_array_equal(got["bucket_offsets"].cpu().numpy(), pt["bucket_offsets"])
    np.testing.assert_array_equal(got["order"].cpu().numpy(), pt["order"])
    np.testing.assert_array_equal(got["widths"].cpu().numpy(), pr["widths"])
    np.testing.assert_array_equal(got["colmap"].cpu().numpy(), pr["colmap"])
    assert got["width"] == gl["width"]
    np.testing.assert_array_equal(got["global_colmap"].cpu().numpy(), gl["colmap"])


def test_msa_wants_device_arrays(sad):
    w = synth.workload(1)
    with pytest.raises(sad.SadError):
        sad.msa(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend)
