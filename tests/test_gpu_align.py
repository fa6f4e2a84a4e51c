"""Alignments with traceback (sad_align_pairs) against the CPU oracle.

Several alignments can share the optimal score, so the test compares what is
unique, the score (equal to the oracle's optimum), and checks that the rest is
valid: the columns consume both sequences exactly, and scoring them column by
column (the oracle's alignment scorer, no dynamic programming) gives that score.
"""
import ctypes

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


def check(sad, res, offs, pairs, S, go, ge, device=False):
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    r, o, pr = res, offs, pairs
    if device:
        import torch
        r, o, pr = (torch.from_numpy(x).cuda() for x in (res, offs, pairs))
    out = sad.align_pairs(r, o, 20, pr, S, go, ge)
    scores = out["scores"].cpu().numpy() if device else out["scores"]
    lens = np.diff(offs)
    oo = out["ops_offsets"].cpu().numpy() if device else out["ops_offsets"]
    np.testing.assert_array_equal(oo, np.concatenate([[0], np.cumsum(lens[pairs].sum(axis=1))]))
    for k, (a, b) in enumerate(pairs):
        x, y = res[offs[a]:offs[a + 1]], res[offs[b]:offs[b + 1]]
        want = oracle.gotoh(x, y, S, go, ge)
        assert int(scores[k]) == want, (k, a, b)
        cols = sad.columns(out, k)
        assert oracle.alignment_score(x, y, cols, S, go, ge) == want, (k, a, b, cols)
    return out


def test_family_pairs(sad):
    w = synth.workload(1)
    rng = np.random.default_rng(1)
    pairs = rng.integers(0, w.n, (300, 2))
    check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend)


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_paper_scale_pairs(sad, device):
    w = synth.workload(2)
    rng = np.random.default_rng(2)
    pairs = rng.integers(0, w.n, (200, 2))
    check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend, device=device)


def test_long_sequences_cross_strips(sad):
    """Queries beyond 256 rows run in strips whose boundary rows pass through a buffer."""
    rng = np.random.default_rng(3)
    lens = [257, 300, 511, 512, 513, 1000, 1999, 2000, 1, 2, 40]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    seqs[1][:257] = seqs[0]                       # a related pair
    res, offs = synth.pack(seqs)
    n = len(seqs)
    pairs = [(a, b) for a in range(n) for b in range(n) if (a * 7 + b) % 3 == 0]
    check(sad, res, offs, pairs, synth.subst_matrix(5), -11, -1)


def test_empty_and_single_residue(sad):
    seqs = [[], [3], [1, 2], [], [7, 7, 7, 7]]
    res, offs = synth.pack(seqs)
    pairs = [(a, b) for a in range(5) for b in range(5)]
    out = check(sad, res, offs, pairs, synth.subst_matrix(6), -11, -1)
    assert sad.columns(out, 0) == ""                       # empty against empty
    assert sad.columns(out, 4) == "YYYY"                   # empty against 4 residues


@pytest.mark.parametrize("params", [(-11, -1), (0, -1), (-3, 0), (0, 0), (-40, -7)])
def test_gap_costs(sad, params):
    go, ge = params
    rng = np.random.default_rng(abs(go) * 10 + abs(ge))
    seqs = [list(rng.integers(0, 20, L)) for L in rng.integers(0, 120, 30)]
    res, offs = synth.pack(seqs)
    pairs = rng.integers(0, 30, (80, 2))
    check(sad, res, offs, pairs, synth.subst_matrix(7), go, ge)


def test_self_alignment_is_all_matches(sad):
    w = synth.workload(1)
    pairs = [(i, i) for i in range(0, w.n, 5)]
    out = check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend)
    lens = np.diff(w.offsets)
    for k, (i, _) in enumerate(pairs):
        assert sad.columns(out, k) == "M" * int(lens[i])


def test_errors(sad):
    w = synth.workload(1)
    with pytest.raises(sad.SadError) as e:
        sad.align_pairs(w.residues, w.offsets, 20, np.array([[0, 64]], np.int32), w.subst, -11, -1)
    assert e.value.code == sad.SAD_EINVAL
    # capacity too small: SAD_ERANGE with the offsets filled
    lib = sad.load()
    ss = sad._seqset(w.residues, w.offsets, 20)
    pairs = np.array([0, 1, 2, 3], np.int32)
    sc = np.zeros(2, np.int32)
    oo = np.zeros(3, np.int64)
    ops = np.zeros(10, np.uint8)
    ol = np.zeros(2, np.int32)
    S = np.ascontiguousarray(w.subst, np.int8)
    rc = lib.sad_align_pairs(None, ctypes.byref(ss), pairs.ctypes.data, 2, S.ctypes.data, -11, -1,
                             sc.ctypes.data, oo.ctypes.data, ops.ctypes.data, 10, ol.ctypes.data, sad.MEM_HOST,
                             None)
    assert rc == sad.SAD_ERANGE
    lens = np.diff(w.offsets)
    assert oo[-1] == lens[0] + lens[1] + lens[2] + lens[3]
