"""Alignments with traceback against the CPU oracle: sad_align_pairs (the
direction bits of every cell kept) and sad_align_pairs_linear (rows split at
the middle down to 256-row blocks, memory linear in the lengths).

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


@pytest.fixture(params=[False, True], ids=["quadratic", "linear"])
def linear(request):
    return request.param


def check(sad, res, offs, pairs, S, go, ge, device=False, linear=False):
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    r, o, pr = res, offs, pairs
    if device:
        import torch
        r, o, pr = (torch.from_numpy(x).cuda() for x in (res, offs, pairs))
    out = sad.align_pairs(r, o, 20, pr, S, go, ge, linear=linear)
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


def test_family_pairs(sad, linear):
    w = synth.workload(1)
    rng = np.random.default_rng(1)
    pairs = rng.integers(0, w.n, (300, 2))
    check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend, linear=linear)


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_paper_scale_pairs(sad, device, linear):
    w = synth.workload(2)
    rng = np.random.default_rng(2)
    pairs = rng.integers(0, w.n, (200, 2))
    check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend, device=device, linear=linear)


def test_long_sequences_cross_strips(sad, linear):
    """Queries beyond 256 rows run in strips whose boundary rows pass through a
    buffer; in linear space they are split at the middle, up to three levels
    deep (2000 rows -> 1000 -> 500 -> 250), with the shorter sequence as rows."""
    rng = np.random.default_rng(3)
    lens = [257, 300, 511, 512, 513, 1000, 1999, 2000, 1, 2, 40]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    seqs[1][:257] = seqs[0]                       # a related pair
    res, offs = synth.pack(seqs)
    n = len(seqs)
    pairs = [(a, b) for a in range(n) for b in range(n) if (a * 7 + b) % 3 == 0]
    check(sad, res, offs, pairs, synth.subst_matrix(5), -11, -1, linear=linear)


@pytest.mark.parametrize("params", [(-11, -1), (0, -1), (-3, 0), (-40, -7)])
def test_long_gaps_across_the_middle(sad, params):
    """Long insertions and deletions placed across the middle rows, so that the
    optimal path crosses a cut inside a gap run (the crossing that saves one
    opening) at several levels of the split, with either sequence as the rows."""
    go, ge = params
    rng = np.random.default_rng(11)
    a, b, c = (list(rng.integers(0, 20, L)) for L in (700, 400, 900))
    mutate = lambda s: [r if rng.random() > 0.1 else int(rng.integers(0, 20)) for r in s]
    seqs = [a + b + c, mutate(a) + mutate(c), mutate(a + b) + c[:300], b + c, a[:513] + c[:513]]
    res, offs = synth.pack(seqs)
    pairs = [(u, v) for u in range(len(seqs)) for v in range(len(seqs))]
    check(sad, res, offs, pairs, synth.subst_matrix(8), go, ge, linear=True)


def test_every_bucket_pair_at_paper_scale_in_linear_space(sad):
    """Every pair u <= v of every bucket of the N = 2000 workload (the buckets
    of the oracle's partition), aligned in linear space: each score equals the
    oracle's score of that pair, and each alignment re-scores to it column by
    column."""
    import torch
    w = synth.workload(2)
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, want_A=False)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    pairs = sad.bucket_pairs(pt["bucket_offsets"], pt["order"])
    assert len(pairs) == len(sc)
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    out = sad.align_pairs(res, offs, 20, torch.from_numpy(pairs).cuda(), w.subst, w.gap_open, w.gap_extend,
                          linear=True)
    np.testing.assert_array_equal(out["scores"].cpu().numpy(), sc)
    ops = out["ops"].cpu().numpy()
    oo, ol = out["ops_offsets"].cpu().numpy(), out["ops_len"].cpu().numpy()
    bad = []
    for k, (a, b) in enumerate(pairs):
        x, y = w.residues[w.offsets[a]:w.offsets[a + 1]], w.residues[w.offsets[b]:w.offsets[b + 1]]
        cols = ops[oo[k]:oo[k] + ol[k]].tobytes()
        if oracle.alignment_score(x, y, cols, w.subst, w.gap_open, w.gap_extend) != int(sc[k]):
            bad.append(k)
    assert not bad, f"{len(bad)} alignments do not re-score to the optimum, first {bad[:5]}"


def test_empty_and_single_residue(sad, linear):
    seqs = [[], [3], [1, 2], [], [7, 7, 7, 7]]
    res, offs = synth.pack(seqs)
    pairs = [(a, b) for a in range(5) for b in range(5)]
    out = check(sad, res, offs, pairs, synth.subst_matrix(6), -11, -1, linear=linear)
    assert sad.columns(out, 0) == ""                       # empty against empty
    assert sad.columns(out, 4) == "YYYY"                   # empty against 4 residues


@pytest.mark.parametrize("params", [(-11, -1), (0, -1), (-3, 0), (0, 0), (-40, -7)])
def test_gap_costs(sad, params, linear):
    go, ge = params
    rng = np.random.default_rng(abs(go) * 10 + abs(ge))
    seqs = [list(rng.integers(0, 20, L)) for L in rng.integers(0, 120, 30)]
    seqs += [list(rng.integers(0, 20, L)) for L in (300, 600, 257)]  # rows split in linear space
    res, offs = synth.pack(seqs)
    pairs = rng.integers(0, 33, (120, 2))
    check(sad, res, offs, pairs, synth.subst_matrix(7), go, ge, linear=linear)


def test_self_alignment_is_all_matches(sad, linear):
    w = synth.workload(1)
    pairs = [(i, i) for i in range(0, w.n, 5)]
    out = check(sad, w.residues, w.offsets, pairs, w.subst, w.gap_open, w.gap_extend, linear=linear)
    lens = np.diff(w.offsets)
    for k, (i, _) in enumerate(pairs):
        assert sad.columns(out, k) == "M" * int(lens[i])


def test_errors(sad, linear):
    w = synth.workload(1)
    with pytest.raises(sad.SadError) as e:
        sad.align_pairs(w.residues, w.offsets, 20, np.array([[0, 64]], np.int32), w.subst, -11, -1, linear=linear)
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
    fn = lib.sad_align_pairs_linear if linear else lib.sad_align_pairs
    rc = fn(None, ctypes.byref(ss), pairs.ctypes.data, 2, S.ctypes.data, -11, -1, sc.ctypes.data, oo.ctypes.data,
            ops.ctypes.data, 10, ol.ctypes.data, sad.MEM_HOST, None)
    assert rc == sad.SAD_ERANGE
    lens = np.diff(w.offsets)
    assert oo[-1] == lens[0] + lens[1] + lens[2] + lens[3]
