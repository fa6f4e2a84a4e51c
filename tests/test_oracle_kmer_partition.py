"""Pins for the oracle's k-mer rank stage and regular-sampling partition.

k-mer similarity (Section 2, r_ij): a_ij = sum over k-mers of the smaller
count, b_ij = min(|x_i|, |x_j|) - k + 1. Checked against an independent
brute force (sorted k-mer tuples, multiset intersection by a two-pointer
merge), the invariants F(x,x) = 1, symmetry and 0 <= a <= b, and hand-worked
examples (tests/golden). Redistribution (Section 2.3.2) is checked by its
defining properties and a hand-worked example.
"""
import json
import os
import random
from collections import Counter

import numpy as np
import pytest

from paper_0901_2742_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def kmer_tuples(seq, k, class_map=None):
    s = [class_map[r] if class_map is not None else r for r in seq]
    return sorted(tuple(s[t:t + k]) for t in range(len(s) - k + 1))


def multiset_intersection_size(a, b):
    i = j = c = 0
    while i < len(a) and j < len(b):
        if a[i] == b[j]:
            c += 1; i += 1; j += 1
        elif a[i] < b[j]:
            i += 1
        else:
            j += 1
    return c


def split(res, offs):
    return [list(res[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)]


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", load("kmer_rank_tiny.json"), ids=lambda c: c["name"])
def test_golden_kmer_rank(orc, case):
    res, offs = synth.pack(case["seqs"])
    r = orc.kmer_rank(res, offs, case["alphabet"], case["k"], case["p"], class_map=case["class_map"],
                      kmer_alphabet=case["kmer_alphabet"])
    assert r["A"].tolist() == case["A"]
    assert r["dcen"].tolist() == case["dcen"]
    assert r["dloc"].tolist() == case["dloc"]
    assert r["la"].tolist() == case["la"]
    assert r["ga"] == case["ga"]
    assert r["key_a"].tolist() == case["key_a"]
    assert r["key_b"].tolist() == case["key_b"]
    pt = orc.partition(r["key_a"], r["key_b"], case["p"])
    assert pt["pivot_idx"].tolist() == case["pivot_idx"]
    assert pt["bucket_offsets"].tolist() == case["bucket_offsets"]
    assert pt["order"].tolist() == case["order"]
    if "scores" in case:
        sp = case["scores_params"]
        so, sc = orc.bucket_pair_scores(res, offs, pt["bucket_offsets"], pt["order"],
                                        np.array(sp["subst"], np.int8), sp["gap_open"],
                                        sp["gap_extend"])
        assert so.tolist() == case["score_offsets"]
        assert sc.tolist() == case["scores"]


@pytest.mark.parametrize("case", load("psrs_tiny.json"), ids=lambda c: c["name"])
def test_golden_psrs(orc, case):
    pt = orc.partition(case["key_a"], case["key_b"], case["p"])
    assert pt["pivot_idx"].tolist() == case["pivot_idx"]
    assert pt["bucket_offsets"].tolist() == case["bucket_offsets"]
    assert pt["order"].tolist() == case["order"]


@pytest.mark.parametrize("k,cm", [(1, None), (2, None), (3, None), (4, "six"), (5, None)])
def test_kmer_matrix_brute_force(orc, k, cm):
    rng = random.Random(k)
    A = 20
    class_map = synth.compressed_class_map() if cm == "six" else None
    ka = 6 if cm == "six" else A
    seqs = []
    for t in range(14):
        L = rng.choice([0, 1, k - 1, k, k + 1, rng.randint(5, 90)])
        base = synth.uniform_residues(100 + t, max(L, 0), A if t % 3 else 3)
        seqs.append(list(base))
    res, offs = synth.pack(seqs)
    r = orc.kmer_rank(res, offs, A, k, 3, class_map=class_map, kmer_alphabet=ka)
    tup = [kmer_tuples(s, k, class_map) for s in seqs]
    n = len(seqs)
    for i in range(n):
        for j in range(n):
            assert r["A"][i, j] == multiset_intersection_size(tup[i], tup[j])
    # the oracle's histograms against a Counter of tuples
    hist = orc.kmer_histograms(res, offs, k, ka, class_map)
    for i in range(n):
        got = {int(c): int(v) for s, c, v in hist if s == i}
        want = Counter(tup[i])
        assert sorted(got.values()) == sorted(want.values())
        assert sum(got.values()) == max(0, len(seqs[i]) - k + 1)


def test_kmer_invariants_on_families(orc):
    w = synth.workload(1)
    r = orc.kmer_rank(w.residues, w.offsets, 20, w.k, w.p)
    A = r["A"].astype(np.int64)
    L = w.lengths()
    B = np.minimum(L[:, None], L[None, :]) - w.k + 1
    assert (A == A.T).all()
    assert (A >= 0).all() and (A <= B).all()
    assert (np.diag(A) == L - w.k + 1).all()          # F(x, x) = 1
    # ancestors: LA in its block, GA one of the LAs, GA's key is F = 1
    n, p = w.n, w.p
    for b in range(p):
        lo, hi = b * n // p, (b + 1) * n // p
        assert lo <= r["la"][b] < hi
        assert r["dloc"][r["la"][b]] == r["dloc"][lo:hi].max()
    assert r["ga"] in r["la"].tolist()
    assert r["key_a"][r["ga"]] == r["key_b"][r["ga"]]
    # the fixed-point self term is exactly 2^32 in both sums
    assert (r["dcen"] >= (1 << 32)).all() and (r["dloc"] >= (1 << 32)).all()


def test_identical_sequences_tie_breaks(orc):
    # every F = 1: LA = first index of each block, GA = 0, all keys tie and the
    # index decides the order
    seqs = [[3, 1, 4, 1, 5, 9, 2, 6]] * 11
    res, offs = synth.pack(seqs)
    r = orc.kmer_rank(res, offs, 20, 3, 4)
    assert r["la"].tolist() == [0, 2, 5, 8]
    assert r["ga"] == 0
    assert (r["dcen"] == 11 * (1 << 32)).all()
    pt = orc.partition(r["key_a"], r["key_b"], 4)
    check_partition(r["key_a"], r["key_b"], 4, pt)


def test_short_sequences_get_zero_key(orc):
    seqs = [[1, 2], [1, 2, 3, 4], [5], [], [1, 2, 3]]
    res, offs = synth.pack(seqs)
    r = orc.kmer_rank(res, offs, 20, 3, 2)
    for i, s in enumerate(seqs):
        if len(s) < 3:
            assert (r["key_a"][i], r["key_b"][i]) == (0, 1)
            assert r["A"][i].sum() == 0


def test_invalid_inputs_rejected(orc):
    res, offs = synth.pack([[1, 2, 25]])
    with pytest.raises(ValueError):
        orc.kmer_rank(res, offs, 20, 3, 2)
    res, offs = synth.pack([[1, 2, 3]])
    with pytest.raises(ValueError):
        orc.kmer_rank(res, offs, 20, 0, 2)
    with pytest.raises(ValueError):
        orc.kmer_rank(res, offs, 20, 3, 0)


def key_less(ka, kb, i, j):
    lhs, rhs = int(ka[i]) * int(kb[j]), int(ka[j]) * int(kb[i])
    return lhs < rhs if lhs != rhs else i < j


def check_partition(ka, kb, p, pt):
    n = len(ka)
    bo, order = pt["bucket_offsets"], pt["order"]
    assert bo[0] == 0 and bo[-1] == n and (np.diff(bo) >= 0).all()
    assert sorted(order.tolist()) == list(range(n))          # every sequence exactly once
    for b in range(p):
        members = order[bo[b]:bo[b + 1]].tolist()
        assert members == sorted(members)                      # ascending index inside
        # ordered ranges: every key of bucket b is below every key of bucket b+1
        if b + 1 < p and bo[b + 1] > bo[b] and bo[b + 2] > bo[b + 1]:
            hi = max(members, key=lambda i: (ka[i] / kb[i], i))
            nxt = order[bo[b + 1]:bo[b + 2]].tolist()
            for j in nxt:
                assert key_less(ka, kb, hi, j)
    # bucket = number of pivots strictly below the key
    piv = pt["pivot_idx"].tolist()
    for b in range(p):
        for i in order[bo[b]:bo[b + 1]]:
            assert sum(key_less(ka, kb, s, i) for s in piv if s >= 0) == b


@pytest.mark.parametrize("n,p", [(64, 4), (2000, 16), (1000, 7), (5, 8), (0, 3), (1, 1), (300, 1),
                                 (17, 17)])
def test_partition_properties(orc, n, p):
    rng = np.random.default_rng(n * 31 + p)
    kb = rng.integers(1, 500, size=n).astype(np.int32)
    ka = (rng.random(n) * (kb + 1)).astype(np.int32).clip(0, kb)
    pt = orc.partition(ka, kb, p)
    check_partition(ka, kb, p, pt)
    if n >= p * p and p > 1:
        # the regular-sampling bound of Section 3: no bucket holds 2N/p or more
        # (checked with slack for ragged blocks)
        w = -(-n // p)
        assert np.diff(pt["bucket_offsets"]).max() <= 2 * w + p


def test_partition_literal_pivot_positions(orc):
    # N >= p: every block is non-empty and the pivots sit at 1-based
    # (m-1)p + floor(p/2) in the sorted sample set Y
    rng = np.random.default_rng(9)
    for p in (2, 3, 4, 5, 8, 16):
        n = 40 * p + 3
        kb = np.full(n, 1000, np.int32)
        ka = rng.permutation(n).astype(np.int32) % 1000
        ys = []
        for b in range(p):
            blk = sorted(range(b * n // p, (b + 1) * n // p), key=lambda i: (ka[i], i))
            w = len(blk)
            ys += [blk[(j * w) // p] for j in range(1, p)]
        ys.sort(key=lambda i: (ka[i], i))
        want = [ys[(m - 1) * p + p // 2 - 1] for m in range(1, p)]
        assert orc.partition(ka, kb, p)["pivot_idx"].tolist() == want


def test_kmer_rows_agree_with_full_rank(orc):
    # the row routine used for sampled checks at full size matches the full stage
    w = synth.workload(4, n_override=400)
    full = orc.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, class_map=w.class_map,
                         kmer_alphabet=w.kmer_alphabet)
    rows = [0, 7, 199, 399, int(full["ga"])]
    part = orc.kmer_rows(w.residues, w.offsets, w.alphabet, w.k, w.p, rows, class_map=w.class_map,
                         kmer_alphabet=w.kmer_alphabet)
    np.testing.assert_array_equal(part["A_rows"], full["A"][rows])
    np.testing.assert_array_equal(part["dloc"], full["dloc"][rows])
    np.testing.assert_array_equal(part["dcen"], full["dcen"][rows])


def test_globalized_rank_with_every_sequence_sampled_is_centralized(orc):
    # s = block size: the strata positions floor((2j+1) w / 2w) = j take every
    # member once, so the sample set is the whole set and G = D-cen exactly
    w = synth.workload(1, seed=31)
    n, p = w.n, w.p
    r = orc.kmer_rank(w.residues, w.offsets, 20, w.k, p)
    assert n % p == 0
    G, smp = orc.global_rank(w.residues, w.offsets, w.k, p, n // p, r["dloc"])
    assert sorted(smp.tolist()) == list(range(n))
    np.testing.assert_array_equal(G, r["dcen"])


def test_globalized_rank_hand_example(orc):
    # the second golden case (class map, k=1): blocks {0,1} and {2,3,4};
    # local D: (1.5, 1.5 | 8/3, 2, 5/3) x 2^32. One sample per block:
    # position floor(w/2): block0 sorted (0,1) -> x1; block1 sorted by dloc (4,3,2) -> x3.
    # G_i = T(i, x1) + T(i, x3) with F column x1 = (1/2, 1, 1, 1, 0), x3 = (1, 1, 1, 1, 0).
    import json
    case = json.load(open(os.path.join(GOLD, "kmer_rank_tiny.json")))["cases"][1]
    res, offs = synth.pack(case["seqs"])
    G, smp = orc.global_rank(res, offs, 1, 2, 1, np.array(case["dloc"], np.uint64),
                             class_map=case["class_map"], kmer_alphabet=2)
    assert smp.tolist() == [1, 3]
    two32 = 1 << 32
    assert G.tolist() == [two32 // 2 + two32, 2 * two32, 2 * two32, 2 * two32, 0]


def test_partition_keys64_matches_rational_partition(orc):
    # 64-bit keys K = floor(a 2^32 / b) order the rational keys exactly for b <= 2^16
    rng = np.random.default_rng(12)
    kb = rng.integers(1, 300, 700).astype(np.int32)
    ka = (rng.random(700) * (kb + 1)).astype(np.int32).clip(0, kb)
    keys = (ka.astype(np.uint64) << np.uint64(32)) // kb.astype(np.uint64)
    for p in (1, 2, 7, 16):
        a = orc.partition(ka, kb, p)
        b = orc.partition_keys64(keys, p)
        for f in ("bucket_offsets", "order", "pivot_idx"):
            np.testing.assert_array_equal(a[f], b[f])
