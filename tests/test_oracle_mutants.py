"""Planted mistakes: each mutant copy of the oracle must fail at least one pin.

A plausible slip anywhere in the oracle (a dropped term, an off-by-one, a
wrong state, a flipped comparison) is written into a copy of oracle.cpp,
compiled on the CPU, and run through a compact battery of the same kinds of
pins the other oracle tests use (brute-force alignments, brute-force k-mer
intersections, hand-worked golden examples, literal pivot positions). The
real oracle passes the battery; every mutant must fail it.
"""
import json
import os
import random
import tempfile

import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth
from test_oracle_gotoh import brute_force, random_symmetric
from test_oracle_kmer_partition import kmer_tuples, multiset_intersection_size, check_partition

GOLD = os.path.join(os.path.dirname(__file__), "golden")

MUTANTS = {
    "gap open dropped in X": ("if (open > NEG_INF) v = open + go + ge;\n                if (X[", "if (open > NEG_INF) v = open + ge;\n                if (X["),
    "gap open dropped in Y": ("if (open > NEG_INF) v = open + go + ge;\n                if (Y[", "if (open > NEG_INF) v = open + ge;\n                if (Y["),
    "match uses wrong residue": ("S[x[i - 1] * alphabet + y[j - 1]]", "S[y[j - 1] * alphabet + y[j - 1]]"),
    "extend from match state": ("X[at(i - 1, j)] + ge)", "M[at(i - 1, j)] + ge)"),
    "max instead of min count": ("a += std::min(kv.second, it->second)", "a += std::max(kv.second, it->second)"),
    "denominator off by one": ("return std::min(li, lj) - k + 1;", "return std::min(li, lj) - k;"),
    "fixed point 2^31": ("return ((uint64_t)a << 32) / (uint64_t)b;", "return ((uint64_t)a << 31) / (uint64_t)b;"),
    "local ancestor tie to last": ("dloc[i] > dloc[best]", "dloc[i] >= dloc[best]"),
    "sample position shifted": ("samples.push_back(blk[(j * w) / p]);", "samples.push_back(blk[((j - 1) * w) / p]);"),
    "pivot rounding up": ("std::max(1, q / 2)", "std::max(1, (q + 1) / 2)"),
    "bucket by pivots <= key": ("if (less(s, i)) c++;", "if (!less(i, s)) c++;"),
    "key denominator ignores GA": ("int64_t b = denom(len[i], len[g], k);", "int64_t b = denom(len[i], len[i], k);"),
    "self term dropped": ("for (int32_t j = 0; j < n; j++) {\n            int64_t a", "for (int32_t j = 0; j < n; j++) {\n            if (j == i) continue;\n            int64_t a"),
    "tree distance with one self score": ("W[u][v] = S(u, u) + S(v, v) - 2 * S(", "W[u][v] = 2 * S(u, u) - 2 * S("),
    "tree comparison without sizes": ("const __int128 lhs = (__int128)W[i][j] * (size[bi] * size[bj]);", "const __int128 lhs = (__int128)W[i][j];"),
    "tree tie to the last pair": ("if (lhs < rhs) {  // on equality", "if (lhs <= rhs) {  // on equality"),
    "tree merge sums one child": ("W[c][x] = W[x][c] = W[bi][x] + W[bj][x];", "W[c][x] = W[x][c] = 2 * W[bi][x];"),
    "profile gaps not scaled by the member counts": ("const int64_t gop = (int64_t)go * np * nq, gex = (int64_t)ge * np * nq;",
                                                     "const int64_t gop = go, gex = ge;"),
    "profile column counts the wrong letter": ("S[a * alphabet + c] * cq[j * alphabet + c];",
                                               "S[a * alphabet + c] * cq[j * alphabet + a];"),
    "profile end tie prefers a gap": ("char state = best_of(m, w, true, true, true, score, 0);",
                                      "char state = best_of(m, w, false, true, true, score, 0);\n"
                                      "            if (state == '?') state = 'M';"),
    "glue anchor before the slot's insertions": (
        "        for (int32_t b = 0; b < p; b++) {\n            start[sl * p + b] = col;\n            col += ins[sl * p + b];\n"
        "        }\n        if (sl < lg) anchor_col[sl] = col++;",
        "        if (sl < lg) anchor_col[sl] = col++;\n        for (int32_t b = 0; b < p; b++) {\n"
        "            start[sl * p + b] = col;\n            col += ins[sl * p + b];\n        }"),
    "glue keeps empty columns": ("        kept += used[x];", "        kept += 1;"),
    "glue profile of the first member only": (
        "for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b + 1]; q++) {\n            const uint8_t* x = res + offs[order[q]];",
        "for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b] + 1; q++) {\n            const uint8_t* x = res + offs[order[q]];"),
    "glue insertion slot one late": ("anchors[col_off[b] + c++] = -(int32_t)(g + 1);", "anchors[col_off[b] + c++] = -(int32_t)g;"),
    "profile of the first member only": ("for (size_t t = 0; t < c.members.size(); t++) {\n                const uint8_t* x",
                                         "for (size_t t = 0; t < 1; t++) {\n                const uint8_t* x"),
}


def battery(lib):
    """Return the list of pin names that fail for this oracle build."""
    failed = []
    # 1. Gotoh vs brute force, including an odd alphabet and both gap regimes
    rng = random.Random(1)
    for _ in range(40):
        A = rng.choice([2, 3, 20])
        S = random_symmetric(rng, A, -6, 9)
        go, ge = rng.choice([0, -3, -11]), rng.choice([-1, -2])
        x = [rng.randrange(A) for _ in range(rng.randint(0, 5))]
        y = [rng.randrange(A) for _ in range(rng.randint(0, 5))]
        if oracle.gotoh(x, y, S, go, ge, lib=lib) != brute_force(x, y, S, go, ge):
            failed.append("gotoh brute force")
            break
    # 2. k-mer matrix vs sorted-tuple intersection
    seqs = [list(synth.uniform_residues(50 + t, rng.randint(2, 40), 3)) for t in range(8)]
    res, offs = synth.pack(seqs)
    r = oracle.kmer_rank(res, offs, 20, 2, 2, lib=lib)
    tup = [kmer_tuples(s, 2) for s in seqs]
    if any(r["A"][i, j] != multiset_intersection_size(tup[i], tup[j])
           for i in range(8) for j in range(8)):
        failed.append("kmer brute force")
    # 3. golden examples (rank, partition, scores)
    with open(os.path.join(GOLD, "kmer_rank_tiny.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        res, offs = synth.pack(c["seqs"])
        r = oracle.kmer_rank(res, offs, c["alphabet"], c["k"], c["p"], class_map=c["class_map"],
                             kmer_alphabet=c["kmer_alphabet"], lib=lib)
        pt = oracle.partition(r["key_a"], r["key_b"], c["p"], lib=lib)
        got = [r["dcen"].tolist(), r["dloc"].tolist(), r["la"].tolist(), r["ga"],
               r["key_a"].tolist(), r["key_b"].tolist(), pt["order"].tolist(),
               pt["pivot_idx"].tolist()]
        want = [c["dcen"], c["dloc"], c["la"], c["ga"], c["key_a"], c["key_b"], c["order"],
                c["pivot_idx"]]
        if got != want:
            failed.append("golden " + c["name"])
    with open(os.path.join(GOLD, "psrs_tiny.json")) as f:
        for c in json.load(f)["cases"]:
            pt = oracle.partition(c["key_a"], c["key_b"], c["p"], lib=lib)
            if pt["order"].tolist() != c["order"] or pt["pivot_idx"].tolist() != c["pivot_idx"]:
                failed.append("golden psrs")
    # 4. partition properties on random keys
    g = np.random.default_rng(3)
    kb = g.integers(1, 300, size=500).astype(np.int32)
    ka = (g.random(500) * (kb + 1)).astype(np.int32).clip(0, kb)
    try:
        check_partition(ka, kb, 7, oracle.partition(ka, kb, 7, lib=lib))
    except AssertionError:
        failed.append("partition properties")
    # 5. guide trees: golden examples and the mean-over-member-pairs invariant
    with open(os.path.join(GOLD, "guide_tree_tiny.json")) as f:
        for c in json.load(f)["cases"][:2]:
            nb = int(round((np.sqrt(8 * len(c["scores"]) + 1) - 1) / 2))
            t = oracle.guide_trees(np.array([0, nb], np.int32), np.array([0, len(c["scores"])]),
                                   np.array(c["scores"], np.int32), lib=lib)
            if any(t[f].tolist() != c[f] for f in ("left", "right", "num", "den")):
                failed.append("golden guide tree " + c["name"])
    nb = 9
    rs = np.random.default_rng(5)
    sc = rs.integers(-30, 30, nb * (nb + 1) // 2).astype(np.int32)
    t = oracle.guide_trees(np.array([0, nb], np.int32), np.array([0, len(sc)]), sc, lib=lib)
    S = {}
    for (u, v), x in zip([(u, v) for u in range(nb) for v in range(u, nb)], sc):
        S[u, v] = S[v, u] = int(x)
    members = {i: [i] for i in range(nb)}
    for m in range(nb - 1):
        a, c = int(t["left"][m]), int(t["right"][m])
        if a not in members or c not in members:
            failed.append("guide tree structure")
            break
        pairs = [(u, v) for u in members[a] for v in members[c]]
        if t["num"][m] != sum(S[u, u] + S[v, v] - 2 * S[u, v] for u, v in pairs) or t["den"][m] != len(pairs):
            failed.append("guide tree member pairs")
            break
        members[nb + m] = members.pop(a) + members.pop(c)
    # 6. guide tree against scipy's average linkage (tie-free distances)
    try:
        from scipy.cluster.hierarchy import linkage
    except ImportError:
        linkage = None
    if linkage is not None:
        nb = 24
        vals = np.random.default_rng(11).choice(10 ** 6, size=nb * (nb - 1) // 2, replace=False) + 1
        sc, cond, k = [], [], 0
        for u in range(nb):
            for v in range(u, nb):
                if u == v:
                    sc.append(0)
                else:
                    sc.append(-int(vals[k]))
                    cond.append(2.0 * vals[k])
                    k += 1
        t = oracle.guide_trees(np.array([0, nb], np.int32), np.array([0, len(sc)]), np.array(sc, np.int32), lib=lib)
        Z = linkage(np.array(cond), method="average")
        if any(sorted((int(Z[m, 0]), int(Z[m, 1]))) != [t["left"][m], t["right"][m]] for m in range(nb - 1)):
            failed.append("guide tree vs scipy")
    # 7. progressive alignment: the golden example, and every merge of random tiny
    #    buckets against the best of all its alignments, enumerated
    import test_oracle_progressive as tp
    with open(os.path.join(GOLD, "progressive_tiny.json")) as f:
        c = json.load(f)
    res, offs = synth.pack(c["seqs"])
    r = oracle.progressive(res, offs, c["bucket_offsets"], c["order"], c["merge_offsets"], c["left"], c["right"],
                           np.array(c["subst"]).ravel(), c["gap_open"], c["gap_extend"], lib=lib)
    if any(r[f].tolist() != c[f] for f in ("widths", "merge_scores", "merge_widths", "colmap")):
        failed.append("golden progressive")
    rng = random.Random(7)
    for _ in range(6):
        A = rng.choice([2, 3])
        S = random_symmetric(rng, A, -4, 6).astype(np.int64).tolist()
        nb = rng.randint(2, 4)
        seqs = [[rng.randrange(A) for _ in range(rng.randint(0, 3))] for _ in range(nb)]
        left, right = tp.random_tree(rng, nb)
        res, offs = synth.pack(seqs)
        r = oracle.progressive(res, offs, [0, nb], list(range(nb)), [0, nb - 1], left, right,
                               np.array(S, np.int8).ravel(), -3, -1, lib=lib)
        rows = tp.rows_of(seqs, [0, nb], list(range(nb)), r["colmap"])[0]
        try:
            tp.check_rows(rows, int(r["widths"][0]))
            tp.check_merges({u: seqs[u] for u in range(nb)}, nb, left, right, r["merge_scores"].tolist(),
                            r["merge_widths"].tolist(), rows, S, -3, -1)
        except AssertionError:
            failed.append("progressive brute force")
            break
    # 8. realignment against the ancestor and the glue: golden examples, brute force
    import test_oracle_glue as tg
    with open(os.path.join(GOLD, "ancestor_glue_tiny.json")) as f:
        g = json.load(f)
    Sg = np.array(g["subst"], np.int8).ravel()
    for c in g["cases"]:
        res, offs = synth.pack(c["seqs"])
        r = oracle.ancestor_glue(res, offs, c["bucket_offsets"], c["order"], c["widths"], c["colmap"], c["ga"], Sg,
                                 g["gap_open"], g["gap_extend"], lib=lib)
        if (r["ga_scores"].tolist() != c["ga_scores"] or r["anchors"].tolist() != c["anchors"]
                or r["width"] != c["width"] or r["colmap"].tolist() != c["global_colmap"]):
            failed.append("golden glue " + c["name"])
    rng = random.Random(8)
    for _ in range(4):
        A = 2
        S = random_symmetric(rng, A, -4, 6).astype(np.int64).tolist()
        sizes = [rng.randint(1, 3) for _ in range(2)]
        seqs, bo, left, right, mo = [], [0], [], [], [0]
        for nb in sizes:
            seqs += [[rng.randrange(A) for _ in range(rng.randint(1, 3))] for _ in range(nb)]
            bo.append(bo[-1] + nb)
            lt, rt = tp.random_tree(rng, nb) if nb > 1 else ([], [])
            left += lt
            right += rt
            mo.append(mo[-1] + max(nb - 1, 0))
        order = list(range(len(seqs)))
        res, offs = synth.pack(seqs)
        flat = np.array(S, np.int8).ravel()
        pr = oracle.progressive(res, offs, bo, order, mo, left, right, flat, -3, -1, lib=lib)
        r = oracle.ancestor_glue(res, offs, bo, order, pr["widths"], pr["colmap"], 0, flat, -3, -1, lib=lib)
        try:
            tg.check_glue(seqs, bo, order, pr["widths"].tolist(), pr["colmap"], 0, S, -3, -1, r)
        except AssertionError:
            failed.append("glue brute force")
            break
    return failed


def test_real_oracle_passes_battery():
    assert battery(oracle._load()) == []


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not found exactly once: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mut.cpp")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(d, "libmut.so")
        os.system(f"g++ -O1 -std=c++17 -fPIC -shared -pthread -o {so} {path}")
        assert os.path.exists(so)
        lib = oracle.load_variant(so)
        try:
            caught = battery(lib)
        except (ValueError, AssertionError, IndexError) as e:   # a pin raised: caught
            caught = [f"raised {type(e).__name__}"]
        assert caught, f"mutant '{name}' passed every pin"
