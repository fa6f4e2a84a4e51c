"""GPU path (through the C ABI) against the CPU oracle, element by element.

Every output is an integer, so the bar is bit-exact: similarity numerators,
fixed-point D sums, ancestors, rank keys, pivots, the bucket layout and every
alignment score. Inputs are the seeded synthetic families (tree-evolved
protein-like sequences) plus adversarial cases.
"""
import numpy as np
import pytest

import oracle
from paper_0901_2742_gb300 import synth

pytestmark = pytest.mark.gpu

_cache = {}


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


def oracle_all(w, key=None):
    if key is None or key not in _cache:
        r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, class_map=w.class_map,
                             kmer_alphabet=w.kmer_alphabet, want_A=w.n <= 2000)
        pt = oracle.partition(r["key_a"], r["key_b"], w.p)
        so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"],
                                           w.subst, w.gap_open, w.gap_extend)
        if key is None:
            return (r, pt, so, sc)
        _cache[key] = (r, pt, so, sc)
    return _cache[key]


def to_np(x):
    if hasattr(x, "cpu"):
        return x.cpu().numpy()
    return np.asarray(x)


def assert_rank_equal(got, want, check_A=True):
    for f in ("dloc", "dcen", "la", "key_a", "key_b"):
        np.testing.assert_array_equal(to_np(got[f]), want[f], err_msg=f)
    assert int(np.asarray(to_np(got["ga"])).reshape(-1)[0]) == want["ga"]
    if check_A and got.get("A") is not None and want["A"] is not None:
        np.testing.assert_array_equal(to_np(got["A"]), want["A"])


def run_gpu(sad, w, mode, device=False):
    res, offs = w.residues, w.offsets
    if device:
        import torch
        res = torch.from_numpy(res).cuda()
        offs = torch.from_numpy(offs).cuda()
    r = sad.kmer_rank(res, offs, w.alphabet, w.k, w.p, cap=w.cap, kmer_alphabet=w.kmer_alphabet,
                      class_map=w.class_map, want_A=w.n <= 2000)
    pt = sad.partition(r["key_a"], r["key_b"], w.p)
    so, sc = sad.bucket_pair_scores(res, offs, w.alphabet, pt["bucket_offsets"], pt["order"], w.subst,
                                    w.gap_open, w.gap_extend, mode=mode)
    if device:
        import torch
        torch.cuda.synchronize()
    return r, pt, so, sc


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["per_bucket", "persistent", "persistent_32"])
def test_small_family_full_parity(sad, device, mode):
    w = synth.workload(1)
    want = oracle_all(w, "cfg1")
    r, pt, so, sc = run_gpu(sad, w, mode, device)
    assert_rank_equal(r, want[0])
    np.testing.assert_array_equal(to_np(pt["bucket_offsets"]), want[1]["bucket_offsets"])
    np.testing.assert_array_equal(to_np(pt["order"]), want[1]["order"])
    np.testing.assert_array_equal(to_np(pt["pivot_idx"]), want[1]["pivot_idx"])
    np.testing.assert_array_equal(to_np(so), want[2])
    np.testing.assert_array_equal(to_np(sc), want[3])


@pytest.mark.parametrize("seed", range(1, 9))
def test_small_family_seed_sweep(sad, seed):
    w = synth.workload(1, seed=seed)
    want = oracle_all(w, f"cfg1s{seed}")
    r, pt, so, sc = run_gpu(sad, w, 1)
    assert_rank_equal(r, want[0])
    np.testing.assert_array_equal(pt["order"], want[1]["order"])
    np.testing.assert_array_equal(sc, want[3])


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["per_bucket", "persistent", "persistent_32"])
def test_paper_scale_plain_full_parity(sad, mode):
    """N = 2000, L ~ N(316, 60), k = 3, p = 16: every output of every stage."""
    w = synth.workload(2)
    want = oracle_all(w, "cfg2")
    r, pt, so, sc = run_gpu(sad, w, mode)
    assert_rank_equal(r, want[0])
    np.testing.assert_array_equal(pt["bucket_offsets"], want[1]["bucket_offsets"])
    np.testing.assert_array_equal(pt["order"], want[1]["order"])
    np.testing.assert_array_equal(so, want[2])
    np.testing.assert_array_equal(sc, want[3])


def test_pipeline_matches_oracle(sad):
    w = synth.workload(2)
    want = oracle_all(w, "cfg2")
    for mem in ("host", "device"):
        res, offs = w.residues, w.offsets
        if mem == "device":
            import torch
            res, offs = torch.from_numpy(res).cuda(), torch.from_numpy(offs).cuda()
        o = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend,
                         cap=w.cap, mode=1)
        total = int(want[2][-1])
        np.testing.assert_array_equal(to_np(o["bucket_offsets"]), want[1]["bucket_offsets"])
        np.testing.assert_array_equal(to_np(o["order"]), want[1]["order"])
        np.testing.assert_array_equal(to_np(o["score_offsets"]), want[2])
        np.testing.assert_array_equal(to_np(o["scores"])[:total], want[3])
        # every rank output (with device arrays the stages write them in place)
        for f in ("dloc", "dcen", "la", "key_a", "key_b"):
            np.testing.assert_array_equal(to_np(o[f]), want[0][f], err_msg=f"{mem} {f}")
        assert int(to_np(o["ga"]).reshape(-1)[0]) == want[0]["ga"]


def make_workload(seqs, p, k=3, alphabet=20, subst=None, go=-11, ge=-1, class_map=None, ka=None):
    res, offs = synth.pack(seqs)
    S = synth.subst_matrix(99, alphabet) if subst is None else subst
    return synth.Workload("adhoc", res, offs, alphabet, S, go, ge, k, p, 0, ka or alphabet, class_map)


def compare_all(sad, w, modes=(0, 1)):
    want = oracle_all(w)
    for mode in modes:
        r, pt, so, sc = run_gpu(sad, w, mode)
        assert_rank_equal(r, want[0])
        np.testing.assert_array_equal(pt["order"], want[1]["order"])
        np.testing.assert_array_equal(pt["bucket_offsets"], want[1]["bucket_offsets"])
        np.testing.assert_array_equal(sc, want[3])


def test_edge_short_and_empty_sequences(sad):
    rng = np.random.default_rng(1)
    seqs = [[], [3], [1, 2], [1, 2, 3], list(rng.integers(0, 20, 40)), [], list(rng.integers(0, 20, 5)),
            [7, 7, 7]]
    compare_all(sad, make_workload(seqs, p=3))


def test_edge_fewer_sequences_than_buckets(sad):
    rng = np.random.default_rng(2)
    for n in (1, 2, 5):
        seqs = [list(rng.integers(0, 20, rng.integers(10, 60))) for _ in range(n)]
        compare_all(sad, make_workload(seqs, p=8))


def test_edge_identical_sequences(sad):
    seqs = [list(synth.uniform_residues(5, 90))] * 37
    compare_all(sad, make_workload(seqs, p=5))


def test_edge_counts_above_255_use_the_residual(sad):
    # homopolymers and short-period repeats: k-mer counts far above 255
    rng = np.random.default_rng(3)
    seqs = [[4] * 700, [4] * 300 + [5] * 300, [4, 5] * 350, [4] * 260, list(rng.integers(0, 20, 300)),
            [4] * 1000 + list(rng.integers(0, 20, 50)), [5] * 600]
    compare_all(sad, make_workload(seqs, p=2))


def test_edge_long_sequences_strip_mining(sad):
    # queries longer than one strip of the widest kernel variant
    rng = np.random.default_rng(4)
    seqs = [list(rng.integers(0, 20, L)) for L in (1100, 1500, 2000, 2000, 1700, 900, 50, 1)]
    compare_all(sad, make_workload(seqs, p=1))


def test_edge_odd_p_and_p_one(sad):
    w = synth.workload(1, seed=77)
    for p in (1, 3, 7):
        w.p = p
        compare_all(sad, w)


def test_compressed_alphabet_k4(sad):
    """Six-letter compressed alphabet, k = 4 (the large-batch k-mer setting) on a small set."""
    w = synth.workload(4, n_override=300)
    w.cap = 0
    compare_all(sad, w, modes=(1,))


@pytest.mark.parametrize("params", [(-11, -1), (0, -1), (-3, 0), (0, 0), (-40, -7)])
def test_gotoh_random_buckets_and_gap_costs(sad, params):
    go, ge = params
    rng = np.random.default_rng(abs(go) * 10 + abs(ge))
    lens = list(rng.integers(0, 6, 10)) + list(rng.integers(1, 400, 40)) + [777, 1025, 1300]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    res, offs = synth.pack(seqs)
    n = len(seqs)
    order = rng.permutation(n).astype(np.int32)
    bo = np.array([0, 1, 1, 12, 30, n], np.int32)   # includes an empty and a singleton bucket
    S = synth.subst_matrix(5)
    want_so, want_sc = oracle.bucket_pair_scores(res, offs, bo, order, S, go, ge)
    for mode in (0, 1, 2):
        so, sc = sad.bucket_pair_scores(res, offs, 20, bo, order, S, go, ge, mode=mode)
        np.testing.assert_array_equal(so, want_so)
        np.testing.assert_array_equal(sc, want_sc)


def test_partition_random_keys_with_ties(sad):
    rng = np.random.default_rng(8)
    for n, p in ((500, 7), (64, 4), (3, 5), (2000, 16), (1000, 1), (4096, 64)):
        kb = rng.integers(1, 40, n).astype(np.int32)
        ka = (rng.random(n) * (kb + 1)).astype(np.int32).clip(0, kb)
        want = oracle.partition(ka, kb, p)
        got = sad.partition(ka, kb, p)
        np.testing.assert_array_equal(got["bucket_offsets"], want["bucket_offsets"])
        np.testing.assert_array_equal(got["order"], want["order"])
        np.testing.assert_array_equal(got["pivot_idx"], want["pivot_idx"])


def test_bad_residue_is_reported(sad):
    res = np.array([1, 2, 30, 4], np.uint8)
    offs = np.array([0, 4], np.int64)
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank(res, offs, 20, 2, 1)
    assert e.value.code == sad.SAD_EINVAL


def test_scores_capacity_too_small(sad):
    w = synth.workload(1)
    want = oracle_all(w, "cfg1")
    bo, order = want[1]["bucket_offsets"], want[1]["order"]
    with pytest.raises(sad.SadError) as e:
        sad.bucket_pair_scores(w.residues, w.offsets, 20, bo, order, w.subst, -11, -1, capacity=10)
    assert e.value.code == sad.SAD_ERANGE


# ---- threshold planes on the tensor cores (cap > 0) ---------------------------

def run_rank_only(sad, w, cap):
    return sad.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, cap=cap,
                         kmer_alphabet=w.kmer_alphabet, class_map=w.class_map, want_A=True)


def test_planes_single_tile(sad):
    """One 128 x 128 tile (N = 64): every numerator from the tcgen05 GEMM."""
    w = synth.workload(1)
    want = oracle_all(w, "cfg1")
    assert_rank_equal(run_rank_only(sad, w, 4), want[0])


@pytest.mark.parametrize("cap", [1, 2, 3, 4, 8])
def test_planes_caps_and_residuals(sad, cap):
    # caps below typical counts force the residual path for many pairs
    rng = np.random.default_rng(cap)
    seqs = [list(rng.integers(0, 4, L)) for L in rng.integers(3, 300, 150)]
    seqs += [[4] * 400, [4, 5] * 200, [1] * 3, []]
    w = make_workload(seqs, p=5, k=2)
    want = oracle_all(w)
    assert_rank_equal(run_rank_only(sad, w, cap), want[0])


def test_planes_paper_scale(sad):
    """N = 2000, cap 4, K = 4 x 8000: ragged last tile row, 136 tiles. Most
    k-blocks of the count >= 3 and >= 4 planes are zero in a panel and are
    skipped; the result is the oracle's all the same."""
    w = synth.workload(3)
    want = oracle_all(w, "cfg2")
    r, pt, so, sc = run_gpu(sad, w, 1)
    assert_rank_equal(r, want[0])
    np.testing.assert_array_equal(pt["order"], want[1]["order"])
    np.testing.assert_array_equal(sc, want[3])
    mma, dense = sad.kmer_gemm_work()
    assert dense == 136 * 250 * 2 * 128 * 128 * 128
    assert 0 < mma < dense


def test_planes_skip_only_zero_kblocks(sad):
    """Counts up to 6 in a few rows of different panels, 1 elsewhere: the
    k-blocks of the high planes are nonzero in some panels only, so some tiles
    run them and some skip them; every D sum and key stays the oracle's."""
    rng = np.random.default_rng(77)
    seqs = []
    for i in range(300):
        L = int(rng.integers(40, 200))
        s = list(rng.integers(0, 20, L))
        if i % 97 == 5:  # a repeat: one 3-mer many times
            s[:18] = [3, 7, 11] * 6
        seqs.append(s)
    res, offs = synth.pack(seqs)
    want = oracle.kmer_rank(res, offs, 20, 3, 4, want_A=True)
    got = sad.kmer_rank(res, offs, 20, 3, 4, cap=4, want_A=True)
    assert_rank_equal(got, want)
    mma, dense = sad.kmer_gemm_work()
    assert 0 < mma < dense


def test_planes_long_sequences_large_plane_sums(sad):
    """Plane sums far above 2^14 in the fp32 tensor-memory accumulator: random
    sequences of 40k-65k residues hold nearly every 3-mer of 20 letters 4 or
    more times, so sum_tau min(c_i, c_j, 4) approaches 4 x 8000 = 32000 (the
    accumulator stays exact below 2^24); short-period repeats and a homopolymer
    tail add counts above the cap and above 255 (the residual and the excess
    lists), and one short sequence gives small ratios beside them. k-mer stage
    only (the rank outputs and every numerator), against the oracle."""
    rng = np.random.default_rng(99)
    seqs = [list(rng.integers(0, 20, L)) for L in (65537, 60000, 52000, 45000, 40000)]
    seqs.append(list(np.tile(rng.integers(0, 20, 7), 8000)[:56000]))         # period 7: 7 k-mers, ~8000 each
    seqs.append(list(rng.integers(0, 20, 30000)) + [0] * 20000)              # homopolymer tail
    seqs.append(list(rng.integers(0, 20, 300)))
    res, offs = synth.pack(seqs)
    want = oracle.kmer_rank(res, offs, 20, 3, 3, want_A=True)
    assert int(np.max(want["A"])) > 2 ** 14
    got = sad.kmer_rank(res, offs, 20, 3, 3, cap=4, want_A=True)
    assert_rank_equal(got, want)


def test_planes_compressed_alphabet(sad):
    """Six-letter alphabet, k = 4, cap 4 (K = 4 x 1344, a partial last k-block)."""
    w = synth.workload(4, n_override=700)
    want = oracle_all(w)
    assert_rank_equal(run_rank_only(sad, w, 4), want[0])


@pytest.mark.parametrize("R", [8, 12, 16, 20, 24, 32])
@pytest.mark.parametrize("G", [8, 16, 32])
def test_every_packed_variant_exact(sad, R, G):
    """Force one packed-kernel variant for every query pair: scores stay exact,
    including queries that need several strips of G x R rows."""
    rng = np.random.default_rng(R * 100 + G)
    lens = list(rng.integers(1, 300, 30)) + [G * R - 1, G * R, G * R + 1, 3 * G * R + 5, 0]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    res, offs = synth.pack(seqs)
    n = len(seqs)
    order = rng.permutation(n).astype(np.int32)
    bo = np.array([0, 9, 20, n], np.int32)
    S = synth.subst_matrix(6)
    want_so, want_sc = oracle.bucket_pair_scores(res, offs, bo, order, S, -11, -1)
    sad.set_score_variants([(2 ** 31 - 1, R, G)])
    try:
        so, sc = sad.bucket_pair_scores(res, offs, 20, bo, order, S, -11, -1, mode=1)
    finally:
        sad.set_score_variants([])
    np.testing.assert_array_equal(so, want_so)
    np.testing.assert_array_equal(sc, want_sc)


@pytest.mark.parametrize("R", [8, 12, 16, 20, 24, 32])
@pytest.mark.parametrize("G", [8, 16, 32])
@pytest.mark.parametrize("gaps", [(-11, -1), (0, 0)])
def test_every_packed_variant_streaming_exact(sad, R, G, gaps):
    """One packed variant forced for query pairs that all fit one strip of
    G x R rows, so the launch streams every group's subjects through one
    wavefront: subjects of odd and even length (1, 2 and 3 residues among them)
    follow each other, each odd one entered through its virtual column 0."""
    go, ge = gaps
    rng = np.random.default_rng(R * 1000 + G * 10 + abs(go))
    lens = list(rng.integers(1, G * R + 1, 40)) + [1, 2, 3, 4, 5, G * R, G * R - 1, 0]
    seqs = [list(rng.integers(0, 20, L)) for L in lens]
    res, offs = synth.pack(seqs)
    n = len(seqs)
    order = rng.permutation(n).astype(np.int32)
    bo = np.array([0, 3, 17, n], np.int32)
    S = synth.subst_matrix(7)
    want_so, want_sc = oracle.bucket_pair_scores(res, offs, bo, order, S, go, ge)
    sad.set_score_variants([(2 ** 31 - 1, R, G)])
    try:
        so, sc = sad.bucket_pair_scores(res, offs, 20, bo, order, S, go, ge, mode=1)
    finally:
        sad.set_score_variants([])
    np.testing.assert_array_equal(so, want_so)
    np.testing.assert_array_equal(sc, want_sc)


def test_autotuned_variants_stay_exact(sad):
    """The autotuner only picks speeds: after tuning on the paper-scale layout
    the scores are still those of the oracle."""
    w = synth.workload(2)
    want = oracle_all(w, "cfg2")
    bo, od = want[1]["bucket_offsets"], want[1]["order"]
    table = sad.autotune_scores(w.residues, w.offsets, w.alphabet, bo, od, w.subst, w.gap_open, w.gap_extend,
                                reps=1)
    try:
        assert len(table) >= 1
        for upper, R, G in table:
            assert R in (8, 12, 16, 20, 24, 32) and G in (8, 16, 32)
        so, sc = sad.bucket_pair_scores(w.residues, w.offsets, w.alphabet, bo, od, w.subst, w.gap_open,
                                        w.gap_extend, mode=1)
        np.testing.assert_array_equal(sc, want[3])
    finally:
        sad.set_score_variants([])


def test_large_uneven_batch_sampled_parity(sad):
    """N = 20000 (400 Zipf families, lognormal lengths to 2000, 6-letter k = 4,
    cap 4, p = 64) through sad_pipeline as the benchmark runs it. The oracle
    recomputes sampled outputs one by one: whole k-mer rows and their D sums
    (including every local ancestor's row), the global ancestor's choice among
    them, the rank keys of sampled sequences, the complete partition of the
    GPU's keys, and sampled alignment scores of every bucket."""
    import torch
    w = synth.workload(4)
    n, p = w.n, w.p
    res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
    o = sad.pipeline(res, offs, w.alphabet, w.k, p, w.subst, w.gap_open, w.gap_extend, cap=w.cap,
                     kmer_alphabet=w.kmer_alphabet, class_map=w.class_map, mode=1)
    torch.cuda.synchronize()
    g = {k: to_np(v) for k, v in o.items()}
    la, ga = g["la"], int(g["ga"][0])
    rng = np.random.default_rng(20000)
    rows = sorted(set(rng.choice(n, 24, replace=False).tolist()) | set(la.tolist()))
    part = oracle.kmer_rows(w.residues, w.offsets, w.alphabet, w.k, p, rows, class_map=w.class_map,
                            kmer_alphabet=w.kmer_alphabet)
    np.testing.assert_array_equal(g["dloc"][rows], part["dloc"])
    np.testing.assert_array_equal(g["dcen"][rows], part["dcen"])
    # local ancestors: argmax of D-loc inside each block (lowest index on ties)
    for b in range(p):
        lo, hi = b * n // p, (b + 1) * n // p
        assert la[b] == lo + int(np.argmax(g["dloc"][lo:hi]))
    # global ancestor: the local ancestor with the largest fixed-point sum to all local ancestors
    L = w.lengths().astype(np.int64)
    ridx = {r: t for t, r in enumerate(rows)}
    scores = []
    for x in la:
        s = 0
        for y in la:
            a = int(part["A_rows"][ridx[int(x)], int(y)])
            b_ = min(L[x], L[y]) - w.k + 1
            s += (a << 32) // b_ if b_ > 0 else 0
        scores.append(s)
    assert ga == int(la[int(np.argmax(scores))])
    # keys of sampled sequences against GA
    gr = oracle.kmer_rows(w.residues, w.offsets, w.alphabet, w.k, p, [ga], class_map=w.class_map,
                          kmer_alphabet=w.kmer_alphabet)["A_rows"][0]
    for i in rows:
        b_ = min(L[i], L[ga]) - w.k + 1
        want = (int(gr[i]), int(b_)) if b_ > 0 else (0, 1)
        assert (int(g["key_a"][i]), int(g["key_b"][i])) == want
    # the whole partition of the GPU keys
    pt = oracle.partition(g["key_a"], g["key_b"], p)
    np.testing.assert_array_equal(g["bucket_offsets"], pt["bucket_offsets"])
    np.testing.assert_array_equal(g["order"][:n], pt["order"])
    # sampled alignment scores: a few pairs of every bucket
    bo, od, so, sc = g["bucket_offsets"], g["order"], g["score_offsets"], g["scores"]
    checked = 0
    for b in range(p):
        nb = int(bo[b + 1] - bo[b])
        if nb == 0:
            continue
        for _ in range(4):
            u, v = sorted(rng.integers(0, nb, 2).tolist())
            xi, yi = int(od[bo[b] + u]), int(od[bo[b] + v])
            x = w.residues[w.offsets[xi]:w.offsets[xi + 1]]
            y = w.residues[w.offsets[yi]:w.offsets[yi + 1]]
            want = oracle.gotoh(x, y, w.subst, w.gap_open, w.gap_extend)
            assert sc[so[b] + oracle.tri_index(u, v, nb)] == want
            checked += 1
    assert checked >= 4 * 60


def test_batched_scores_graph_capture_and_replay(sad):
    """On a created stream the batched score launches are captured into a CUDA
    graph once and replayed while the launch set is unchanged; a different
    layout recaptures. Every run is exact."""
    import torch
    w = synth.workload(2)
    want = oracle_all(w, "cfg2")
    bo, od = want[1]["bucket_offsets"], want[1]["order"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        res, offs = torch.from_numpy(w.residues).cuda(), torch.from_numpy(w.offsets).cuda()
        dbo, dod = torch.from_numpy(bo).cuda(), torch.from_numpy(od).cuda()
        l0 = sad.launch_count()
        for _ in range(3):
            so, sc = sad.bucket_pair_scores(res, offs, w.alphabet, dbo, dod, w.subst, w.gap_open, w.gap_extend,
                                            mode=1)
            s.synchronize()
            np.testing.assert_array_equal(sc.cpu().numpy(), want[3])
        assert sad.launch_count() > l0
        # a different layout (one bucket fewer) must not replay the old graph
        bo2 = np.array([0, bo[2]] + list(bo[3:]), np.int32)
        want2 = oracle.bucket_pair_scores(w.residues, w.offsets, bo2, od, w.subst, w.gap_open, w.gap_extend)
        so2, sc2 = sad.bucket_pair_scores(res, offs, w.alphabet, torch.from_numpy(bo2).cuda(), dod, w.subst,
                                          w.gap_open, w.gap_extend, mode=1)
        s.synchronize()
        np.testing.assert_array_equal(sc2.cpu().numpy(), want2[1])


def test_planes_wide_tiles_full_matrix(sad):
    """N = 5000 (enough 128 x 256 tiles to fill the GPU): the persistent wide-tile
    GEMM with double-buffered accumulators, every numerator of the full matrix,
    every D sum and key, with heavy excess residuals (6-letter alphabet, k = 4)."""
    w = synth.workload(4, n_override=5000)
    want = oracle_all(w)
    got = run_rank_only(sad, w, 4)
    assert_rank_equal(got, want[0])
