"""Host-side helpers of bench.py (no GPU): the device-idle summary of the
tracer's timeline, and the rule that the recorded DRAM traffic of the score
kernels and of the plane GEMM is reported only for the source that was
profiled, the refinement's least-padding start and the sparse lookup count."""
import os

import bench


def test_device_gaps_per_step():
    spans = [("prepare", 0.0, 1.0), ("count", 1.5, 2.0), ("scores_packed", 3.0, 5.0),
             ("prepare", 10.0, 11.0), ("count", 11.1, 12.0), ("scores_packed", 12.5, 14.0)]
    g = bench.device_gaps(spans)
    assert g["traced_span_ms"] == 4.5          # (5 - 0 + 14 - 10) / 2
    assert abs(g["busy_ms"] - 3.45) < 1e-12    # (1 + 0.5 + 2 + 1 + 0.9 + 1.5) / 2
    assert abs(g["idle_ms"] - 1.05) < 1e-12
    assert abs(g["gap_after_ms"]["prepare"] - 0.3) < 1e-12
    assert abs(g["gap_after_ms"]["count"] - 0.75) < 1e-12
    assert "scores_packed" not in g["gap_after_ms"]  # last stage of each step
    assert bench.device_gaps([]) is None


def test_traffic_only_for_the_profiled_kernel(monkeypatch):
    import hashlib
    import os
    with open(os.path.join(bench.ROOT, "paper_0901_2742_gb300", "csrc", "gotoh.cu")) as f:
        src = f.read()
    h = hashlib.sha256(src[:src.index(bench.DEVICE_CODE_END)].encode()).hexdigest()
    want = bench.SCORE_TRAFFIC["bytes_per_step"] if h == bench.SCORE_TRAFFIC["gotoh_device_sha256"] else None
    assert bench.score_traffic() == want
    stale = dict(bench.SCORE_TRAFFIC, gotoh_device_sha256="0" * 64)
    monkeypatch.setattr(bench, "SCORE_TRAFFIC", stale)
    assert bench.score_traffic() is None


def test_sparse_lookup_count_brute_force():
    """The sorted-list path's lookup count: per row block of 8 rows, one lookup
    per k-mer entry of every column j >= the block's first row; distinct k-mers
    counted here with Python sets."""
    import numpy as np
    from paper_0901_2742_gb300 import synth
    w = synth.workload(1)
    w.k = 4
    L = np.diff(w.offsets)
    distinct = [len({tuple(w.residues[w.offsets[i] + t:w.offsets[i] + t + w.k]) for t in range(L[i] - w.k + 1)})
                for i in range(w.n)]
    assert list(bench._kmer_distinct_counts(w)) == distinct
    want = sum(distinct[j] for b0 in range(0, w.n, 8) for j in range(b0, w.n))
    r = bench.sparse_kmer_roofline(w, 1.0)
    assert r["lookups_per_launch"] == want
    assert r["kmer_space"] == w.kmer_alphabet ** 4
    assert abs(r["frac"] - want / 1e-3 / (bench.SMS * 32 * bench.SM_MAX_MHZ * 1e6)) < 1e-12


def test_least_padding_seed_table():
    """The refinement's second start: per bin the smallest strip G R that holds
    the bin's rows, then R <= 24, then G nearest 16; the open-ended bin keeps
    its variant."""
    t = bench.least_padding_table([(256, 32, 8), (320, 24, 16), (384, 24, 16), (512, 32, 16), (2 ** 31 - 1, 20, 32)])
    assert t == [(256, 16, 16), (320, 20, 16), (384, 24, 16), (512, 16, 32), (2 ** 31 - 1, 20, 32)]
    for u, R, G in t[:-1]:
        assert R * G >= u
        assert R in bench.VARIANT_R and G in bench.VARIANT_G
    assert bench.least_padding_table([(100, 8, 8)]) == [(100, 8, 16)]


def test_gemm_traffic_only_for_the_profiled_source(monkeypatch):
    import hashlib
    with open(os.path.join(bench.ROOT, "paper_0901_2742_gb300", "csrc", "kmer_tc.cu")) as f:
        h = hashlib.sha256(f.read().encode()).hexdigest()
    want = bench.GEMM_TRAFFIC["bytes_per_launch"] if h == bench.GEMM_TRAFFIC["kmer_tc_sha256"] else None
    assert bench.gemm_traffic() == want
    monkeypatch.setattr(bench, "GEMM_TRAFFIC", dict(bench.GEMM_TRAFFIC, kmer_tc_sha256="0" * 64))
    assert bench.gemm_traffic() is None
