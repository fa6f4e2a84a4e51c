"""Host-side helpers of bench.py (no GPU): the device-idle summary of the
tracer's timeline, and the rule that the recorded DRAM traffic of the score
kernels is reported only for the kernel source that was profiled."""
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
