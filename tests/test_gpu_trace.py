"""The tracer's timeline (sad_trace_timeline) on a real pipeline call.

Every stage of one call runs on the call's stream, one after the other, so the
traced intervals must be ordered, must not overlap, must add up per stage to
the accumulated times that sad_trace_read reports, and must cover each stage
the call ran exactly as often as that count says.
"""
import numpy as np
import pytest

from paper_0901_2742_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sad():
    from paper_0901_2742_gb300 import build, sad as s
    build.build()
    s.load()
    return s


def test_timeline_matches_stage_totals(sad):
    import torch
    torch.cuda.set_device(0)
    w = synth.workload(1)
    res = torch.from_numpy(w.residues).cuda()
    offs = torch.from_numpy(w.offsets).cuda()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        out = sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1)
        sad.trace_enable(True)
        for _ in range(3):
            sad.pipeline(res, offs, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1, out=out)
    torch.cuda.synchronize()
    totals = sad.trace_read()
    spans = sad.trace_timeline()
    sad.trace_enable(False)
    assert len(spans) == sum(c for _, c in totals.values())
    assert spans[0][1] == pytest.approx(0.0, abs=1e-6)
    for name, (ms, cnt) in totals.items():
        mine = [(a, b) for s, a, b in spans if s == name]
        assert len(mine) == cnt, name
        assert sum(b - a for a, b in mine) == pytest.approx(ms, rel=1e-3, abs=1e-3), name
    for (s0, a0, b0), (s1, a1, b1) in zip(spans, spans[1:]):
        assert b0 >= a0 and a1 >= a0
        assert a1 >= b0 - 1e-3, f"{s0} [{a0}, {b0}] overlaps {s1} [{a1}, {b1}]"
    # three calls of the same stages: each stage that ran, ran three times
    assert all(c % 3 == 0 for _, c in totals.values())
    assert totals["scores_packed"][1] == 3 and totals["allpairs"][1] == 3


def test_timeline_is_empty_before_any_read(sad):
    sad.trace_enable(True)
    assert sad.trace_timeline() == []
    sad.trace_enable(False)
