"""Serving loop (sad_server_*): continuous batching of partition-and-score jobs.

Jobs of different N run concurrently on one GPU; each result must be
bit-identical to the same job run alone, and to the oracle. Failures are made
on the host side (a budget too small, a bad residue code, a cancelled job);
none of them faults or hangs the GPU.
"""
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


def job_workloads(count, seed0=500):
    rng = np.random.default_rng(seed0)
    return [synth.workload(5, seed=seed0 + i, n_override=int(rng.integers(100, 1200))) for i in range(count)]


def alone(sad, w):
    o = sad.pipeline(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend, mode=1,
                     want_rank=False)
    total = int(o["score_offsets"][-1])
    return o["bucket_offsets"], o["order"][:w.n], o["score_offsets"], o["scores"][:total]


def submit(srv, w):
    return srv.submit(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend)


def test_results_identical_alone_and_in_the_mix(sad):
    ws = job_workloads(16)
    ref = [alone(sad, w) for w in ws]
    with sad.Server(slots=4) as srv:
        ids = [submit(srv, w) for w in ws]
        for jid, w, (bo, od, so, sc) in zip(ids, ws, ref):
            assert srv.wait(jid, 120000) == sad.SAD_OK, srv.error()
            got = srv.result(jid, w.n)
            np.testing.assert_array_equal(got["bucket_offsets"], bo)
            np.testing.assert_array_equal(got["order"], od)
            np.testing.assert_array_equal(got["score_offsets"], so)
            np.testing.assert_array_equal(got["scores"], sc)
            assert got["latency_ms"] > 0
            srv.release(jid)
        st = srv.stats()
        assert st["done"] == len(ws) and st["failed"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"]
    # one job against the oracle as well
    w = ws[0]
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p)
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    so, sc = oracle.bucket_pair_scores(w.residues, w.offsets, pt["bucket_offsets"], pt["order"], w.subst,
                                       w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(ref[0][3], sc)


def test_admission_refused_when_the_budget_is_short(sad):
    w = job_workloads(1, seed0=900)[0]
    with sad.Server(slots=1, hbm_budget=1 << 20) as srv:
        with pytest.raises(sad.SadError) as e:
            submit(srv, w)
        assert e.value.code == sad.SAD_ENOMEM


def test_malformed_job_fails_alone(sad):
    ws = job_workloads(4, seed0=700)
    bad = synth.workload(5, seed=777, n_override=200)
    bad.residues = bad.residues.copy()
    bad.residues[5] = 25          # residue code outside the 20-letter alphabet
    with sad.Server(slots=2) as srv:
        ids = [submit(srv, w) for w in ws[:2]] + [submit(srv, bad)] + [submit(srv, w) for w in ws[2:]]
        rcs = [srv.wait(j, 120000) for j in ids]
        assert rcs[2] == sad.SAD_EINVAL
        assert [rc for i, rc in enumerate(rcs) if i != 2] == [sad.SAD_OK] * 4
        ref = alone(sad, ws[3])
        np.testing.assert_array_equal(srv.result(ids[4], ws[3].n)["scores"], ref[3])
        assert srv.stats()["failed"] == 1


def test_cancel_a_queued_job(sad):
    big = synth.workload(5, seed=801, n_override=3000)
    small = job_workloads(3, seed0=810)
    with sad.Server(slots=1) as srv:
        first = submit(srv, big)
        queued = [submit(srv, w) for w in small]
        srv.cancel(queued[1])
        assert srv.wait(queued[1], 120000) == sad.SAD_ECANCELED
        assert srv.wait(first, 120000) == sad.SAD_OK
        assert srv.wait(queued[0], 120000) == sad.SAD_OK
        assert srv.wait(queued[2], 120000) == sad.SAD_OK
        assert srv.stats()["cancelled"] == 1


def test_jobs_in_the_mix_overlap_on_the_device(sad):
    """Continuous batching: jobs submitted together run on the device at the same
    time (their device intervals, from CUDA events on the workers' streams,
    intersect), and every result is the job's result alone."""
    ws = job_workloads(8, seed0=600)
    ref = [alone(sad, w) for w in ws]
    with sad.Server(slots=4) as srv:
        ids = [submit(srv, w) for w in ws]
        for jid in ids:
            assert srv.wait(jid, 120000) == sad.SAD_OK, srv.error()
        spans = [srv.span(j) for j in ids]
        for jid, w, r in zip(ids, ws, ref):
            np.testing.assert_array_equal(srv.result(jid, w.n)["scores"], r[3])
    assert all(0 <= a < b for a, b in spans)
    overlapping = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                      if max(spans[i][0], spans[j][0]) < min(spans[i][1], spans[j][1]))
    assert overlapping >= 3, spans
    # busy time of the union is below the sum of the intervals: work ran side by side
    union, end = 0.0, -1.0
    for a, b in sorted(spans):
        if a > end:
            union += b - a
            end = b
        elif b > end:
            union += b - end
            end = b
    assert union < 0.9 * sum(b - a for a, b in spans)
