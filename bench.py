#!/usr/bin/env python
"""Benchmark of the Sample-Align-D data-parallel core on GB300.

One step = the whole hot path over one batch: k-mer counts, all-pairs k-mer
similarity with the fixed-point D sums, local/global ancestors, rank keys,
regular-sampling partition into p buckets, and every within-bucket
affine-gap alignment score (one sad_pipeline call). The workload is N = 2000
tree-evolved sequences with lengths ~ Normal(316, 60) clipped to [50, 800],
k = 3 over 20 letters, p = 16 buckets (seeded synthetic data standing in for
the paper's 2000 genome proteins of mean length 316).

value    = alignment cells of the scored pairs / device time of the step
           (GCUPS), inputs resident in HBM, L2 flushed between steps
e2e      = the same through the C ABI with pinned host buffers (the copies in
           the timed region)
roofline = the alignment kernel (the dominant one) against the integer-ALU
           issue peak
--impl reference runs the CPU oracle (the method as plainly written) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gotoh GCUPS + k-mer sim pairs/s (exact vs oracle); N=2000,L≈316 wall time"
# DPX instructions per DP cell: add-max (E), add-max (F), 3-way max (H); the two
# adds per cell are plain integer adds that also issue to the FMA pipe. The
# packed kernels do one row of two problems per 16x2 instruction: 1.5 per cell.
DPX_PER_CELL = 3
SMS = 152
SM_MAX_MHZ = 2070.0
# integer lanes per clock per SM: 4 sub-partitions x 16 INT32 lanes; the DPX
# instructions issue there. bench.py measures the rate they actually retire
# with sad_probe_alu in every run and reports it beside this unit count.
DPX_OPS_PER_CLK_SM = 64
# DRAM bytes (read + write) of the packed score launches of one step of this
# benchmark, summed from one ncu capture; reported while the score kernels'
# source is the one that was measured (sha256 of the device code of
# csrc/gotoh.cu: the text before its host-side planning), else null.
SCORE_TRAFFIC = {"bytes_per_step": 2182912,
                 "gotoh_device_sha256": "6dd60525784cc9be35dca38569972b6aef1059923cb06113568575d78e4605db"}
DEVICE_CODE_END = "// Host-side plan: per bucket, members sorted by length"
# DRAM bytes (read + write) of one plane-GEMM launch of this benchmark's N = 2000
# step, from one ncu capture (the launch list of the timed steps); reported while
# csrc/kmer_tc.cu is the source that was measured (sha256 of the file), else null.
GEMM_TRAFFIC = {"bytes_per_launch": 35881344,
                "kmer_tc_sha256": "af73c47a07d298c124e865cb084937f233099f78adef37bf3de8bbdd28acec9f"}


def score_traffic():
    import hashlib
    path = os.path.join(ROOT, "paper_0901_2742_gb300", "csrc", "gotoh.cu")
    with open(path) as f:
        src = f.read()
    end = src.find(DEVICE_CODE_END)
    if end < 0 or SCORE_TRAFFIC["bytes_per_step"] is None:
        return None
    if hashlib.sha256(src[:end].encode()).hexdigest() != SCORE_TRAFFIC["gotoh_device_sha256"]:
        return None
    return SCORE_TRAFFIC["bytes_per_step"]


def gemm_traffic():
    import hashlib
    with open(os.path.join(ROOT, "paper_0901_2742_gb300", "csrc", "kmer_tc.cu")) as f:
        src = f.read()
    if hashlib.sha256(src.encode()).hexdigest() != GEMM_TRAFFIC["kmer_tc_sha256"]:
        return None
    return GEMM_TRAFFIC["bytes_per_launch"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return None


def workload_cells(lengths, bucket_offsets, order):
    L = np.asarray(lengths, dtype=np.int64)
    bo, od = np.asarray(bucket_offsets), np.asarray(order)
    cells = 0
    for b in range(len(bo) - 1):
        m = L[od[bo[b]:bo[b + 1]]]
        s = int(m.sum())
        cells += (s * s + int((m * m).sum())) // 2
    return cells


def aggregate_ranks(ms_step: float, units: float, dist=None, device=None):
    """Whole-job throughput over replicas: every rank processed `units` in its
    own ms_step; the job takes the slowest rank's time. Returns
    (max ms_step over ranks, summed units, world size)."""
    if dist is None or not dist.is_initialized():
        return ms_step, units, 1
    import torch
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item()), dist.get_world_size()


def device_gaps(spans):
    """Device idle time inside the traced part of each step, from the tracer's
    timeline: a step's intervals start with its 'prepare' stage; the gap after a
    stage is the time from its end to the start of the next traced interval of
    the same step (host work and synchronisation between launches)."""
    steps, cur = [], []
    from paper_0901_2742_gb300 import sad
    spans = [sp for sp in spans if sp[0] not in sad.NESTED_STAGES]
    for sp in spans:
        if sp[0] == "prepare" and cur:
            steps.append(cur)
            cur = []
        cur.append(sp)
    if cur:
        steps.append(cur)
    if not steps:
        return None
    gap_after, busy, span = {}, 0.0, 0.0
    for st in steps:
        busy += sum(b - a for _, a, b in st)
        span += st[-1][2] - st[0][1]
        for (s0, _, b0), (_, a1, _) in zip(st, st[1:]):
            gap_after[s0] = gap_after.get(s0, 0.0) + (a1 - b0)
    k = len(steps)
    return {"traced_span_ms": span / k, "busy_ms": busy / k, "idle_ms": (span - busy) / k,
            "gap_after_ms": {s: g / k for s, g in gap_after.items()}}


def progressive_report(sad, w, res_d, offs_d, out_d, tr, bo, od, reps=3):
    """Time sad_progressive_align on the step's buckets and guide trees (the
    traced span: device time including the per-level host reads; the DP cells
    of all merges, the product of the two children's widths), then
    sad_ancestor_glue on its alignments and the step's global ancestor."""
    import torch
    sad.trace_enable(True)
    for _ in range(reps):
        pa = sad.progressive_align(res_d, offs_d, w.alphabet, out_d["bucket_offsets"], out_d["order"][:w.n],
                                   tr["merge_offsets"], tr["left"], tr["right"], w.subst, w.gap_open,
                                   w.gap_extend)
    torch.cuda.synchronize()
    span = sad.trace_read()["prog"]
    sad.trace_enable(False)
    lens = np.diff(w.offsets)[od]
    mo, lt, rt = (tr[f].cpu().numpy() for f in ("merge_offsets", "left", "right"))
    mw = pa["merge_widths"].cpu().numpy()
    cells, levels = 0, 0
    for b in range(len(bo) - 1):
        nb = int(bo[b + 1] - bo[b])
        width = list(lens[bo[b]:bo[b + 1]]) + [0] * max(nb - 1, 0)
        depth = [0] * (2 * nb)
        for k in range(max(nb - 1, 0)):
            m = int(mo[b]) + k
            cells += int(width[lt[m]]) * int(width[rt[m]])
            width[nb + k] = int(mw[m])
            depth[nb + k] = 1 + max(depth[lt[m]], depth[rt[m]])
            levels = max(levels, depth[nb + k])
    ms = span[0] / max(span[1], 1)
    # then every bucket's alignment against the global ancestor, joined through it
    ga = int(out_d["ga"].reshape(-1)[0].item())
    sad.trace_enable(True)
    for _ in range(reps):
        gl = sad.ancestor_glue(res_d, offs_d, w.alphabet, out_d["bucket_offsets"], out_d["order"][:w.n],
                               pa["widths"], pa["colmap"], ga, w.subst, w.gap_open, w.gap_extend)
    torch.cuda.synchronize()
    gspan = sad.trace_read()["prog"]
    sad.trace_enable(False)
    glue = {"kernel": "k_bucket_profiles + k_prof_scores + k_prof_dp (each bucket against the ancestor) + "
                      "k_anchors + k_glue_layout + k_joined + k_glue_residues",
            "ms": gspan[0] / max(gspan[1], 1), "ancestor": ga, "ancestor_length": int(np.diff(w.offsets)[ga]),
            "joined_width": int(gl["width"])}
    return {"kernel": "k_prof_dp (profile-profile affine-gap DP with traceback, one CTA per merge, one warp "
                      "per 64-row strip) + k_prof_scores + k_colmap", "glue": glue,
            "ms": ms, "merges": int(len(lt)), "tree_levels": int(levels), "dp_cells": int(cells),
            "gcups": cells / (ms * 1e-3) / 1e9 if ms > 0 else None,
            "alignment_widths": [int(x) for x in pa["widths"].cpu().numpy()]}


def msa_report(sad, w, res_d, offs_d, kw, reps=3):
    """Wall time of the whole method as one job (sad.msa: device arrays in, the
    joined alignment out), synchronised on both sides, after one warm-up call."""
    import torch
    args = (res_d, offs_d, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend)
    opts = dict(cap=kw["cap"], kmer_alphabet=kw["kmer_alphabet"], class_map=kw["class_map"])
    r = sad.msa(*args, **opts)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sad.msa(*args, **opts)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    return {"call": "sad.msa (pipeline, guide trees, progressive alignment, glue)",
            "ms": 1e3 * sum(times) / len(times), "joined_width": int(r["width"]), "reps": reps}


def alu_probe(sad, warps=16):
    """The rates the DP roofline is derived for, measured on this GPU by the
    library's register-only probe (sad_probe_alu): DPX lanes per clock per SM
    of the two 16x2 DPX instructions alone, and DP rows of two problems per
    clock per SM of the packed row mix (3 DPX + 2 adds)."""
    add, _ = sad.probe_alu("viaddmax_s16x2", warps)
    mx3, _ = sad.probe_alu("vimax3_s16x2", warps)
    _, rows = sad.probe_alu("row_dpx3_add2", warps)
    return {"viaddmax_s16x2_lanes_per_clk_sm": add, "vimax3_s16x2_lanes_per_clk_sm": mx3,
            "row_mix_rows_per_clk_sm": rows, "warps_per_sm": warps}


def probe_table(args):
    """--probe-alu: every mix of sad_probe_alu at 4, 8, 16 and 32 warps per SM."""
    import torch
    from paper_0901_2742_gb300 import build, sad
    build.build()
    torch.cuda.set_device(0)
    rows = []
    for mix in sad.PROBE_MIXES:
        for warps in (4, 8, 16, 32):
            lanes, r = sad.probe_alu(mix, warps)
            rows.append({"mix": mix, "warps_per_sm": warps, "lanes_per_clk_sm": round(lanes, 2),
                         "rows_per_clk_sm": round(r, 2) if r else None})
    print(json.dumps({"mode": "probe_alu", "gpu": torch.cuda.get_device_name(0), "table": rows}))
    return 0


def score_forms(sad, w, res_d, offs_d, out_d, flush, reps=3):
    """The three forms of the alignment-score stage on the same bucket layout
    and GPU: one launch per bucket (32-bit DP), one persistent launch over all
    buckets (32-bit DP), and the persistent launch with two problems per 16x2
    lane. Their score arrays must be equal. Kernel time from the tracer (the
    score launches only), call time from the host clock (synchronised on both
    sides, including the host's planning); L2 cleared before each call."""
    import torch
    n = w.n
    args = (res_d, offs_d, w.alphabet, out_d["bucket_offsets"], out_d["order"][:n], w.subst, w.gap_open,
            w.gap_extend)
    forms, ref = {}, None
    for name, mode, stage in (("per_bucket", sad.PER_BUCKET, "scores"),
                              ("persistent_32bit", sad.PERSISTENT_32, "scores"),
                              ("persistent_packed", sad.PERSISTENT, "scores_packed")):
        sad.bucket_pair_scores(*args, mode=mode)  # warm-up (plans, graphs, module load)
        torch.cuda.synchronize()
        sad.trace_enable(True)
        wall = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            so, sc = sad.bucket_pair_scores(*args, mode=mode)
            torch.cuda.synchronize()
            wall.append(time.perf_counter() - t0)
        tr = sad.trace_read()[stage]
        sad.trace_enable(False)
        got = sc.cpu().numpy()
        if ref is None:
            ref = got
        forms[name] = {"kernel_ms": tr[0] / reps, "call_ms": 1e3 * statistics.median(wall),
                       "launches_per_call": tr[1] / reps, "scores_equal_to_per_bucket": bool(np.array_equal(got, ref))}
    assert all(f["scores_equal_to_per_bucket"] for f in forms.values()), "score forms disagree"
    pb, p32, pk = (forms[k]["kernel_ms"] for k in ("per_bucket", "persistent_32bit", "persistent_packed"))
    forms["speedup_batching_32bit"] = pb / p32 if p32 > 0 else None
    forms["speedup_packing"] = p32 / pk if pk > 0 else None
    forms["speedup_total"] = pb / pk if pk > 0 else None
    return forms


def serving_report(jobs_n=200, slots=4, seed=5005):
    """Serving workload: a Poisson stream of partition-and-score jobs with N
    uniform in 100..5000 and lengths lognormal(median 300, sigma 0.55) in
    [50, 1500] (k = 3, p = 4), admitted by device memory into a continuous-
    batching server. Offline capacity = every job submitted at once; the
    stream then arrives at 0.7 x that rate. Every streamed result is compared
    with its offline run."""
    import threading

    from paper_0901_2742_gb300 import sad, synth
    rng = np.random.default_rng(seed)
    sizes = rng.integers(100, 5001, jobs_n)
    jobs = [synth.workload(5, seed=10_000 + i, n_override=int(sizes[i])) for i in range(jobs_n)]

    def run_offline():
        with sad.Server(slots=slots) as srv:
            t0 = time.perf_counter()
            ids = [srv.submit(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open, w.gap_extend)
                   for w in jobs]
            for j in ids:
                assert srv.wait(j) == sad.SAD_OK, srv.error()
            span = time.perf_counter() - t0
            outs = [srv.result(j, w.n) for j, w in zip(ids, jobs)]
            return span, outs, srv.stats()

    run_offline()  # warm-up (workspaces, module load)
    span, outs, st_off = run_offline()
    total_cells = 0
    for w, o in zip(jobs, outs):
        total_cells += workload_cells(w.lengths(), o["bucket_offsets"], o["order"])
    capacity = jobs_n / span
    rate = 0.7 * capacity
    gaps = -np.log(1.0 - synth.uniform_f64(seed + 1, jobs_n)) / rate
    arrivals = np.cumsum(gaps)
    with sad.Server(slots=slots) as srv:
        ids = [None] * jobs_n
        t0 = time.perf_counter()

        def feeder():
            for i, w in enumerate(jobs):
                delay = arrivals[i] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                ids[i] = srv.submit(w.residues, w.offsets, w.alphabet, w.k, w.p, w.subst, w.gap_open,
                                    w.gap_extend)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        for j in ids:
            assert srv.wait(j) == sad.SAD_OK, srv.error()
        span_stream = time.perf_counter() - t0
        st = srv.stats()
        same = all(np.array_equal(srv.result(j, w.n)["scores"], o["scores"]) for j, w, o in zip(ids, jobs, outs))
        # jobs on the device at once: the sum of the jobs' device intervals over their union
        spans = sorted(srv.span(j) for j in ids)
        union, end = 0.0, -1.0
        for a, b in spans:
            if a > end:
                union, end = union + b - a, b
            elif b > end:
                union, end = union + b - end, b
        concurrency = sum(b - a for a, b in spans) / union if union > 0 else None
    return {"metric": "jobs/s with p50/p99 latency (Poisson arrivals)", "value": st["jobs_per_s"],
            "unit": "jobs/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "arrival_rate_jobs_per_s": rate, "offline_jobs_per_s": capacity,
            "offline_gcups": total_cells / span / 1e9, "stream_gcups": total_cells / span_stream / 1e9,
            "offline_p50_ms": st_off["p50_ms"], "offline_p99_ms": st_off["p99_ms"],
            "jobs": jobs_n, "slots": slots, "results_identical_to_offline": bool(same),
            "device_concurrency": concurrency,
            "config": {"workload": "N ~ U{100..5000}, L ~ logN(300, 0.55) in [50, 1500], k=3, p=4, "
                                   "gap -11/-1"}}


def _kmer_distinct_counts(w):
    """Distinct k-mers of every sequence (host, numpy): the list lengths of the
    sorted-list path, for its lookup count."""
    L = np.diff(w.offsets)
    cm = w.class_map if w.class_map is not None else np.arange(w.alphabet, dtype=np.uint8)
    A2 = w.kmer_alphabet
    out = np.zeros(w.n, np.int64)
    for i in range(w.n):
        x = cm[w.residues[w.offsets[i]:w.offsets[i + 1]]].astype(np.int64)
        m = len(x) - w.k + 1
        if m <= 0:
            continue
        code = np.zeros(m, np.int64)
        for t in range(w.k):
            code = code * A2 + x[t:t + m]
        out[i] = len(np.unique(code))
    return out


def sparse_kmer_roofline(w, ap_ms):
    """The sorted-list k-mer path's all-pairs launch against the shared-memory
    port bound: one table lookup per column-list entry and row block of up to 8
    rows (columns j >= the block's first row), 32 lookups per clock per SM. The
    table is a byte per k-mer code (a presence bit per row) where the k-mer
    space fits shared memory, else a hash table of the rows' sorted lists."""
    nd = _kmer_distinct_counts(w)
    rb = (w.n + 7) // 8
    suffix = np.concatenate([np.cumsum(nd[::-1])[::-1], [0]])
    lookups = int(sum(suffix[min(8 * b, w.n)] for b in range(rb)))
    ap_s = ap_ms * 1e-3
    peak_lk = SMS * 32 * SM_MAX_MHZ * 1e6
    space = int(w.kmer_alphabet ** w.k)
    return {"bound": "shared-memory port",
            "kernel": "k_sparse_pairs (sorted k-mer lists, 8 rows per table: " +
                      ("a byte per k-mer code)" if space <= 230400 else "a hash table of the rows' lists)"),
            "kernel_ms": ap_ms, "lookups_per_launch": lookups,
            "achieved": lookups / ap_s / 1e12, "peak": peak_lk / 1e12, "unit": "T lookups/s",
            "frac": lookups / ap_s / peak_lk, "pairs_per_s": w.n * (w.n + 1) / 2 / ap_s,
            "distinct_kmers_per_sequence": float(nd.mean()), "kmer_space": space,
            "peak_basis": f"{SMS} SMs x 32 shared-memory lookups/clk x {SM_MAX_MHZ:.0f} MHz"}


def sparse_kmer_report(sad, w, res_d, offs_d, ks=(4, 5), reps=5):
    """The sorted-list k-mer path (cap -1) on this step's sequences at the
    longer words the planes cannot hold (20^4 and 20^5 codes): the k-mer stage
    alone (sad_kmer_rank, device arrays), its all-pairs launch timed by the
    tracer, against the shared-memory port bound."""
    import copy
    import torch
    rep = {"workload": f"the step's N={w.n} sequences over {w.kmer_alphabet} letters, cap -1"}
    for k in ks:
        wk = copy.copy(w)
        wk.k = k
        kw = dict(cap=-1, kmer_alphabet=w.kmer_alphabet, class_map=w.class_map)
        sad.kmer_rank(res_d, offs_d, w.alphabet, k, w.p, **kw)
        torch.cuda.synchronize()
        sad.trace_enable(True)
        for _ in range(reps):
            sad.kmer_rank(res_d, offs_d, w.alphabet, k, w.p, **kw)
        torch.cuda.synchronize()
        t = sad.trace_read()
        sad.trace_enable(False)
        r = sparse_kmer_roofline(wk, t["allpairs"][0] / max(t["allpairs"][1], 1))
        r["kmer_stage_ms"] = (t["count"][0] + t["allpairs"][0] + t["rank"][0]) / reps
        rep[f"k{k}"] = r
    return rep


def kmer_large_report(sad, peak_fp8, reps=5):
    """The threshold-plane GEMM on the large uneven workload (N = 20000, k = 4
    over the 6-letter classes, cap 4, K = 4 x 1344 bytes per sequence): the
    k-mer stage alone (sad_kmer_rank, device arrays), the GEMM launch timed by
    its own trace interval, against the same fp8 peak as the main line."""
    import torch
    from paper_0901_2742_gb300 import synth
    w = synth.workload(4)
    res = torch.from_numpy(w.residues).cuda()
    offs = torch.from_numpy(w.offsets).cuda()
    kw = dict(cap=4, kmer_alphabet=w.kmer_alphabet, class_map=w.class_map)
    sad.kmer_rank(res, offs, w.alphabet, w.k, w.p, **kw)
    torch.cuda.synchronize()
    sad.trace_enable(True)
    for _ in range(reps):
        sad.kmer_rank(res, offs, w.alphabet, w.k, w.p, **kw)
    torch.cuda.synchronize()
    t = sad.trace_read()
    sad.trace_enable(False)
    flops, dense = sad.kmer_gemm_work()
    ms = t["plane_gemm"][0] / max(t["plane_gemm"][1], 1)
    ach = flops / (ms * 1e-3) / 1e12
    stage = (t["count"][0] + t["allpairs"][0] + t["rank"][0]) / reps
    return {"workload": w.name, "kernel_ms": ms, "flops_per_launch": flops, "achieved": ach, "peak": peak_fp8,
            "frac": ach / peak_fp8, "unit": "TFLOP/s (fp8 e4m3)", "kmer_stage_ms": stage,
            "pairs_per_s": w.n * (w.n + 1) / 2 / (stage * 1e-3)}


def alignment_report(sad, w, res_d, offs_d, out_d, reps=2):
    """Every pair u <= v of every bucket of the step aligned (columns, not only
    scores) in linear space (sad_align_pairs_linear) and with every cell's
    direction bits kept (sad_align_pairs), on the same pairs: time per call
    (CUDA events on the stream around the call's kernel, from the tracer),
    GCUPS over the pairs' cells, and the device memory each form needs."""
    import torch
    pairs = sad.bucket_pairs(out_d["bucket_offsets"], out_d["order"][:w.n])
    L = np.diff(w.offsets).astype(np.int64)
    cells = int((L[pairs[:, 0]] * L[pairs[:, 1]]).sum())
    pairs_d = torch.from_numpy(pairs).to(res_d.device)
    rep = {"pairs": int(len(pairs)), "cells": cells}
    scores = {}
    for name, linear in (("linear", True), ("quadratic", False)):
        out = sad.align_pairs(res_d, offs_d, w.alphabet, pairs_d, w.subst, w.gap_open, w.gap_extend, linear=linear)
        torch.cuda.synchronize()
        sad.trace_enable(True)
        for _ in range(reps):
            out = sad.align_pairs(res_d, offs_d, w.alphabet, pairs_d, w.subst, w.gap_open, w.gap_extend,
                                  linear=linear)
        torch.cuda.synchronize()
        t = sad.trace_read()["align"]
        sad.trace_enable(False)
        ms = t[0] / reps
        scores[name] = out["scores"].cpu().numpy()
        rep[name] = {"ms": ms, "gcups": cells / (ms * 1e-3) / 1e9 if ms > 0 else None,
                     "launches_per_call": t[1] / reps}
    mx = int(L.max())
    rep["linear"]["kernel"] = "k_align_linear (rows split at the middle down to 256-row blocks)"
    rep["linear"]["device_bytes_per_warp"] = sad.align_linear_bytes_per_warp(mx)
    rep["linear"]["bytes_per_residue"] = (sad.align_linear_bytes_per_warp(mx + 1000) -
                                          sad.align_linear_bytes_per_warp(mx)) / 1000
    # direction words of the quadratic form: 4 bits per cell of every 256-row strip
    m, n = L[pairs[:, 0]], L[pairs[:, 1]]
    words = ((m + 255) // 256) * (n + 31) * 32 * ((m > 0) & (n > 0))
    rep["quadratic"]["kernel"] = "k_gotoh_trace (direction bits of every cell, batches within 1 GiB)"
    rep["quadratic"]["direction_bytes_all_pairs"] = int(4 * words.sum())
    rep["quadratic"]["direction_bytes_largest_pair"] = int(4 * words.max())
    rep["scores_equal"] = bool(np.array_equal(scores["linear"], scores["quadratic"]))
    return rep


VARIANT_R = (8, 12, 16, 20, 24, 32)
VARIANT_G = (8, 16, 32)


def least_padding_table(table):
    """Per bin of `table` (rows_le, R, G) the variant with the smallest strip
    G R that holds the bin's longest rows; ties to R <= 24, then to G nearest
    16 (at N = 2000 the 385-512 bin ran 12 % faster with R = 16, G = 32 than with
    R = 32, G = 16). The open-ended last bin keeps its variant."""
    out = []
    for u, r0, g0 in table:
        best = None
        if u < 2 ** 31 - 1:
            for R in VARIANT_R:
                for G in VARIANT_G:
                    if R * G >= u:
                        k = (R * G, 0 if R <= 24 else 1, abs(G - 16))
                        if best is None or k < best[0]:
                            best = (k, R, G)
        out.append((u, best[1], best[2]) if best else (u, r0, g0))
    return out


def refine_variants(sad, step, flush, table, reps=10, passes=2):
    """Coordinate descent over the per-bin variants of the score kernels, timed
    on this benchmark's own step (L2 flush, then the whole pipeline call; the
    mean of the score stage over `reps` steps). Some tables run in two modes
    (the score launches of the variants share the GPU, and their order on it
    varies: one measured 2.51 ms in some runs and 2.64-2.75 ms in most), and the
    library's autotuner can land on one whose fast mode its own timing loop
    meets; the mean over the step's own runs counts the slow mode. A change is
    kept when it gains 0.5 % and then wins two A/B comparisons of both tables
    measured again side by side."""
    import torch

    def measure(tb):
        sad.set_score_variants(tb)
        flush.zero_()
        step()  # new launch set: graph capture outside the timing
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            sad.trace_enable(True)
            step()
            torch.cuda.synchronize()
            ms.append(sad.trace_read()["scores_packed"][0])
            sad.trace_enable(False)
        return statistics.mean(ms)

    table = [tuple(t) for t in table]
    start = measure(table)
    # a second start: per bin the variant of least padding
    lp = least_padding_table(table)
    seed = None
    if lp != table:
        a1, b1, a2, b2 = measure(table), measure(lp), measure(table), measure(lp)
        seed = {"table": [{"rows_le": u, "R": r, "G": g} for u, r, g in lp], "scores_ms": (b1 + b2) / 2,
                "library_table_again_ms": (a1 + a2) / 2}
        if b1 + b2 < a1 + a2:
            table = lp
    best = measure(table)
    tried = 0
    for _ in range(passes):
        improved = False
        for e in range(len(table)):
            for R in VARIANT_R:
                for G in VARIANT_G:
                    if (R, G) == table[e][1:]:
                        continue
                    cand = list(table)
                    cand[e] = (table[e][0], R, G)
                    tried += 1
                    t = measure(cand)
                    if t < 0.995 * best:
                        wins, now, again = 0, best, t
                        for _ in range(2):
                            now, again = measure(table), measure(cand)
                            wins += again < 0.995 * now
                        if wins == 2:
                            table, best, improved = cand, again, True
                        else:
                            best = max(best, now)
        if not improved:
            break
    sad.set_score_variants(table)
    return table, start, best, tried, seed


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def clock_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                              "-lms", "50"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except (OSError, FileNotFoundError):
        return None, None


def clock_sampler_stop(proc, f, path, device_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as fh:
        for line in fh:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_sample(w, target_s=8.0):
    """Time the CPU oracle on a bounded sample of the workload: the full k-mer
    rank and partition, and the alignment scores of as many buckets as fit in
    about target_s seconds. Returns a cpu_baseline dict (GCUPS extrapolated
    to the whole step; the alignment time scales with cells)."""
    import oracle
    cores = oracle.default_threads()
    t0 = time.perf_counter()
    r = oracle.kmer_rank(w.residues, w.offsets, w.alphabet, w.k, w.p, class_map=w.class_map,
                         kmer_alphabet=w.kmer_alphabet, want_A=False, nthreads=cores)
    t1 = time.perf_counter()
    pt = oracle.partition(r["key_a"], r["key_b"], w.p)
    t2 = time.perf_counter()
    bo, od = pt["bucket_offsets"], pt["order"]
    L = w.lengths()
    total_cells = workload_cells(L, bo, od)
    done_cells, t_al, b = 0, 0.0, 0
    while b < w.p and (t_al < target_s or done_cells == 0):
        sub_bo = np.array([0, bo[b + 1] - bo[b]], np.int32)
        sub_od = od[bo[b]:bo[b + 1]].astype(np.int32)
        s0 = time.perf_counter()
        oracle.bucket_pair_scores(w.residues, w.offsets, sub_bo, sub_od, w.subst, w.gap_open,
                                  w.gap_extend, nthreads=cores)
        t_al += time.perf_counter() - s0
        done_cells += workload_cells(L, sub_bo, sub_od)
        b += 1
    t_step = (t1 - t0) + (t2 - t1) + t_al * total_cells / max(done_cells, 1)
    return {"value": total_cells / t_step / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": (f"full k-mer rank ({t1 - t0:.2f} s) and partition of N={w.n}; alignment of "
                       f"{b}/{w.p} buckets ({done_cells:.3e} of {total_cells:.3e} cells, "
                       f"{t_al:.2f} s), scaled to all cells"),
            "kmer_pairs_per_s": w.n * (w.n + 1) / 2 / (t1 - t0),
            "align_gcups": done_cells / t_al / 1e9}


def run_reference(args, ws, rank):
    from paper_0901_2742_gb300 import synth
    if rank != 0:
        return 0
    w = synth.workload(2)
    for _ in range(args.warmup):
        oracle_sample(w, target_s=1.0)
    vals, times = [], []
    base = None
    for _ in range(args.steps):
        s0 = time.perf_counter()
        base = oracle_sample(w, target_s=2.0)
        times.append(time.perf_counter() - s0)
        vals.append(base["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded tree-evolved families)",
            "config": {"workload": w.name, "n": w.n, "p": w.p, "k": w.k},
            "cpu_baseline": dict(base, value=v),
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_serving(args):
    """--serving: the serving workload with --jobs jobs; prints one JSON line."""
    import torch
    from paper_0901_2742_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    line = dict(serving_report(args.jobs, args.slots, args.seed), mode="serving")
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--serving", action="store_true", help="Poisson job stream through the server")
    ap.add_argument("--jobs", type=int, default=200)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--seed", type=int, default=5005)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", type=int, default=2, help="2: N=2000 paper scale; 4: N=20000")
    ap.add_argument("--cap", type=int, default=4,
                    help="0: uint8 CUDA-core k-mer path; >0 tensor-core planes; -1 sorted k-mer lists")
    ap.add_argument("--k", type=int, default=None, help="k-mer length instead of the workload's (20 letters: "
                    "k >= 4 needs the sorted-list path, --cap=-1)")
    ap.add_argument("--mode", type=int, default=1, help="0: per-bucket launches, 1: persistent")
    ap.add_argument("--no-tune", action="store_true", help="skip the per-length-bin variant autotuner")
    ap.add_argument("--no-refine", action="store_true",
                    help="keep the autotuner's table (no refinement on this benchmark's own step)")
    ap.add_argument("--variants", default=None,
                    help="fixed score-variant table instead of the autotuner: rows:R:G,... (rows ascending)")
    ap.add_argument("--global-samples", type=int, default=0,
                    help="s > 0: partition by the globalized rank against s samples per block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reports outside the timed region (score forms, serving, MSA stages)")
    ap.add_argument("--serving-jobs", type=int, default=40, help="jobs of the serving report in the bench line")
    ap.add_argument("--probe-alu", action="store_true", help="print the integer-pipe probe table and exit")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.serving:
        return run_serving(args) if rank == 0 else 0
    if args.probe_alu:
        return probe_table(args) if rank == 0 else 0

    import torch
    from paper_0901_2742_gb300 import build, sad, synth
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = synth.workload(args.workload)
    w.cap = args.cap
    if args.k is not None and args.k != w.k:
        w.name = w.name.replace(f"k={w.k}", f"k={args.k}")
        w.k = args.k
    n, p = w.n, w.p
    dev = torch.device("cuda", local)
    # work on a created stream: the library replays its batched score graph there
    # (the legacy default stream cannot be captured into a CUDA graph)
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    res_d = torch.from_numpy(w.residues).to(dev)
    offs_d = torch.from_numpy(w.offsets).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB of L2
    gs = args.global_samples
    kw = dict(cap=w.cap, kmer_alphabet=w.kmer_alphabet, class_map=w.class_map, mode=args.mode,
              global_samples=gs)
    out_d = sad.pipeline(res_d, offs_d, w.alphabet, w.k, p, w.subst, w.gap_open, w.gap_extend, **kw)
    torch.cuda.synchronize()
    bo = out_d["bucket_offsets"].cpu().numpy()
    od = out_d["order"].cpu().numpy()[:n]
    cells = workload_cells(w.lengths(), bo, od)
    pairs_scored = int(sum((bo[b + 1] - bo[b]) * (bo[b + 1] - bo[b] + 1) // 2 for b in range(p)))
    tuning = None
    t_tune = 0.0
    if args.mode == 1 and args.variants:
        tuning = [tuple(int(x) for x in v.split(":")) for v in args.variants.split(",")]
        sad.set_score_variants(tuning)
    elif args.mode == 1 and not args.no_tune:
        # pick the packed-kernel variant per query-length bin on this layout (outside the timed region)
        t_tune = time.perf_counter()
        tuning = sad.autotune_scores(res_d, offs_d, w.alphabet, out_d["bucket_offsets"],
                                     out_d["order"][:n], w.subst, w.gap_open, w.gap_extend)
        t_tune = time.perf_counter() - t_tune

    def step():
        sad.pipeline(res_d, offs_d, w.alphabet, w.k, p, w.subst, w.gap_open, w.gap_extend, out=out_d,
                     **kw)

    refine = None
    if tuning and args.mode == 1 and not args.variants and not args.no_refine:
        t_ref = time.perf_counter()
        tuned = list(tuning)
        tuning, ms0, ms1, tried, seed = refine_variants(sad, step, flush, tuning)
        refine = {"library_table": [{"rows_le": u, "R": r, "G": g} for u, r, g in tuned],
                  "library_table_scores_ms": ms0, "least_padding_start": seed, "refined_scores_ms": ms1,
                  "candidates": tried, "seconds": round(time.perf_counter() - t_ref, 2)}

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    # the clock samples of the timed region go to $SAD_CLOCKS_DIR (default: the temp directory)
    import tempfile
    clock_path = os.path.join(os.environ.get("SAD_CLOCKS_DIR") or tempfile.gettempdir(), f"clocks_rank{rank}.csv")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler, sf = clock_sampler_start(clock_path)
    time.sleep(0.3)
    sad.trace_enable(True)
    l0 = sad.launch_count()
    t0 = time.perf_counter()
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = sad.launch_count() - l0
    trace = sad.trace_read()
    timeline = device_gaps(sad.trace_timeline())
    sad.trace_enable(False)
    clocks = clock_sampler_stop(sampler, sf, clock_path, local)
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step, all_cells, _ = aggregate_ranks(sum(ms) / len(ms), float(cells), dist, dev)
    value = all_cells / (ms_step * 1e-3) / 1e9
    kmer_ms = (trace["count"][0] + trace["allpairs"][0] + trace["rank"][0]) / args.steps
    packed = trace["scores_packed"][1] > 0
    sc_ms, sc_n = trace["scores_packed"] if packed else trace["scores"]
    score_ms = sc_ms / max(sc_n, 1)
    score_launches_per_step = sc_n / args.steps
    ops_per_cell = DPX_PER_CELL / 2 if packed else DPX_PER_CELL   # 16x2: one instruction, two cells
    achieved = ops_per_cell * cells / (sc_ms / args.steps * 1e-3) / 1e12
    peak = SMS * DPX_OPS_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    probe = alu_probe(sad)
    mix_rows = probe["row_mix_rows_per_clk_sm"]

    # the k-mer all-pairs launch against the tensor-core peak (fp8: 2 x the measured bf16 burst),
    # counting the MMAs it issued (zero k-blocks of a panel are skipped)
    kmer_roofline = None
    flops, dense_flops = (sad.kmer_gemm_work() if w.cap > 0 else (0, 0))
    # the plane GEMM launch alone (its own trace interval around the kernel)
    ap_ms = trace["plane_gemm"][0] / max(trace["plane_gemm"][1], 1)
    peaks = measured_peaks()
    if flops > 0 and ap_ms > 0:
        bf16 = peaks["bf16_tflops"] if peaks else 1900.0
        peak_fp8 = 2.0 * bf16
        ach = flops / (ap_ms * 1e-3) / 1e12
        kmer_roofline = {"bound": "tensor", "achieved": ach, "peak": peak_fp8, "unit": "TFLOP/s (fp8 e4m3)",
                         "frac": ach / peak_fp8,
                         "traffic": gemm_traffic() if args.workload == 2 and w.k == 3 else None,
                         "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the "
                                          "N=2000 step, while csrc/kmer_tc.cu is the source captured",
                         "kernel": "k_plane_gemm2 (threshold-plane GEMM, tcgen05 kind::f8f6f4, fused D sums)",
                         "kernel_ms": ap_ms, "flops_per_launch": flops, "dense_flops_per_launch": dense_flops,
                         "kblocks_run_frac": flops / dense_flops if dense_flops else None,
                         "peak_basis": ("fp8 dense = 2 x the bf16 dense burst (the nominal fp8:bf16 ratio, "
                                        "4.5:2.25 PFLOP/s); bf16 " + (f"{bf16:.1f} TFLOP/s measured, of measured"
                                        if peaks else "1.9 PFLOP/s, of fallback") +
                                        "; int8 MMA (kind::i8) does not assemble for sm_103a"),
                         "pairs_per_s": n * (n + 1) / 2 / (ap_ms * 1e-3)}
        if not args.no_extras and args.workload == 2:
            kmer_roofline["large_batch"] = kmer_large_report(sad, peak_fp8)

    # the three forms of the score stage on this step's layout (outside the timed region)
    forms = None if args.no_extras else score_forms(sad, w, res_d, offs_d, out_d, flush)
    # the sorted-list k-mer path: on this step when it runs it (cap -1), else on the step's
    # sequences at k = 4 and 5 (outside the timed region)
    sparse_roofline = None
    if w.cap < 0:
        sparse_roofline = sparse_kmer_roofline(w, trace["allpairs"][0] / max(trace["allpairs"][1], 1))
    elif not args.no_extras:
        sparse_roofline = sparse_kmer_report(sad, w, res_d, offs_d)
    # the per-bucket guide trees (the progressive aligner's first step) on this step's own device
    # outputs, outside the timed region; the tracer times the tree kernel on its stream
    sad.trace_enable(True)
    tree_reps = 5
    for _ in range(tree_reps):
        tr = sad.guide_trees(out_d["bucket_offsets"], out_d["score_offsets"], out_d["scores"])
    torch.cuda.synchronize()
    tree_trace = sad.trace_read()["tree"]
    sad.trace_enable(False)
    sizes = np.diff(bo.astype(np.int64))
    guide_trees = {"kernel": "k_guide_trees (average linkage, one CTA per bucket, exact rational argmin)",
                   "ms": tree_trace[0] / max(tree_trace[1], 1), "buckets": int(p),
                   "largest_bucket": int(sizes.max()), "merges": int(tr["left"].shape[0])}
    # then the progressive alignment of every bucket along its tree (also outside the timed region)
    progressive = progressive_report(sad, w, res_d, offs_d, out_d, tr, bo, od)
    alignments = None if args.no_extras else alignment_report(sad, w, res_d, offs_d, out_d)
    msa = msa_report(sad, w, res_d, offs_d, kw)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        res_h = torch.from_numpy(w.residues).pin_memory().numpy()
        offs_h = torch.from_numpy(w.offsets).pin_memory().numpy()
        cap_scores = pairs_scored

        def pinned(shape, dt):
            return torch.zeros(shape, dtype=dt).pin_memory().numpy()

        out_h = {"bucket_offsets": pinned(p + 1, torch.int32), "order": pinned(n, torch.int32),
                 "score_offsets": pinned(p + 1, torch.int64), "scores": pinned(cap_scores, torch.int32),
                 "dloc": pinned(n, torch.int64).view(np.uint64), "dcen": pinned(n, torch.int64).view(np.uint64),
                 "la": pinned(p, torch.int32), "ga": pinned(1, torch.int32), "key_a": pinned(n, torch.int32),
                 "key_b": pinned(n, torch.int32)}
        if gs > 0:
            out_h["G"] = pinned(n, torch.int64).view(np.uint64)
            out_h["sample_idx"] = pinned(p * gs, torch.int32)

        def step_h():
            sad.pipeline(res_h, offs_h, w.alphabet, w.k, p, w.subst, w.gap_open, w.gap_extend,
                         capacity=cap_scores, out=out_h, **kw)

        for _ in range(2):
            step_h()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            step_h()
            times.append(time.perf_counter() - s0)
        e2e_s = sum(times) / len(times)
        h2d = w.residues.nbytes + w.offsets.nbytes
        d2h = 4 * pairs_scored + 8 * (p + 1) + 4 * (p + 1) + 4 * n + 8 * n * 2 + 4 * p + 4 + 4 * n * 2
        d2h += (8 * n + 4 * p * gs) if gs > 0 else 0
        e2e = {"value": ws * cells / e2e_s / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w)
    serving = None
    if ws == 1 and not args.no_extras and args.serving_jobs > 0:
        serving = serving_report(args.serving_jobs, args.slots, args.seed)
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16x2" if packed else "int32",
        "data": "synthetic (seeded tree-evolved families)",
        "config": {"workload": w.name, "n": n, "p": p, "k": w.k,
                   "kmer_path": ("sorted k-mer lists, CUDA cores" if w.cap < 0 else "uint8 min-sum, CUDA cores"
                                 if w.cap == 0 else f"cap-{w.cap} threshold planes, tensor cores"),
                   "scores_mode": "persistent" if args.mode == 1 else "one launch per bucket",
                   "rank": (f"globalized, {gs} samples per block" if gs > 0
                            else "centralized against the global ancestor"),
                   "parallelism": f"replicas x{ws}", "l2": "flushed between timed steps (256 MiB write)",
                   "score_variants": ([{"rows_le": u, "R": r, "G": g} for u, r, g in tuning]
                                      if tuning else "cost model"),
                   "autotune_s": round(t_tune, 3) if tuning and not args.variants else None,
                   "score_variant_refinement": refine},
        "kmer_pairs_per_s": n * (n + 1) / 2 / (kmer_ms * 1e-3) if kmer_ms > 0 else None,
        "stage_ms": {k: v[0] / args.steps for k, v in trace.items()},
        "device_timeline": timeline,
        "pairs_scored": pairs_scored, "cells": cells,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (DPX pipe)",
                     "frac": achieved / peak, "traffic": (score_traffic() if packed else None),
                     "kernel": ("k_gotoh_pair16 (alignment scores, two problems per 16x2 lane)" if packed
                                else "k_gotoh_items (alignment scores, 32-bit DP)"),
                     "kernel_ms": score_ms, "launches_per_step": score_launches_per_step,
                     "gcups": cells / (sc_ms / args.steps * 1e-3) / 1e9,
                     "peak_gcups": peak * 1e12 / ops_per_cell / 1e9,
                     "mix_peak_gcups": (2 * mix_rows * SMS * SM_MAX_MHZ * 1e6 / 1e9) if packed else None,
                     "frac_of_mix_peak": ((cells / (sc_ms / args.steps * 1e-3)) /
                                          (2 * mix_rows * SMS * SM_MAX_MHZ * 1e6)) if packed else None,
                     "peak_basis": f"{SMS} SMs x {DPX_OPS_PER_CLK_SM} integer lanes/clk (4 sub-partitions x 16) x "
                                   f"{SM_MAX_MHZ:.0f} MHz; {ops_per_cell:g} DPX instructions per cell (the adds "
                                   "issue to the FMA pipe too)",
                     "probe": probe,
                     "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the score launches "
                                      "of one step, while the score kernels' device code is the one captured"},
        "kmer_roofline": kmer_roofline,
        "sparse_kmer_roofline": sparse_roofline,
        "score_forms": forms,
        "serving": serving,
        "guide_trees": guide_trees,
        "progressive": progressive,
        "alignments": alignments,
        "msa": msa,
        "gpu_launches": int(launches),
        "wall_s": wall,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if gs > 0:
        from paper_0901_2742_gb300 import rank_stats
        line["rank_table"] = rank_stats.rank_table(out_d["dcen"][:n].cpu().numpy().view(np.uint64),
                                                   out_d["G"][:n].cpu().numpy().view(np.uint64),
                                                   out_d["sample_idx"].cpu().numpy())
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
