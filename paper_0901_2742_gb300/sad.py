"""Thin ctypes binding of libsad (include/sad.h).

Argument marshalling only: every step of the method runs in the CUDA
library. Arrays may be numpy arrays (host memory; the call is synchronous and
returns numpy arrays) or CUDA torch tensors (device memory; results are CUDA
tensors, enqueued on the current torch stream unless ``stream`` is given).
There is no CPU fallback: if the library is missing or the GPU unusable, the
calls raise.

The whole method on device tensors (residue codes 0..alphabet-1 concatenated,
int64 offsets of n + 1 entries)::

    out = sad.msa(residues, offsets, 20, 3, 16, subst, -11, -1, cap=4)
    # out["bucket_offsets"], out["order"]: the p buckets of the k-mer rank partition
    # out["colmap"]: each residue's column in its bucket's alignment
    # out["width"], out["global_colmap"]: the joined alignment of all sequences

or step by step: pipeline (rank, partition, pair scores), guide_trees,
progressive_align, ancestor_glue; align_pairs gives pairwise alignments.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SAD_OK, SAD_EINVAL, SAD_ENOMEM, SAD_ECUDA, SAD_ETIMEOUT = 0, -1, -2, -3, -4
SAD_EBUSY, SAD_ERANGE, SAD_ENOTFOUND, SAD_ECANCELED = -5, -6, -7, -8
MEM_HOST, MEM_DEVICE = 0, 1
PER_BUCKET, PERSISTENT, PERSISTENT_32 = 0, 1, 2

_NAMES = {SAD_EINVAL: "EINVAL", SAD_ENOMEM: "ENOMEM", SAD_ECUDA: "ECUDA", SAD_ETIMEOUT: "ETIMEOUT",
          SAD_EBUSY: "EBUSY", SAD_ERANGE: "ERANGE", SAD_ENOTFOUND: "ENOTFOUND",
          SAD_ECANCELED: "ECANCELED"}


class SadError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sad error {code} ({_NAMES.get(code, '?')}): {msg}")
        self.code = code


class SeqSet(ctypes.Structure):
    _fields_ = [("residues", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("alphabet", ctypes.c_int32)]


class KmerParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("kmer_alphabet", ctypes.c_int32),
                ("class_map", ctypes.c_void_p), ("cap", ctypes.c_int32), ("p", ctypes.c_int32),
                ("global_samples", ctypes.c_int32)]


class RankOut(ctypes.Structure):
    _fields_ = [("dloc", ctypes.c_void_p), ("dcen", ctypes.c_void_p), ("la", ctypes.c_void_p),
                ("ga", ctypes.c_void_p), ("key_a", ctypes.c_void_p), ("key_b", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("G", ctypes.c_void_p), ("sample_idx", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libsad.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libsad.so is not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "sad_ctx_create": (ctypes.c_int, [i32, ctypes.POINTER(ctypes.c_void_p)]),
        "sad_ctx_destroy": (ctypes.c_int, [P]),
        "sad_last_error": (ctypes.c_char_p, []),
        "sad_version": (ctypes.c_char_p, []),
        "sad_kmer_rank": (ctypes.c_int, [P, ctypes.POINTER(SeqSet), ctypes.POINTER(KmerParams),
                                         ctypes.POINTER(RankOut), i32, P]),
        "sad_partition": (ctypes.c_int, [P, i32, P, P, i32, P, P, P, i32, P]),
        "sad_partition_keys64": (ctypes.c_int, [P, i32, P, i32, P, P, P, i32, P]),
        "sad_align_pairs": (ctypes.c_int, [P, P, P, i32, P, i32, i32, P, P, P, i64, P, i32, P]),
        "sad_partition_noalloc": (ctypes.c_int, [i32, P, P, i32, P, P, P, P]),
        "sad_align_pairs_linear": (ctypes.c_int, [P, P, P, i32, P, i32, i32, P, P, P, i64, P, i32, P]),
        "sad_align_linear_bytes_per_warp": (ctypes.c_int64, [i32]),
        "sad_scores_size": (ctypes.c_int, [P, i32, i32, ctypes.POINTER(ctypes.c_int64)]),
        "sad_bucket_pair_scores": (ctypes.c_int, [P, ctypes.POINTER(SeqSet), P, P, i32, P, i32, i32,
                                                  i32, P, P, i64, i32, P]),
        "sad_scores_set_variants": (ctypes.c_int, [P, P, P, P, i32]),
        "sad_scores_autotune": (ctypes.c_int, [P, ctypes.POINTER(SeqSet), P, P, i32, P, i32, i32, P, i32, i32,
                                               i32, P]),
        "sad_scores_get_variants": (ctypes.c_int, [P, P, P, P, i32, ctypes.POINTER(ctypes.c_int32)]),
        "sad_trace_enable": (ctypes.c_int, [P, i32]),
        "sad_trace_read": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), i32]),
        "sad_kmer_gemm_work": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "sad_probe_alu": (ctypes.c_int, [i32, i32, i32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
        "sad_guide_trees": (ctypes.c_int, [P, P, i32, P, P, P, P, P, P, P, i32, P]),
        "sad_progressive_align": (ctypes.c_int, [P, P, P, P, i32, P, P, P, P, i32, i32, P, P, P, P, i32, P]),
        "sad_ancestor_glue": (ctypes.c_int, [P, P, P, P, i32, P, P, i32, P, i32, i32, P, P, P, P, i32, P]),
        "sad_progressive_columns": (ctypes.c_int, [P, i32]),
        "sad_progressive_wait_limit": (ctypes.c_int, [P, i64]),
        "sad_trace_timeline": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(ctypes.c_int32)]),
        "sad_launch_count": (ctypes.c_uint64, []),
        "sad_pipeline": (ctypes.c_int, [P, ctypes.POINTER(SeqSet), ctypes.POINTER(KmerParams), P, i32,
                                        i32, i32, ctypes.POINTER(RankOut), P, P, P, P, i64, i32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != SAD_OK:
        raise SadError(rc, load().sad_last_error().decode(errors="replace"))


def version() -> str:
    return load().sad_version().decode()


# ---- argument helpers -------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _torch():
    import torch
    return torch


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr() if x.numel() else None
    return x.ctypes.data if x.size else None


def _host(x, dtype):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _mode(*arrays) -> int:
    dev = [_is_torch(a) and a.is_cuda for a in arrays if a is not None]
    if any(dev) and not all(dev):
        raise ValueError("mix of host and device arrays")
    return MEM_DEVICE if dev and all(dev) else MEM_HOST


def _stream(stream, mem):
    if mem == MEM_HOST:
        return stream
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _empty(shape, dtype, mem, like=None):
    if mem == MEM_HOST:
        return np.zeros(shape, dtype=dtype)
    torch = _torch()
    tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.uint64,
           np.uint8: torch.uint8}[dtype]
    dev = like.device if like is not None else "cuda"
    return torch.empty(shape, dtype=tdt, device=dev)


def _as(x, dtype, mem):
    if mem == MEM_DEVICE:
        torch = _torch()
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
        return x.to(tdt).contiguous()
    return _host(x, dtype)


def _seqset(residues, offsets, alphabet):
    n = (offsets.shape[0] if _is_torch(offsets) else len(offsets)) - 1
    return SeqSet(_ptr(residues), _ptr(offsets), n, alphabet)


class Context:
    """An explicit sad_ctx (owns cached workspaces) bound to one device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(load().sad_ctx_create(device, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            _check(load().sad_ctx_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ctx(ctx):
    return None if ctx is None else ctx.handle


STAGES = ("prepare", "count", "allpairs", "rank", "partition", "scores", "scores_packed", "global", "align",
          "tree", "prog", "plane_gemm")
NESTED_STAGES = ("plane_gemm",)  # intervals that lie inside another stage's interval


def trace_enable(on: bool = True, ctx=None):
    """Record CUDA events around every stage of the context's calls."""
    _check(load().sad_trace_enable(_ctx(ctx), 1 if on else 0))


def trace_read(ctx=None) -> dict:
    """{stage: (device ms, intervals)} accumulated since the last read."""
    ms = (ctypes.c_double * len(STAGES))()
    cnt = (ctypes.c_int32 * len(STAGES))()
    _check(load().sad_trace_read(_ctx(ctx), ms, cnt, len(STAGES)))
    return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES)}


def trace_timeline(ctx=None) -> list:
    """[(stage, start ms, end ms)] of the intervals the last trace_read consumed,
    in start order, relative to the first one's start."""
    lib = load()
    n = ctypes.c_int32(0)
    _check(lib.sad_trace_timeline(_ctx(ctx), None, None, None, 0, ctypes.byref(n)))
    m = n.value
    st = (ctypes.c_int32 * max(m, 1))()
    t0 = (ctypes.c_double * max(m, 1))()
    t1 = (ctypes.c_double * max(m, 1))()
    _check(lib.sad_trace_timeline(_ctx(ctx), st, t0, t1, m, ctypes.byref(n)))
    return [(STAGES[st[i]], t0[i], t1[i]) for i in range(min(m, n.value))]


def guide_trees(bucket_offsets, score_offsets, scores, ctx=None, stream=None) -> dict:
    """sad_guide_trees: dict(merge_offsets[p+1], left, right, num, den) -- in
    bucket b merge k joins clusters left < right into nb + k at num / den."""
    mem = _mode(bucket_offsets, score_offsets, scores)
    bo = _as(bucket_offsets, np.int32, mem)
    so = _as(score_offsets, np.int64, mem)
    sc = _as(scores, np.int32, mem)
    p = bo.shape[0] - 1
    bo_h = bo.cpu().numpy() if mem == MEM_DEVICE else bo
    M = int(np.maximum(np.diff(bo_h.astype(np.int64)) - 1, 0).sum())
    mo = _empty(p + 1, np.int64, mem, bo)
    left, right = _empty(max(M, 1), np.int32, mem, bo), _empty(max(M, 1), np.int32, mem, bo)
    num, den = _empty(max(M, 1), np.int64, mem, bo), _empty(max(M, 1), np.int64, mem, bo)
    _check(load().sad_guide_trees(_ctx(ctx), _ptr(bo), p, _ptr(so), _ptr(sc), _ptr(mo), _ptr(left), _ptr(right),
                                  _ptr(num), _ptr(den), mem, _stream(stream, mem)))
    return {"merge_offsets": mo, "left": left[:M], "right": right[:M], "num": num[:M], "den": den[:M]}


def kmer_gemm_work(ctx=None) -> tuple:
    """(flops of the MMAs the last threshold-plane GEMM issued, flops of all
    its tiles' k-blocks): zero k-blocks of a panel are skipped."""
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().sad_kmer_gemm_work(_ctx(ctx), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


PROBE_MIXES = {"viaddmax_s32": 0, "vimax3_s32": 1, "viaddmax_s16x2": 2, "vimax3_s16x2": 3, "iadd": 4,
               "row_dpx3_add2": 5, "row_dpx5": 6, "row_dpx3": 7}


def probe_alu(mix: str, warps_per_sm: int = 16, iters: int = 4096) -> tuple:
    """sad_probe_alu on the current device: (lanes per clock per SM, rows per
    clock per SM) of one register-only instruction mix (PROBE_MIXES)."""
    lanes, rows = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().sad_probe_alu(PROBE_MIXES[mix], warps_per_sm, iters, ctypes.byref(lanes), ctypes.byref(rows)))
    return lanes.value, rows.value


def set_score_variants(table, ctx=None):
    """table: list of (upper_rows, R, G); [] restores the default (per pair the
    least-padding variant, the cost model for pairs longer than every strip)."""
    n = len(table)
    up = np.array([t[0] for t in table] or [0], np.int32)
    R = np.array([t[1] for t in table] or [0], np.int32)
    G = np.array([t[2] for t in table] or [0], np.int32)
    _check(load().sad_scores_set_variants(_ctx(ctx), up.ctypes.data, R.ctypes.data, G.ctypes.data, n))


DEFAULT_TUNING_BINS = (64, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1536, 2048, 4096, 2 ** 31 - 1)


def autotune_scores(residues, offsets, alphabet, bucket_offsets, order, subst, gap_open, gap_extend,
                    bins=DEFAULT_TUNING_BINS, reps=3, ctx=None, stream=None):
    """sad_scores_autotune on this layout; returns the stored variant table."""
    mem = _mode(residues, offsets, bucket_offsets, order)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    bo, od = _as(bucket_offsets, np.int32, mem), _as(order, np.int32, mem)
    S = _host(subst, np.int8)
    up = np.asarray(bins, np.int32)
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_scores_autotune(_ctx(ctx), ctypes.byref(ss), _ptr(bo), _ptr(od), bo.shape[0] - 1, S.ctypes.data,
                                      gap_open, gap_extend, up.ctypes.data, len(up), reps, mem,
                                      _stream(stream, mem)))
    return get_score_variants(ctx)


def get_score_variants(ctx=None):
    up, R, G = (np.zeros(16, np.int32) for _ in range(3))
    nb = ctypes.c_int32()
    _check(load().sad_scores_get_variants(_ctx(ctx), up.ctypes.data, R.ctypes.data, G.ctypes.data, 16,
                                          ctypes.byref(nb)))
    return [(int(up[i]), int(R[i]), int(G[i])) for i in range(nb.value)]


def launch_count() -> int:
    """Kernels launched by libsad in this process."""
    return int(load().sad_launch_count())


# ---- the calls --------------------------------------------------------------

def kmer_rank(residues, offsets, alphabet: int, k: int, p: int, cap: int = 0,
              kmer_alphabet: int | None = None, class_map=None, want_A: bool = False,
              global_samples: int = 0, ctx=None, stream=None) -> dict:
    """sad_kmer_rank: dict(dloc, dcen, la, ga, key_a, key_b, A, G, sample_idx).

    With ``global_samples`` = s >= 1 the globalized rank G[n] against s
    samples per block and the sample slots sample_idx[p*s] are filled too.
    """
    mem = _mode(residues, offsets)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    n = offs.shape[0] - 1
    cm = None if class_map is None else _host(class_map, np.uint8)
    ka = kmer_alphabet if kmer_alphabet is not None else alphabet
    params = KmerParams(k, ka, None if cm is None else cm.ctypes.data, cap, p, global_samples)
    gs = global_samples
    out = dict(dloc=_empty(max(n, 0), np.uint64, mem, offs), dcen=_empty(max(n, 0), np.uint64, mem, offs),
               la=_empty(p, np.int32, mem, offs), ga=_empty(1, np.int32, mem, offs),
               key_a=_empty(max(n, 0), np.int32, mem, offs), key_b=_empty(max(n, 0), np.int32, mem, offs),
               A=_empty((n, n), np.int32, mem, offs) if want_A else None,
               G=_empty(max(n, 0), np.uint64, mem, offs) if gs > 0 else None,
               sample_idx=_empty(p * gs, np.int32, mem, offs) if gs > 0 else None)
    ro = RankOut(*[_ptr(out[x]) if out[x] is not None and (n > 0 or x in ("la", "ga", "sample_idx")) else None
                   for x in ("dloc", "dcen", "la", "ga", "key_a", "key_b", "A", "G", "sample_idx")])
    # the C side requires non-NULL output pointers even for n == 0
    dummy = _empty(8, np.int64, mem, offs)
    for f in ("dloc", "dcen", "key_a", "key_b") + (("G",) if gs > 0 else ()):
        if getattr(ro, f) is None:
            setattr(ro, f, _ptr(dummy))
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_kmer_rank(_ctx(ctx), ctypes.byref(ss), ctypes.byref(params), ctypes.byref(ro), mem,
                                _stream(stream, mem)))
    out["ga"] = int(out["ga"][0]) if mem == MEM_HOST else out["ga"]
    return out


def partition(key_a, key_b, p: int, ctx=None, stream=None) -> dict:
    """sad_partition: dict(bucket_offsets, order, pivot_idx)."""
    mem = _mode(key_a, key_b)
    ka, kb = _as(key_a, np.int32, mem), _as(key_b, np.int32, mem)
    n = ka.shape[0]
    bo = _empty(p + 1, np.int32, mem, ka)
    order = _empty(n, np.int32, mem, ka)
    piv = _empty(max(p - 1, 0), np.int32, mem, ka)
    _check(load().sad_partition(_ctx(ctx), n, _ptr(ka), _ptr(kb), p, _ptr(bo), _ptr(order),
                                _ptr(piv) if p > 1 else None, mem, _stream(stream, mem)))
    return dict(bucket_offsets=bo, order=order, pivot_idx=piv)


def partition_keys64(keys, p: int, ctx=None, stream=None) -> dict:
    """sad_partition_keys64 on uint64 rank keys: dict(bucket_offsets, order, pivot_idx)."""
    mem = _mode(keys)
    ky = _as(keys, np.uint64, mem)
    n = ky.shape[0]
    bo = _empty(p + 1, np.int32, mem, ky)
    order = _empty(n, np.int32, mem, ky)
    piv = _empty(max(p - 1, 0), np.int32, mem, ky)
    _check(load().sad_partition_keys64(_ctx(ctx), n, _ptr(ky), p, _ptr(bo), _ptr(order),
                                       _ptr(piv) if p > 1 else None, mem, _stream(stream, mem)))
    return dict(bucket_offsets=bo, order=order, pivot_idx=piv)


def scores_size(bucket_offsets) -> int:
    mem = _mode(bucket_offsets)
    bo = _as(bucket_offsets, np.int32, mem)
    t = ctypes.c_int64()
    _check(load().sad_scores_size(_ptr(bo), bo.shape[0] - 1, mem, ctypes.byref(t)))
    return t.value


def bucket_pair_scores(residues, offsets, alphabet: int, bucket_offsets, order, subst,
                       gap_open: int, gap_extend: int, mode: int = PERSISTENT, capacity=None, ctx=None,
                       stream=None):
    """sad_bucket_pair_scores: (score_offsets int64[p+1], scores int32[total])."""
    mem = _mode(residues, offsets, bucket_offsets, order)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    bo, od = _as(bucket_offsets, np.int32, mem), _as(order, np.int32, mem)
    p = bo.shape[0] - 1
    S = _host(subst, np.int8)
    total = scores_size(bo)
    cap = total if capacity is None else capacity
    so = _empty(p + 1, np.int64, mem, bo)
    sc = _empty(max(cap, 1), np.int32, mem, bo)
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_bucket_pair_scores(_ctx(ctx), ctypes.byref(ss), _ptr(bo), _ptr(od), p, S.ctypes.data,
                                         gap_open, gap_extend, mode, _ptr(so), _ptr(sc), cap, mem,
                                         _stream(stream, mem)))
    return so, sc[:total]


def align_pairs(residues, offsets, alphabet: int, pairs, subst, gap_open: int, gap_extend: int, ctx=None,
                stream=None, linear: bool = False) -> dict:
    """sad_align_pairs (linear=False: direction bits of every cell) or
    sad_align_pairs_linear (linear=True: memory linear in the lengths):
    dict(scores, ops_offsets, ops, ops_len); pairs is (npairs, 2) sequence ids.

    ``columns(out, k)`` turns pair k's columns into a str over M, X, Y.
    """
    mem = _mode(residues, offsets, pairs)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    pr = _as(pairs, np.int32, mem)
    npairs = pr.shape[0] if pr.ndim > 1 else pr.shape[0] // 2
    S = _host(subst, np.int8)
    offs_h = offs.cpu().numpy() if mem == MEM_DEVICE else offs
    pr_h = pr.cpu().numpy() if mem == MEM_DEVICE else pr
    lens = np.diff(offs_h)
    ids = pr_h.reshape(-1)
    ids = ids[(ids >= 0) & (ids < len(lens))]   # the library reports ids out of range
    cap = int(lens[ids].sum()) if npairs else 0
    sc = _empty(max(npairs, 1), np.int32, mem, offs)
    oo = _empty(npairs + 1, np.int64, mem, offs)
    ops = _empty(max(cap, 1), np.uint8, mem, offs)
    ol = _empty(max(npairs, 1), np.int32, mem, offs)
    ss = _seqset(res, offs, alphabet)
    fn = load().sad_align_pairs_linear if linear else load().sad_align_pairs
    _check(fn(_ctx(ctx), ctypes.byref(ss), _ptr(pr), npairs, S.ctypes.data, gap_open, gap_extend, _ptr(sc), _ptr(oo),
              _ptr(ops), cap, _ptr(ol), mem, _stream(stream, mem)))
    return dict(scores=sc[:npairs], ops_offsets=oo, ops=ops, ops_len=ol[:npairs])


def align_linear_bytes_per_warp(max_len: int) -> int:
    """Device bytes of one warp of sad_align_pairs_linear for sequences of up to max_len residues."""
    return int(load().sad_align_linear_bytes_per_warp(int(max_len)))


def bucket_pairs(bucket_offsets, order):
    """Every pair (u <= v) of every bucket as sequence ids, in the layout of the
    score triangles: an int32 (npairs, 2) numpy array (host arrays or tensors in)."""
    bo = bucket_offsets.cpu().numpy() if _is_torch(bucket_offsets) else np.asarray(bucket_offsets)
    od = order.cpu().numpy() if _is_torch(order) else np.asarray(order)
    out = []
    for b in range(len(bo) - 1):
        m = od[bo[b]:bo[b + 1]].astype(np.int32)
        iu, iv = np.triu_indices(len(m))
        out.append(np.stack([m[iu], m[iv]], axis=1))
    return np.concatenate(out).astype(np.int32) if out else np.zeros((0, 2), np.int32)


def progressive_align(residues, offsets, alphabet: int, bucket_offsets, order, merge_offsets, left, right, subst,
                      gap_open: int, gap_extend: int, ctx=None, stream=None) -> dict:
    """sad_progressive_align: dict(widths[p], merge_scores[M], merge_widths[M],
    colmap) -- one multiple alignment per bucket along its guide tree; colmap
    gives the column of every residue of order[0], order[1], ... in turn."""
    mem = _mode(residues, offsets, bucket_offsets, order, merge_offsets)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    bo, od = _as(bucket_offsets, np.int32, mem), _as(order, np.int32, mem)
    mo, lt, rt = _as(merge_offsets, np.int64, mem), _as(left, np.int32, mem), _as(right, np.int32, mem)
    S = _host(subst, np.int8)
    p = bo.shape[0] - 1
    offs_h = offs.cpu().numpy() if mem == MEM_DEVICE else offs
    od_h = od.cpu().numpy() if mem == MEM_DEVICE else od
    mo_h = mo.cpu().numpy() if mem == MEM_DEVICE else mo
    lens = np.diff(offs_h)
    ids = od_h[(od_h >= 0) & (od_h < len(lens))]   # the library reports ids out of range
    total = int(lens[ids].sum())
    M = int(mo_h[-1])
    widths = _empty(p, np.int32, mem, offs)
    ms, mw = _empty(max(M, 1), np.int64, mem, offs), _empty(max(M, 1), np.int32, mem, offs)
    cm = _empty(max(total, 1), np.int32, mem, offs)
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_progressive_align(_ctx(ctx), ctypes.byref(ss), _ptr(bo), _ptr(od), p, _ptr(mo), _ptr(lt),
                                        _ptr(rt), S.ctypes.data, gap_open, gap_extend, _ptr(widths), _ptr(ms),
                                        _ptr(mw), _ptr(cm), mem, _stream(stream, mem)))
    return dict(widths=widths, merge_scores=ms[:M], merge_widths=mw[:M], colmap=cm[:total])


def progressive_columns(columns: int, ctx=None):
    """sad_progressive_columns: force 1 or 2 columns per profile-DP lane step, 0 = per batch."""
    _check(load().sad_progressive_columns(_ctx(ctx), int(columns)))


def progressive_wait_limit(polls: int, ctx=None):
    """sad_progressive_wait_limit: bound of the profile DP's strip hand-off wait
    (polls of 32 ns); 0 restores the default."""
    _check(load().sad_progressive_wait_limit(_ctx(ctx), int(polls)))


def ancestor_glue(residues, offsets, alphabet: int, bucket_offsets, order, widths, colmap, ga: int, subst,
                  gap_open: int, gap_extend: int, ctx=None, stream=None) -> dict:
    """sad_ancestor_glue: dict(ga_scores[p], anchors[sum widths], width, colmap) -- every
    bucket's alignment realigned against sequence ga and all joined through
    its positions; colmap gives the joined column of every residue."""
    mem = _mode(residues, offsets, bucket_offsets, order, widths, colmap)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    bo, od = _as(bucket_offsets, np.int32, mem), _as(order, np.int32, mem)
    wd, cm = _as(widths, np.int32, mem), _as(colmap, np.int32, mem)
    S = _host(subst, np.int8)
    p = bo.shape[0] - 1
    wd_h = wd.cpu().numpy() if mem == MEM_DEVICE else wd
    total_w = int(np.asarray(wd_h, np.int64).sum())
    scores = _empty(p, np.int64, mem, offs)
    anchors = _empty(max(total_w, 1), np.int32, mem, offs)
    gw = _empty(1, np.int32, mem, offs)
    gcm = _empty(max(cm.shape[0], 1), np.int32, mem, offs)
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_ancestor_glue(_ctx(ctx), ctypes.byref(ss), _ptr(bo), _ptr(od), p, _ptr(wd), _ptr(cm), int(ga),
                                    S.ctypes.data, gap_open, gap_extend, _ptr(scores), _ptr(anchors), _ptr(gw),
                                    _ptr(gcm), mem, _stream(stream, mem)))
    width = int(gw[0].item()) if mem == MEM_DEVICE else int(gw[0])
    return dict(ga_scores=scores, anchors=anchors[:total_w], width=width, colmap=gcm[:cm.shape[0]])


def msa(residues, offsets, alphabet: int, k: int, p: int, subst, gap_open: int, gap_extend: int, cap: int = 0,
        kmer_alphabet: int | None = None, class_map=None, ctx=None, stream=None) -> dict:
    """The whole method on device arrays: sad_pipeline (k-mer rank, partition,
    pair scores), sad_guide_trees, sad_progressive_align and sad_ancestor_glue
    with the pipeline's global ancestor. Returns dict(bucket_offsets, order, ga,
    widths, colmap (each residue's column in its bucket's alignment), width,
    global_colmap (its column in the joined alignment)); both colmaps run over
    the residues of order[0], order[1], ... in turn."""
    mem = _mode(residues, offsets)
    if mem != MEM_DEVICE:
        raise SadError(SAD_EINVAL, "msa takes device arrays (torch CUDA tensors)")
    o = pipeline(residues, offsets, alphabet, k, p, subst, gap_open, gap_extend, cap=cap,
                 kmer_alphabet=kmer_alphabet, class_map=class_map, mode=PERSISTENT, ctx=ctx, stream=stream)
    n = int(offsets.shape[0]) - 1
    total = int(o["score_offsets"][-1].item())
    t = guide_trees(o["bucket_offsets"], o["score_offsets"], o["scores"][:max(total, 1)], ctx=ctx, stream=stream)
    order = o["order"][:n]
    pa = progressive_align(residues, offsets, alphabet, o["bucket_offsets"], order, t["merge_offsets"], t["left"],
                           t["right"], subst, gap_open, gap_extend, ctx=ctx, stream=stream)
    ga = int(o["ga"].reshape(-1)[0].item())
    gl = ancestor_glue(residues, offsets, alphabet, o["bucket_offsets"], order, pa["widths"], pa["colmap"], ga, subst,
                       gap_open, gap_extend, ctx=ctx, stream=stream)
    return dict(bucket_offsets=o["bucket_offsets"], order=order, ga=ga, widths=pa["widths"], colmap=pa["colmap"],
                width=gl["width"], global_colmap=gl["colmap"])


def columns(out: dict, k: int) -> str:
    """Columns of pair k of an align_pairs result as a str over M, X, Y."""
    def h(x):
        return x.cpu().numpy() if _is_torch(x) else x
    o, n = int(h(out["ops_offsets"])[k]), int(h(out["ops_len"])[k])
    return bytes(h(out["ops"])[o:o + n]).decode()


def pipeline(residues, offsets, alphabet: int, k: int, p: int, subst, gap_open: int, gap_extend: int,
             cap: int = 0, kmer_alphabet: int | None = None, class_map=None, mode: int = PERSISTENT,
             capacity: int | None = None, want_rank: bool = True, global_samples: int = 0, ctx=None,
             stream=None, out=None) -> dict:
    """sad_pipeline: rank outputs, bucket layout and scores in one call.

    ``out`` may carry preallocated buffers (keys as in the returned dict) so
    that repeated calls reuse them.
    """
    mem = _mode(residues, offsets)
    res, offs = _as(residues, np.uint8, mem), _as(offsets, np.int64, mem)
    n = offs.shape[0] - 1
    cm = None if class_map is None else _host(class_map, np.uint8)
    ka = kmer_alphabet if kmer_alphabet is not None else alphabet
    params = KmerParams(k, ka, None if cm is None else cm.ctypes.data, cap, p, global_samples)
    S = _host(subst, np.int8)
    if capacity is None:
        capacity = n * (n + 1) // 2  # any layout fits
    o = dict(out or {})
    o.setdefault("bucket_offsets", _empty(p + 1, np.int32, mem, offs))
    o.setdefault("order", _empty(max(n, 1), np.int32, mem, offs))
    o.setdefault("score_offsets", _empty(p + 1, np.int64, mem, offs))
    o.setdefault("scores", _empty(max(capacity, 1), np.int32, mem, offs))
    ro = None
    if want_rank:
        for key, shape, dt in (("dloc", n, np.uint64), ("dcen", n, np.uint64), ("la", p, np.int32),
                               ("ga", 1, np.int32), ("key_a", n, np.int32), ("key_b", n, np.int32)):
            o.setdefault(key, _empty(max(shape, 1), dt, mem, offs))
        if global_samples > 0:
            o.setdefault("G", _empty(max(n, 1), np.uint64, mem, offs))
            o.setdefault("sample_idx", _empty(p * global_samples, np.int32, mem, offs))
        ro = RankOut(_ptr(o["dloc"]), _ptr(o["dcen"]), _ptr(o["la"]), _ptr(o["ga"]), _ptr(o["key_a"]),
                     _ptr(o["key_b"]), None, _ptr(o.get("G")) if global_samples > 0 else None,
                     _ptr(o.get("sample_idx")) if global_samples > 0 else None)
    ss = _seqset(res, offs, alphabet)
    _check(load().sad_pipeline(_ctx(ctx), ctypes.byref(ss), ctypes.byref(params), S.ctypes.data, gap_open,
                               gap_extend, mode, ctypes.byref(ro) if ro is not None else None,
                               _ptr(o["bucket_offsets"]), _ptr(o["order"]), _ptr(o["score_offsets"]),
                               _ptr(o["scores"]), capacity, mem, _stream(stream, mem)))
    return o


# ---- serving ------------------------------------------------------------------

class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("hbm_budget", ctypes.c_int64),
                ("queue_capacity", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("residues", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("alphabet", ctypes.c_int32), ("kmer", KmerParams), ("subst", ctypes.c_void_p),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int64), ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int32), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("jobs_per_s", ctypes.c_double),
                ("budget_bytes", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELLED = range(5)


def _bind_server(lib):
    if getattr(lib, "_server_bound", False):
        return lib
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "sad_server_create": [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)],
        "sad_server_submit": [P, ctypes.POINTER(Job), ctypes.POINTER(u64)],
        "sad_server_poll": [P, u64, ctypes.POINTER(i32)],
        "sad_server_wait": [P, u64, i64],
        "sad_server_result": [P, u64, P, P, P, P, i64, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)],
        "sad_server_release": [P, u64],
        "sad_server_cancel": [P, u64],
        "sad_server_get_stats": [P, ctypes.POINTER(ServerStats)],
        "sad_server_job_span": [P, u64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "sad_server_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = args
    lib._server_bound = True
    return lib


class Server:
    """Continuous-batching server of partition-and-score jobs (sad_server_*)."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 0, queue_capacity: int = 4096):
        self.lib = _bind_server(load())
        h = ctypes.c_void_p()
        cfg = ServerConfig(device, slots, hbm_budget, queue_capacity)
        _check(self.lib.sad_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, residues, offsets, alphabet, k, p, subst, gap_open, gap_extend, cap=0,
               kmer_alphabet=None, class_map=None, global_samples=0) -> int:
        res, offs = _host(residues, np.uint8), _host(offsets, np.int64)
        S = _host(subst, np.int8)
        cm = None if class_map is None else _host(class_map, np.uint8)
        kp = KmerParams(k, kmer_alphabet or alphabet, None if cm is None else cm.ctypes.data, cap, p,
                        global_samples)
        job = Job(res.ctypes.data, offs.ctypes.data, len(offs) - 1, alphabet, kp, S.ctypes.data, gap_open,
                  gap_extend)
        jid = ctypes.c_uint64()
        _check(self.lib.sad_server_submit(self.handle, ctypes.byref(job), ctypes.byref(jid)))
        self._keep[jid.value] = p
        return jid.value

    def poll(self, job_id) -> int:
        st = ctypes.c_int32()
        rc = self.lib.sad_server_poll(self.handle, job_id, ctypes.byref(st))
        if rc not in (SAD_OK,) and st.value != JOB_FAILED:
            _check(rc)
        return st.value

    def wait(self, job_id, timeout_ms: int = -1) -> int:
        """Returns the status code (SAD_OK, SAD_EBUSY on timeout, SAD_ECANCELED, or the job's error)."""
        return self.lib.sad_server_wait(self.handle, job_id, timeout_ms)

    def error(self) -> str:
        return self.lib.sad_last_error().decode(errors="replace")

    def result(self, job_id, n: int) -> dict:
        p = self._keep[job_id]
        cnt = ctypes.c_int64()
        lat = ctypes.c_double()
        _check(self.lib.sad_server_result(self.handle, job_id, None, None, None, None, 0, ctypes.byref(cnt),
                                          None) if False else SAD_OK)
        rc = self.lib.sad_server_result(self.handle, job_id, None, None, None, None, 1 << 62,
                                        ctypes.byref(cnt), ctypes.byref(lat))
        _check(rc)
        bo = np.zeros(p + 1, np.int32)
        order = np.zeros(max(n, 1), np.int32)
        so = np.zeros(p + 1, np.int64)
        sc = np.zeros(max(cnt.value, 1), np.int32)
        _check(self.lib.sad_server_result(self.handle, job_id, bo.ctypes.data, order.ctypes.data, so.ctypes.data,
                                          sc.ctypes.data, len(sc), ctypes.byref(cnt), ctypes.byref(lat)))
        return dict(bucket_offsets=bo, order=order[:n], score_offsets=so, scores=sc[:cnt.value],
                    latency_ms=lat.value)

    def span(self, job_id) -> tuple:
        """(start, end) in ms after the server's creation of the job's device work."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.sad_server_job_span(self.handle, job_id, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def release(self, job_id):
        _check(self.lib.sad_server_release(self.handle, job_id))
        self._keep.pop(job_id, None)

    def cancel(self, job_id):
        _check(self.lib.sad_server_cancel(self.handle, job_id))

    def stats(self) -> dict:
        st = ServerStats()
        _check(self.lib.sad_server_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            _check(self.lib.sad_server_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
