"""CPU oracle for the Sample-Align-D data-parallel core (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this package. It is a plain, slow, obviously correct
restatement of the method (``oracle.cpp``) and shares no code with the CUDA
library in ``paper_0901_2742_gb300``; neither imports the other.

Functions follow the paper:
  kmer_rank           Section 2 (r_ij, D_i, R_i) and the ancestor steps of the
                      algorithm box (local/global ancestor), in exact integers
  partition           Section 2.3.2 regular-sampling redistribution
  gotoh               the per-bucket sequential aligner of Section 2.3.3, as
                      global affine-gap (Gotoh) scores
  align               one optimal alignment (traceback through the same tables)
  alignment_score     the score of a given alignment, from its columns
  bucket_pair_scores  all pairs u <= v inside every bucket
  guide_trees         average-linkage (UPGMA) tree of every bucket from its
                      pair scores, the progressive aligner's first step
  progressive         progressive profile alignment of every bucket along its
                      guide tree (one multiple alignment per bucket)
  ancestor_glue       every bucket's alignment realigned against the global
                      ancestor and all buckets joined through its positions

Parity status: every function here is pinned by tests that do not reuse this
code (brute-force alignment enumeration, sorted-list k-mer intersection,
hand-worked examples under tests/golden, closed forms and invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SO = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(force: bool = False, defines: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile the oracle with g++ (plain -O2; no vector intrinsics)."""
    so = out or _SO
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if force or defines or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        cmd += [f"-D{d}" for d in defines]
        subprocess.check_call(cmd)
        os.replace(tmp, so)
    return so


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.orc_kmer_histograms.restype = i64
    lib.orc_kmer_histograms.argtypes = [P, P, i32, P, i32, i32, P, i64]
    lib.orc_kmer_rank.restype = ctypes.c_int
    lib.orc_kmer_rank.argtypes = [P, P, i32, i32, P, i32, i32, i32, i32, P, P, P, P, P, P, P]
    lib.orc_kmer_rows.restype = ctypes.c_int
    lib.orc_kmer_rows.argtypes = [P, P, i32, i32, P, i32, i32, i32, P, i32, i32, P, P, P]
    lib.orc_global_rank.restype = ctypes.c_int
    lib.orc_global_rank.argtypes = [P, P, i32, P, i32, i32, i32, i32, i32, P, P, P]
    lib.orc_partition_keys64.restype = ctypes.c_int
    lib.orc_partition_keys64.argtypes = [i32, P, i32, P, P, P]
    lib.orc_partition.restype = ctypes.c_int
    lib.orc_partition.argtypes = [i32, P, P, i32, P, P, P]
    lib.orc_gotoh.restype = i64
    lib.orc_gotoh.argtypes = [P, i32, P, i32, P, i32, i32, i32]
    lib.orc_align.restype = i64
    lib.orc_align.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, P]
    lib.orc_alignment_score.restype = ctypes.c_int
    lib.orc_alignment_score.argtypes = [P, i32, P, i32, P, i32, P, i32, i32, i32, P]
    lib.orc_bucket_pair_scores.restype = ctypes.c_int
    lib.orc_bucket_pair_scores.argtypes = [P, P, i32, P, P, i32, P, i32, i32, i32, i32, P, P]
    lib.orc_guide_trees.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.orc_progressive.restype = ctypes.c_int
    lib.orc_progressive.argtypes = [P, P, i32, P, P, i32, P, P, P, P, i32, i32, i32, i32, P, P, P, P]
    lib.orc_ancestor_glue.restype = ctypes.c_int
    lib.orc_ancestor_glue.argtypes = [P, P, i32, P, P, i32, P, P, i32, P, i32, i32, i32, i32, P, P, P, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(path: str):
    """Load a separately compiled oracle build (used to plant mistakes in tests)."""
    return _bind(ctypes.CDLL(path))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return np.ascontiguousarray(np.asarray(a, dtype=dt))


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


def kmer_histograms(residues, offsets, k, kmer_alphabet, class_map=None, lib=None):
    """Per-sequence k-mer counts as an int64 (count, 3) array of (seq, code, count)."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    cm = None if class_map is None else _c(class_map, np.uint8)
    n = len(offs) - 1
    cap = max(1, int(offs[-1]))
    out = np.empty((cap, 3), dtype=np.int64)
    got = lib.orc_kmer_histograms(_ptr(res), _ptr(offs), n, _ptr(cm), kmer_alphabet, k,
                                  out.ctypes.data, cap)
    assert got >= 0
    return out[:got]


def kmer_rank(residues, offsets, alphabet, k, p, class_map=None, kmer_alphabet=None,
              want_A=True, nthreads=None, lib=None):
    """Returns dict(A, dloc, dcen, la, ga, key_a, key_b); raises ValueError on bad input."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    n = len(offs) - 1
    cm = None if class_map is None else _c(class_map, np.uint8)
    ka = kmer_alphabet if kmer_alphabet is not None else alphabet
    A = np.zeros((n, n), dtype=np.int32) if want_A else None
    dloc = np.zeros(n, np.uint64)
    dcen = np.zeros(n, np.uint64)
    la = np.zeros(p, np.int32)
    ga = np.zeros(1, np.int32)
    key_a = np.zeros(n, np.int32)
    key_b = np.zeros(n, np.int32)
    rc = lib.orc_kmer_rank(_ptr(res), _ptr(offs), n, alphabet, _ptr(cm), ka, k, p,
                           nthreads or default_threads(), _ptr(A), _ptr(dloc), _ptr(dcen),
                           _ptr(la), _ptr(ga), _ptr(key_a), _ptr(key_b))
    if rc != 0:
        raise ValueError("oracle kmer_rank: invalid arguments")
    return dict(A=A, dloc=dloc, dcen=dcen, la=la, ga=int(ga[0]), key_a=key_a, key_b=key_b)


def kmer_rows(residues, offsets, alphabet, k, p, rows, class_map=None, kmer_alphabet=None, nthreads=None,
              lib=None):
    """Selected rows of the k-mer stage: dict(A_rows[len(rows), n], dloc, dcen) for those rows."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    n = len(offs) - 1
    cm = None if class_map is None else _c(class_map, np.uint8)
    ka = kmer_alphabet if kmer_alphabet is not None else alphabet
    rw = _c(rows, np.int32)
    A = np.zeros((len(rw), n), np.int32)
    dloc = np.zeros(len(rw), np.uint64)
    dcen = np.zeros(len(rw), np.uint64)
    rc = lib.orc_kmer_rows(_ptr(res), _ptr(offs), n, alphabet, _ptr(cm), ka, k, p, _ptr(rw), len(rw),
                           nthreads or default_threads(), _ptr(A), _ptr(dloc), _ptr(dcen))
    if rc != 0:
        raise ValueError("oracle kmer_rows: invalid arguments")
    return dict(A_rows=A, dloc=dloc, dcen=dcen)


def global_rank(residues, offsets, k, p, s, dloc, class_map=None, kmer_alphabet=20, nthreads=None, lib=None):
    """Globalized rank sums G[n] against s samples per block, and the sample indices [p*s]."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    n = len(offs) - 1
    cm = None if class_map is None else _c(class_map, np.uint8)
    dl = _c(dloc, np.uint64)
    G = np.zeros(max(n, 1), np.uint64)
    smp = np.zeros(p * s, np.int32)
    rc = lib.orc_global_rank(_ptr(res), _ptr(offs), n, _ptr(cm), kmer_alphabet, k, p, s,
                             nthreads or default_threads(), _ptr(dl), _ptr(G), _ptr(smp))
    if rc != 0:
        raise ValueError("oracle global_rank: invalid arguments")
    return G[:n], smp


def partition_keys64(keys, p, lib=None):
    """Regular sampling on uint64 keys: dict(bucket_offsets, order, pivot_idx)."""
    lib = lib or _load()
    ky = _c(keys, np.uint64)
    n = len(ky)
    bo = np.zeros(p + 1, np.int32)
    order = np.zeros(max(n, 1), np.int32)
    piv = np.zeros(max(p - 1, 1), np.int32)
    rc = lib.orc_partition_keys64(n, _ptr(ky), p, _ptr(bo), _ptr(order), _ptr(piv))
    if rc != 0:
        raise ValueError("oracle partition_keys64: invalid arguments")
    return dict(bucket_offsets=bo, order=order[:n], pivot_idx=piv[:max(p - 1, 0)])


def partition(key_a, key_b, p, lib=None):
    """Returns dict(bucket_offsets[p+1], order[n], pivot_idx[p-1])."""
    lib = lib or _load()
    ka, kb = _c(key_a, np.int32), _c(key_b, np.int32)
    n = len(ka)
    bo = np.zeros(p + 1, np.int32)
    order = np.zeros(max(n, 1), np.int32)
    piv = np.zeros(max(p - 1, 1), np.int32)
    rc = lib.orc_partition(n, _ptr(ka), _ptr(kb), p, _ptr(bo), _ptr(order), _ptr(piv))
    if rc != 0:
        raise ValueError("oracle partition: invalid arguments")
    return dict(bucket_offsets=bo, order=order[:n], pivot_idx=piv[:max(p - 1, 0)])


def gotoh(x, y, subst, gap_open, gap_extend, lib=None) -> int:
    lib = lib or _load()
    x, y = _c(x, np.uint8), _c(y, np.uint8)
    S = _c(subst, np.int8)
    return int(lib.orc_gotoh(_ptr(x), len(x), _ptr(y), len(y), _ptr(S), S.shape[0], gap_open,
                             gap_extend))


def align(x, y, subst, gap_open, gap_extend, lib=None):
    """One optimal alignment: (score, columns) with columns a str over M, X, Y."""
    lib = lib or _load()
    x, y = _c(x, np.uint8), _c(y, np.uint8)
    S = _c(subst, np.int8)
    buf = ctypes.create_string_buffer(max(1, len(x) + len(y)))
    n = ctypes.c_int32(0)
    sc = lib.orc_align(_ptr(x), len(x), _ptr(y), len(y), _ptr(S), S.shape[0], gap_open, gap_extend, buf,
                       ctypes.byref(n))
    return int(sc), buf.raw[:n.value].decode()


def alignment_score(x, y, columns, subst, gap_open, gap_extend, lib=None):
    """Score of a given alignment (str or bytes over M, X, Y); None if it is not an alignment of x and y."""
    lib = lib or _load()
    x, y = _c(x, np.uint8), _c(y, np.uint8)
    S = _c(subst, np.int8)
    cols = columns.encode() if isinstance(columns, str) else bytes(columns)
    out = ctypes.c_int64(0)
    rc = lib.orc_alignment_score(_ptr(x), len(x), _ptr(y), len(y), cols, len(cols), _ptr(S), S.shape[0],
                                 gap_open, gap_extend, ctypes.byref(out))
    return None if rc != 0 else int(out.value)


def bucket_pair_scores(residues, offsets, bucket_offsets, order, subst, gap_open, gap_extend,
                       nthreads=None, lib=None):
    """Returns (score_offsets int64[p+1], scores int32[total])."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    bo, od = _c(bucket_offsets, np.int32), _c(order, np.int32)
    S = _c(subst, np.int8)
    p = len(bo) - 1
    nb = np.diff(bo).astype(np.int64)
    total = int((nb * (nb + 1) // 2).sum())
    so = np.zeros(p + 1, np.int64)
    scores = np.zeros(max(total, 1), np.int32)
    rc = lib.orc_bucket_pair_scores(_ptr(res), _ptr(offs), len(offs) - 1, _ptr(bo), _ptr(od), p,
                                    _ptr(S), S.shape[0], gap_open, gap_extend,
                                    nthreads or default_threads(), _ptr(so), _ptr(scores))
    if rc != 0:
        raise ValueError("oracle bucket_pair_scores: invalid arguments")
    return so, scores[:total]


def guide_trees(bucket_offsets, score_offsets, scores, lib=None):
    """Average-linkage guide tree of every bucket (see oracle.cpp): returns
    dict(merge_offsets int64[p+1], left, right int32[M], num, den int64[M]); in
    bucket b merge k joins clusters left < right into nb + k at distance num/den."""
    lib = lib or _load()
    bo = _c(bucket_offsets, np.int32)
    so, sc = _c(score_offsets, np.int64), _c(scores, np.int32)
    p = len(bo) - 1
    nb = np.diff(bo).astype(np.int64)
    M = int(np.maximum(nb - 1, 0).sum())
    mo = np.zeros(p + 1, np.int64)
    left, right = np.zeros(max(M, 1), np.int32), np.zeros(max(M, 1), np.int32)
    num, den = np.zeros(max(M, 1), np.int64), np.zeros(max(M, 1), np.int64)
    lib.orc_guide_trees(_ptr(bo), p, _ptr(so), _ptr(sc if sc.size else np.zeros(1, np.int32)), _ptr(mo),
                        _ptr(left), _ptr(right), _ptr(num), _ptr(den))
    return {"merge_offsets": mo, "left": left[:M], "right": right[:M], "num": num[:M], "den": den[:M]}


def progressive(residues, offsets, bucket_offsets, order, merge_offsets, left, right, subst, gap_open, gap_extend,
                nthreads=None, lib=None):
    """Progressive alignment of every bucket along its guide tree (see
    oracle.cpp): dict(widths int32[p], merge_scores int64[M], merge_widths
    int32[M], colmap int32[residues]); colmap runs over the residues of
    order[0], order[1], ... and gives each one's column in its bucket's
    alignment."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    bo, od = _c(bucket_offsets, np.int32), _c(order, np.int32)
    mo, lf, rt = _c(merge_offsets, np.int64), _c(left, np.int32), _c(right, np.int32)
    sub = _c(subst, np.int8)
    n, p = len(offs) - 1, len(bo) - 1
    alphabet = int(round(np.sqrt(sub.size)))
    M = int(mo[-1])
    total = int(sum(offs[od[q] + 1] - offs[od[q]] for q in range(len(od))))
    widths = np.zeros(p, np.int32)
    ms, mw = np.zeros(max(M, 1), np.int64), np.zeros(max(M, 1), np.int32)
    colmap = np.zeros(max(total, 1), np.int32)
    one = np.zeros(1, np.int32)
    rc = lib.orc_progressive(_ptr(res if res.size else np.zeros(1, np.uint8)), _ptr(offs), n, _ptr(bo),
                             _ptr(od if od.size else one), p, _ptr(mo), _ptr(lf if lf.size else one),
                             _ptr(rt if rt.size else one), _ptr(sub), alphabet, int(gap_open), int(gap_extend),
                             nthreads or default_threads(), _ptr(widths), _ptr(ms), _ptr(mw), _ptr(colmap))
    if rc != 0:
        raise ValueError("orc_progressive: the merges do not form a tree")
    return {"widths": widths, "merge_scores": ms[:M], "merge_widths": mw[:M], "colmap": colmap[:total]}


def ancestor_glue(residues, offsets, bucket_offsets, order, widths, colmap, ga, subst, gap_open, gap_extend,
                  nthreads=None, lib=None):
    """Realignment of every bucket's alignment against sequence ga and the glue
    (see oracle.cpp): dict(ga_scores int64[p], anchors int32[sum widths],
    width int, colmap int32[residues])."""
    lib = lib or _load()
    res, offs = _c(residues, np.uint8), _c(offsets, np.int64)
    bo, od = _c(bucket_offsets, np.int32), _c(order, np.int32)
    wd, cm = _c(widths, np.int32), _c(colmap, np.int32)
    sub = _c(subst, np.int8)
    n, p = len(offs) - 1, len(bo) - 1
    alphabet = int(round(np.sqrt(sub.size)))
    sc = np.zeros(p, np.int64)
    an = np.zeros(max(int(wd.sum()), 1), np.int32)
    gw = np.zeros(1, np.int32)
    gc = np.zeros(max(cm.size, 1), np.int32)
    one = np.zeros(1, np.int32)
    rc = lib.orc_ancestor_glue(_ptr(res if res.size else np.zeros(1, np.uint8)), _ptr(offs), n, _ptr(bo),
                               _ptr(od if od.size else one), p, _ptr(wd), _ptr(cm if cm.size else one), int(ga),
                               _ptr(sub), alphabet, int(gap_open), int(gap_extend), nthreads or default_threads(),
                               _ptr(sc), _ptr(an), _ptr(gw), _ptr(gc))
    if rc != 0:
        raise ValueError("orc_ancestor_glue: invalid arguments")
    return {"ga_scores": sc, "anchors": an[:int(wd.sum())], "width": int(gw[0]), "colmap": gc[:cm.size]}


def tri_index(u: int, v: int, nb: int) -> int:
    """Position of pair (u, v), u <= v, in a bucket's row-major upper triangle."""
    return u * nb - u * (u - 1) // 2 + (v - u)
