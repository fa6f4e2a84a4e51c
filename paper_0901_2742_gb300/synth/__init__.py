"""Seeded synthetic inputs: protein families, substitution matrices, workloads.

This module generates inputs only. Both the CUDA path's tests and the CPU
oracle's checks consume what it produces; it contains none of the method's
arithmetic. The generator itself is C (``synth.c``) so that a seed gives the
same sequences on every host architecture.

The paper's datasets (rose-generated families of N = 5000..20000 with L ~ 300,
and 2000 genome proteins of mean length 316, Section 4) are not available;
tree-evolved families with the same sizes and length mix stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "_build", "libsadsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with the host C compiler (seconds)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_families.restype = ctypes.c_int64
        lib.synth_families.argtypes = [
            ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p]
        lib.synth_subst.restype = None
        lib.synth_subst.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        lib.synth_uniform.restype = None
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
        lib.synth_uniform_f64.restype = None
        lib.synth_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


LEN_UNIFORM, LEN_NORMAL, LEN_LOGNORMAL = 0, 1, 2


def families(seed: int, family_sizes, root_len: int, len_dist: int, p1: float, p2: float,
             lo: int, hi: int, sub_total: float = 0.3, indel_total: float = 0.02,
             indel_mean: float = 3.0, alphabet: int = 20):
    """Tree-evolved families -> (residues uint8[total], offsets int64[n+1])."""
    lib = _load()
    sizes = np.ascontiguousarray(np.asarray(family_sizes, dtype=np.int32))
    n = int(sizes.sum())
    cap = max(1, n * hi)
    res = np.empty(cap, dtype=np.uint8)
    offs = np.empty(n + 1, dtype=np.int64)
    total = lib.synth_families(seed, len(sizes), sizes.ctypes.data, root_len, len_dist, p1, p2,
                               lo, hi, sub_total, indel_total, indel_mean, alphabet,
                               res.ctypes.data, cap, offs.ctypes.data)
    if total < 0:
        raise RuntimeError("synth_families: residue buffer too small")
    return res[:total].copy(), offs


def subst_matrix(seed: int, alphabet: int = 20, diag=(4, 11), off=(-4, 3)) -> np.ndarray:
    """Seeded symmetric int8 substitution matrix (alphabet x alphabet)."""
    out = np.empty((alphabet, alphabet), dtype=np.int8)
    _load().synth_subst(seed, alphabet, diag[0], diag[1], off[0], off[1], out.ctypes.data)
    return out


def uniform_residues(seed: int, count: int, alphabet: int = 20) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint8)
    _load().synth_uniform(seed, count, alphabet, out.ctypes.data)
    return out[:count]


def uniform_f64(seed: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.float64)
    _load().synth_uniform_f64(seed, count, out.ctypes.data)
    return out[:count]


def zipf_sizes(n_total: int, n_families: int, exponent: float) -> np.ndarray:
    """Family sizes proportional to f^-exponent, largest-remainder rounding, min 1."""
    w = np.arange(1, n_families + 1, dtype=np.float64) ** (-exponent)
    spare = n_total - n_families                      # every family gets 1 first
    share = w / w.sum() * spare
    base = np.floor(share).astype(np.int64)
    rem = spare - int(base.sum())
    frac_order = np.argsort(-(share - base), kind="stable")
    base[frac_order[:rem]] += 1
    return (base + 1).astype(np.int32)


def pack(seqs) -> tuple[np.ndarray, np.ndarray]:
    """List of residue arrays -> (concatenated uint8, int64 offsets)."""
    lens = [len(s) for s in seqs]
    offs = np.zeros(len(seqs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    res = np.concatenate([np.asarray(s, dtype=np.uint8) for s in seqs]) if seqs else np.zeros(0, np.uint8)
    return np.ascontiguousarray(res), offs


@dataclass
class Workload:
    """One seeded input set plus the method parameters that go with it."""
    name: str
    residues: np.ndarray          # uint8 codes 0..alphabet-1, concatenated
    offsets: np.ndarray           # int64, n+1
    alphabet: int
    subst: np.ndarray             # int8 alphabet x alphabet, symmetric
    gap_open: int
    gap_extend: int
    k: int
    p: int
    cap: int                      # 0: uint8 min-sum path; >0: threshold planes with this cap
    kmer_alphabet: int
    class_map: np.ndarray | None  # uint8[alphabet] -> 0..kmer_alphabet-1, or None
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


def compressed_class_map(alphabet: int = 20, classes: int = 6) -> np.ndarray:
    """Residue r -> floor(classes * r / alphabet): the 6-letter compressed alphabet."""
    return (np.arange(alphabet) * classes // alphabet).astype(np.uint8)


def workload(cfg: int, seed: int | None = None, n_override: int | None = None) -> Workload:
    """Seeded workloads with the shapes of the five benchmark configurations.

    1: N=64, one family, L ~ U[80,120], k=3, p=4, no cap.
    2: N=2000, 40 families x 50, L ~ Normal(316, 60) clipped [50, 800], k=3, p=16, uint8 path.
    3: the data of 2 with threshold planes (cap 4).
    4: N=20000, 400 Zipf(1.2) families, L ~ lognormal(median 300, sigma 0.6) clipped
       [50, 2000], 6-letter compressed alphabet, k=4, cap 4, p=64.
    5: one serving job: N given by n_override (100..5000), L ~ lognormal(300, 0.55)
       clipped [50, 1500], parameters of 1.
    """
    if seed is None:
        seed = 1000 + (2 if cfg == 3 else cfg)
    S = subst_matrix(seed * 7919 + 17)
    common = dict(alphabet=20, subst=S, gap_open=-11, gap_extend=-1)
    if cfg == 1:
        n = n_override or 64
        res, offs = families(seed, [n], 100, LEN_UNIFORM, 0, 0, 80, 120)
        return Workload("N=64 L~U[80,120] one family k=3 p=4", res, offs, k=3, p=4, cap=0,
                        kmer_alphabet=20, class_map=None, **common)
    if cfg in (2, 3):
        n = n_override or 2000
        fams = [50] * (n // 50) + ([n % 50] if n % 50 else [])
        res, offs = families(seed, fams, 316, LEN_NORMAL, 316.0, 60.0, 50, 800)
        cap = 0 if cfg == 2 else 4
        name = f"N={n} L~N(316,60)[50,800] {n // 50}x50 families k=3 p=16"
        return Workload(name, res, offs, k=3, p=16, cap=cap, kmer_alphabet=20, class_map=None,
                        **common)
    if cfg == 4:
        n = n_override or 20000
        nf = max(1, min(400, n // 50)) if n_override else 400
        sizes = zipf_sizes(n, nf, 1.2)
        res, offs = families(seed, sizes, 300, LEN_LOGNORMAL, 300.0, 0.6, 50, 2000)
        return Workload("N=20000 L~logN(300,0.6)[50,2000] 400 Zipf(1.2) families 6-letter k=4 "
                        "cap-4 p=64", res, offs, k=4, p=64, cap=4, kmer_alphabet=6,
                        class_map=compressed_class_map(), **common)
    if cfg == 5:
        n = n_override or 1000
        nf = max(1, n // 50)
        fams = [n // nf + (1 if i < n % nf else 0) for i in range(nf)]
        res, offs = families(seed, fams, 300, LEN_LOGNORMAL, 300.0, 0.55, 50, 1500)
        return Workload(f"serving job N={n} L~logN(300,0.55)[50,1500] k=3 p=4", res, offs, k=3,
                        p=4, cap=0, kmer_alphabet=20, class_map=None, **common)
    raise ValueError(f"unknown workload {cfg}")
