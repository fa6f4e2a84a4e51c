"""Summary statistics of the k-mer ranks, centralized against globalized
(Section 2.3.1, Table 1), computed on the host from the exact fixed-point
sums the library returns. This is a report for display, outside the exact
integer path: nothing orders or partitions by these floating-point values.

Rank of sequence i (Section 2, R_i = log(0.1 + D_i), natural logarithm):
  centralized  D_i = (1/N) sum over all j of r_ij          = dcen_i / (N 2^32)
  globalized   D_i = (1/S) sum over the S sample slots of r = G_i / (S 2^32)
where S counts the sample slots that hold a sequence. The deviation
statistics are those of R_glob - R_cen over the sequences: the variance
about the centralized rank is the mean of the squared differences, and the
standard deviation its square root.
"""
from __future__ import annotations

import math

import numpy as np

_TWO32 = float(1 << 32)


def ranks(dcen, G, sample_idx):
    """(R_central, R_global) as float64 arrays."""
    dcen = np.asarray(dcen, dtype=np.uint64)
    G = np.asarray(G, dtype=np.uint64)
    n = dcen.shape[0]
    slots = int((np.asarray(sample_idx) >= 0).sum())
    if n == 0 or slots == 0:
        raise ValueError("ranks need at least one sequence and one sample slot")
    d_cen = dcen.astype(np.float64) / (n * _TWO32)
    d_glob = G.astype(np.float64) / (slots * _TWO32)
    return np.log(0.1 + d_cen), np.log(0.1 + d_glob)


def rank_table(dcen, G, sample_idx) -> dict:
    """The rows of Table 1 for one set: extremes and means of both ranks, and
    the variance and standard deviation of the globalized rank about the
    centralized one."""
    rc, rg = ranks(dcen, G, sample_idx)
    dev = rg - rc
    var = float(np.mean(dev * dev))
    return {
        "max_central": float(rc.max()), "min_central": float(rc.min()), "avg_central": float(rc.mean()),
        "max_global": float(rg.max()), "min_global": float(rg.min()), "avg_global": float(rg.mean()),
        "var_wrt_central": var, "sd_wrt_central": math.sqrt(var),
    }
