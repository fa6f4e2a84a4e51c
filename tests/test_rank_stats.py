"""Table-1 statistics of the rank report (host arithmetic, no GPU)."""
import math

import numpy as np
import pytest

from paper_0901_2742_gb300 import rank_stats

TWO32 = 1 << 32


def test_ranks_at_hand_values():
    # N = 2 sequences; D = 0.9 gives log(1.0) = 0 and D = e - 0.1 gives 1
    n = 2
    dcen = np.array([int(0.9 * n * TWO32), int(0.4 * n * TWO32)], np.uint64)
    slots = np.array([0, 1, -1], np.int32)            # two filled slots
    G = np.array([int((math.e - 0.1) * 2 * TWO32), int(0.9 * 2 * TWO32)], np.uint64)
    rc, rg = rank_stats.ranks(dcen, G, slots)
    np.testing.assert_allclose(rc, [0.0, math.log(0.5)], atol=1e-9)
    np.testing.assert_allclose(rg, [1.0, 0.0], atol=1e-9)
    t = rank_stats.rank_table(dcen, G, slots)
    assert t["max_central"] == pytest.approx(0.0, abs=1e-9)
    assert t["min_central"] == pytest.approx(math.log(0.5))
    assert t["avg_global"] == pytest.approx(0.5)
    dev = np.array([1.0, -math.log(0.5)])
    assert t["var_wrt_central"] == pytest.approx(float(np.mean(dev ** 2)))
    assert t["sd_wrt_central"] == pytest.approx(math.sqrt(t["var_wrt_central"]))


def test_identical_ranks_have_zero_deviation():
    # every sequence sampled once: G equals dcen and the slot count is N
    dcen = np.array([5 * TWO32, 3 * TWO32, 7 * TWO32, 1 * TWO32], np.uint64)
    t = rank_stats.rank_table(dcen, dcen, np.arange(4))
    assert t["var_wrt_central"] == 0.0
    assert t["avg_central"] == t["avg_global"]


def test_empty_input_is_rejected():
    with pytest.raises(ValueError):
        rank_stats.rank_table(np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(3, np.int32))
    with pytest.raises(ValueError):
        rank_stats.rank_table(np.ones(2, np.uint64), np.ones(2, np.uint64), np.full(3, -1))
