"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/sad.h declares. Argument validation that happens before any device
work is checked too (no GPU is touched)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "sad.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sad_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0901_2742_gb300 import build, sad
    build.build()
    return sad.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sad_kmer_rank", "sad_partition", "sad_bucket_pair_scores", "sad_pipeline",
                 "sad_scores_size", "sad_ctx_create", "sad_ctx_destroy", "sad_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    from paper_0901_2742_gb300 import build
    assert "compute_103a" in build.ARCH and "sm_103a" in build.ARCH


def test_version_and_error_string(lib):
    from paper_0901_2742_gb300 import sad
    assert "sm_103a" in sad.version()
    assert isinstance(lib.sad_last_error(), bytes)


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_0901_2742_gb300 import sad
    res = np.zeros(4, np.uint8)
    offs = np.array([0, 4], np.int64)
    for kw in (dict(k=0, p=2), dict(k=3, p=0), dict(k=3, p=2, cap=9), dict(k=9, p=2),
               dict(k=3, p=2, global_samples=-1), dict(k=3, p=2, global_samples=1025),
               dict(k=4, p=2, cap=4), dict(k=3, p=2, cap=-2), dict(k=8, p=2, cap=-1)):
        with pytest.raises(sad.SadError) as e:
            sad.kmer_rank(res, offs, 20, **kw)
        assert e.value.code == sad.SAD_EINVAL
    for p in (0, 1025):
        with pytest.raises(sad.SadError) as e:
            sad.partition_keys64(np.zeros(3, np.uint64), p)
        assert e.value.code == sad.SAD_EINVAL
    # asymmetric substitution matrix and positive gap costs
    S = np.zeros((20, 20), np.int8)
    S[0, 1] = 1
    with pytest.raises(sad.SadError) as e:
        sad.bucket_pair_scores(res, offs, 20, np.array([0, 1], np.int32), np.array([0], np.int32), S, -11, -1)
    assert e.value.code == sad.SAD_EINVAL
    with pytest.raises(sad.SadError) as e:
        sad.bucket_pair_scores(res, offs, 20, np.array([0, 1], np.int32), np.array([0], np.int32),
                               np.zeros((20, 20), np.int8), 3, -1)
    assert e.value.code == sad.SAD_EINVAL


def test_scores_size_host(lib):
    from paper_0901_2742_gb300 import sad
    assert sad.scores_size(np.array([0, 3, 3, 7], np.int32)) == 6 + 0 + 10


def test_linear_alignment_scratch_grows_with_the_length(lib):
    from paper_0901_2742_gb300 import sad
    b = [sad.align_linear_bytes_per_warp(L) for L in (100, 1000, 10000)]
    # 152 bytes per residue of the longer sequence: 6 int32 vectors and 32 direction words
    assert b[1] - b[0] == 900 * 152 and b[2] - b[1] == 9000 * 152
    assert sad.align_linear_bytes_per_warp(-1) == -1
