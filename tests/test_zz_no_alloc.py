"""sad_partition_noalloc: the partition for callers that cannot allocate.

Some callers cannot call cudaMalloc (a latency-critical loop, a callback, an
embedding whose device memory another framework owns). For them the library
exports a partition entry point whose scratch is a fixed device array instead
of an allocated workspace. This test drives it through the C ABI on device
buffers and checks it against the ordinary sad_partition, element by element
(the results are integers, so exactly equal), on two calls in a row with
different sizes, so that contents left in the shared array by the first call
cannot leak into the second. It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_0901_2742_gb300 import build, sad
    build.build()
    sad.load()
    return sad, torch


def random_keys(seed, n):
    rng = np.random.default_rng(seed)
    kb = rng.integers(1, 60, n).astype(np.int32)
    ka = (rng.random(n) * (kb + 1)).astype(np.int32).clip(0, kb)
    return ka, kb


def noalloc(sad, torch, ka, kb, p):
    lib = sad.load()
    n = len(ka)
    dka = torch.from_numpy(ka).cuda()
    dkb = torch.from_numpy(kb).cuda()
    bo = torch.full((p + 1,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    piv = torch.full((max(p - 1, 1),), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sad_partition_noalloc(n, dka.data_ptr(), dkb.data_ptr(), p, bo.data_ptr(), order.data_ptr(),
                                   piv.data_ptr() if p > 1 else None, stream)
    assert rc == 0, lib.sad_last_error().decode()
    torch.cuda.synchronize()
    return bo.cpu().numpy(), order.cpu().numpy()[:n], piv.cpu().numpy()[:max(p - 1, 0)]


def test_noalloc_matches_partition_on_two_calls(env):
    sad, torch = env
    for seed, n, p in ((11, 5000, 16), (12, 1999, 7)):
        ka, kb = random_keys(seed, n)
        want = sad.partition(ka, kb, p)
        bo, order, piv = noalloc(sad, torch, ka, kb, p)
        np.testing.assert_array_equal(bo, want["bucket_offsets"])
        np.testing.assert_array_equal(order, want["order"])
        np.testing.assert_array_equal(piv, want["pivot_idx"])


def test_noalloc_rejects_sizes_beyond_its_array(env):
    sad, _ = env
    lib = sad.load()
    rc = lib.sad_partition_noalloc(262145, None, None, 4, None, None, None, None)
    assert rc == sad.SAD_EINVAL and b"262144" in lib.sad_last_error()
    rc = lib.sad_partition_noalloc(10, None, None, 257, None, None, None, None)
    assert rc == sad.SAD_EINVAL and b"256" in lib.sad_last_error()
