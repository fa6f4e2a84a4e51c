"""sad_partition_noalloc: the partition for callers that cannot allocate.

Some callers cannot call cudaMalloc (a latency-critical loop, a callback, an
embedding whose device memory another framework owns). For them the library
exports a partition entry point whose scratch is a fixed device array instead
of an allocated workspace. This test drives it through the C ABI on device
buffers and checks it element by element (the results are integers, so
exactly equal) against the ordinary sad_partition and against the CPU oracle:
on two calls in a row with different sizes, so that contents left in the
shared array by the first call cannot leak into the second; after a call with
a bad key, whose error flag must not outlive that call; on the degenerate
sizes (no keys, one bucket, fewer keys than buckets); and it checks that,
after one warm-up call, a call leaves the device's free memory unchanged. It
is collected last on purpose.
"""
import numpy as np
import pytest

import oracle

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


class Call:
    """Device buffers of one sad_partition_noalloc call, made before the call
    so that the call itself is the only thing that could touch device memory."""

    def __init__(self, sad, torch, ka, kb, p):
        self.lib, self.torch = sad.load(), torch
        self.n, self.p = len(ka), p
        self.ka = torch.from_numpy(np.ascontiguousarray(ka, np.int32)).cuda()
        self.kb = torch.from_numpy(np.ascontiguousarray(kb, np.int32)).cuda()
        self.bo = torch.full((p + 1,), -7, dtype=torch.int32, device="cuda")
        self.order = torch.full((max(self.n, 1),), -7, dtype=torch.int32, device="cuda")
        self.piv = torch.full((max(p - 1, 1),), -7, dtype=torch.int32, device="cuda")
        self.stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()

    def run(self):
        return self.lib.sad_partition_noalloc(self.n, self.ka.data_ptr(), self.kb.data_ptr(), self.p,
                                              self.bo.data_ptr(), self.order.data_ptr(),
                                              self.piv.data_ptr() if self.p > 1 else None, self.stream)

    def result(self):
        self.torch.cuda.synchronize()
        return (self.bo.cpu().numpy(), self.order.cpu().numpy()[:self.n],
                self.piv.cpu().numpy()[:max(self.p - 1, 0)])


def noalloc(sad, torch, ka, kb, p):
    c = Call(sad, torch, ka, kb, p)
    rc = c.run()
    assert rc == 0, c.lib.sad_last_error().decode()
    return c.result()


def check_equal(got, want):
    bo, order, piv = got
    np.testing.assert_array_equal(bo, want["bucket_offsets"])
    np.testing.assert_array_equal(order, want["order"])
    np.testing.assert_array_equal(piv, want["pivot_idx"])


def test_noalloc_matches_partition_and_oracle_on_two_calls(env):
    sad, torch = env
    for seed, n, p in ((11, 5000, 16), (12, 1999, 7)):
        ka, kb = random_keys(seed, n)
        got = noalloc(sad, torch, ka, kb, p)
        check_equal(got, sad.partition(ka, kb, p))
        check_equal(got, oracle.partition(ka, kb, p))


def test_noalloc_degenerate_sizes(env):
    sad, torch = env
    for seed, n, p in ((21, 0, 4), (22, 300, 1), (23, 3, 8), (24, 1, 1)):
        ka, kb = random_keys(seed, n)
        got = noalloc(sad, torch, ka, kb, p)
        want = sad.partition(ka, kb, p)
        np.testing.assert_array_equal(got[0], want["bucket_offsets"])
        np.testing.assert_array_equal(got[1], want["order"])
        if n > 0:
            check_equal(got, oracle.partition(ka, kb, p))


def test_noalloc_bad_key_then_good_keys(env):
    sad, torch = env
    ka, kb = random_keys(31, 700)
    bad = ka.copy()
    bad[123] = kb[123] + 1  # key_a > key_b
    c = Call(sad, torch, bad, kb, 5)
    assert c.run() == sad.SAD_EINVAL
    assert b"key" in c.lib.sad_last_error()
    # the status word is cleared by the next call: good keys give the right result
    check_equal(noalloc(sad, torch, ka, kb, 5), oracle.partition(ka, kb, 5))


def test_noalloc_leaves_free_memory_unchanged_after_warm_up(env):
    sad, torch = env
    ka, kb = random_keys(41, 20000)
    c = Call(sad, torch, ka, kb, 64)
    assert c.run() == 0  # warm-up: the library's device code (and the array) is loaded by now
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert c.run() == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    check_equal(c.result(), oracle.partition(ka, kb, 64))


def test_noalloc_rejects_sizes_beyond_its_array(env):
    sad, _ = env
    lib = sad.load()
    rc = lib.sad_partition_noalloc(262145, None, None, 4, None, None, None, None)
    assert rc == sad.SAD_EINVAL and b"262144" in lib.sad_last_error()
    rc = lib.sad_partition_noalloc(10, None, None, 257, None, None, None, None)
    assert rc == sad.SAD_EINVAL and b"256" in lib.sad_last_error()
