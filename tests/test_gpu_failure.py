"""Failure detection on the GPU without a fault: the staging kernel's bounded
mbarrier wait, run on a barrier whose phase nothing completes, gives up after
its limit, reports KB_DEV_TIMEOUT through the device status word, and leaves
the context usable; on a barrier that completes, it returns at once."""
import time

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _clean_hash_still_works(cuda_lib, oracle_mod):
    import torch

    n = 4096
    msgs = W.uniform_messages(n, 64, seed=77)
    out = torch.empty(n * 32, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch_uniform(torch.from_numpy(msgs).cuda(), 64, 64, 1, 32, out, n)
    want = oracle_mod.hash_batch(msgs, np.arange(n, dtype=np.uint64) * np.uint64(64), np.full(n, 64, np.uint64),
                                 np.full(n, 1, np.uint8), np.full(n, 32, np.uint32))
    assert np.array_equal(out.cpu().numpy(), want)
    assert cuda_lib.keccak_last_error() == 0


def test_wait_that_nothing_completes_times_out_and_reports(cuda_lib, oracle_mod):
    import torch

    cuda_lib.keccak_last_error()  # start from a clean status word
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cuda_lib.wait_timeout_probe(20_000_000)  # 20 ms
    status = cuda_lib.keccak_last_error()    # synchronises
    elapsed = time.perf_counter() - t0
    assert status & cuda_lib.KB_DEV_TIMEOUT
    assert 0.015 < elapsed < 5.0
    _clean_hash_still_works(cuda_lib, oracle_mod)


def test_wait_that_completes_returns_at_once(cuda_lib, oracle_mod):
    cuda_lib.keccak_last_error()
    t0 = time.perf_counter()
    cuda_lib.wait_timeout_probe(2_000_000_000, arrive=True)  # would take 2 s if it timed out
    assert cuda_lib.keccak_last_error() == 0
    assert time.perf_counter() - t0 < 1.0
    _clean_hash_still_works(cuda_lib, oracle_mod)
