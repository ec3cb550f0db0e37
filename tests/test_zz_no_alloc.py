"""keccak_batch_noalloc: the ragged batch entry point for callers that cannot
allocate device memory (a process under a fixed, pre-reserved memory budget,
or a host where cudaMalloc's device-wide synchronisation is not allowed).

It must give exactly the digests of keccak_batch, the entry point that keeps
its scratch in allocated arenas, on two calls in a row: the second call runs
on the scratch array the first one left behind.  This file is collected last
so that a run stopping at its first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint64): np.int64, np.dtype(np.uint32): np.int32}.get(a.dtype)
    return torch.from_numpy(a.view(view) if view is not None else a).cuda()


def _run(torch, lib, fn, b):
    # The device copies stay referenced until the work has finished.
    args = [_dev(torch, a) for a in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.full((max(b.total_out(), 1),), 0xEE, dtype=torch.uint8, device="cuda")
    status = fn(*[t.data_ptr() for t in args], out.data_ptr(), b.n, torch.cuda.current_stream().cuda_stream)
    assert status == 0, status
    torch.cuda.synchronize()
    result = out.cpu().numpy()[: b.total_out()]
    del args
    return result


def test_noalloc_matches_keccak_batch_on_two_calls_in_a_row():
    import torch

    from paper_1902_05320_gb300 import binding

    lib = binding.load()
    first = W.ragged_batch(20000, seed=901, max_len=3000, gap=5)
    second = W.ragged_batch(7000, seed=902, max_len=9000, gap=3)  # smaller: stale scratch must not leak in
    got1 = _run(torch, lib, lib.keccak_batch_noalloc, first)
    got2 = _run(torch, lib, lib.keccak_batch_noalloc, second)
    want1 = _run(torch, lib, lib.keccak_batch, first)
    want2 = _run(torch, lib, lib.keccak_batch, second)
    # Bit-exact, the tolerance of every digest test.
    assert np.array_equal(got1, want1)
    assert np.array_equal(got2, want2)


def test_noalloc_size_limit_and_empty_batch():
    import torch

    from paper_1902_05320_gb300 import binding

    lib = binding.load()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.keccak_batch_noalloc(None, None, None, None, None, None, 0, stream) == binding.KB_OK
    # One message beyond the maximum is refused before anything is read.
    too_many = binding.KB_NOALLOC_MAX_MESSAGES + 1
    assert lib.keccak_batch_noalloc(1 << 20, 1 << 20, 1 << 20, 1 << 20, 1 << 20, 1 << 20, too_many,
                                    stream) == binding.KB_ERR_TOO_LARGE
    # The largest allowed batch still matches keccak_batch.
    b = W.ragged_batch(binding.KB_NOALLOC_MAX_MESSAGES, seed=903, max_len=200)
    assert np.array_equal(_run(torch, lib, lib.keccak_batch_noalloc, b), _run(torch, lib, lib.keccak_batch, b))
