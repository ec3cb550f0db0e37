"""keccak_batch_noalloc: the ragged batch entry point for callers that cannot
allocate device memory (a process under a fixed, pre-reserved memory budget,
or a host where cudaMalloc's device-wide synchronisation is not allowed).

It must give exactly the digests of keccak_batch, the entry point that keeps
its scratch in allocated arenas, and of the CPU oracle, on two calls in a
row: the second call runs on the scratch array the first one left behind.
This file is collected last so that a run stopping at its first failure has
run every other test first.
"""
import os
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


def _oracle(oracle_mod, b):
    return oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens, len(os.sched_getaffinity(0)))


def test_noalloc_matches_keccak_batch_on_two_calls_in_a_row(oracle_mod):
    import torch

    from paper_1902_05320_gb300 import binding

    lib = binding.load()
    first = W.ragged_batch(20000, seed=901, max_len=3000, gap=5)
    second = W.ragged_batch(7000, seed=902, max_len=9000, gap=3)  # smaller: stale scratch must not leak in
    got1 = _run(torch, lib, lib.keccak_batch_noalloc, first)
    got2 = _run(torch, lib, lib.keccak_batch_noalloc, second)
    want1 = _run(torch, lib, lib.keccak_batch, first)
    want2 = _run(torch, lib, lib.keccak_batch, second)
    # Bit-exact, the tolerance of every digest test, against keccak_batch and
    # against the oracle.
    assert np.array_equal(got1, want1)
    assert np.array_equal(got2, want2)
    assert np.array_equal(got1, _oracle(oracle_mod, first))
    assert np.array_equal(got2, _oracle(oracle_mod, second))


def test_noalloc_skips_bad_descriptors(oracle_mod):
    # Messages with a variant outside 0..5 or a SHA3 output size that is not
    # the digest size are skipped: their output bytes keep the fill, and every
    # other message still gets its digest.
    import torch

    from paper_1902_05320_gb300 import binding

    lib = binding.load()
    b = W.ragged_batch(3000, seed=904, max_len=4000, gap=2)
    bad_variant = [5, 700, 2999]
    sha3 = [i for i in range(b.n) if b.variants[i] < 4 and i not in bad_variant][:3]
    b.variants[bad_variant] = 9
    b.out_lens[sha3] += 1
    got = _run(torch, lib, lib.keccak_batch_noalloc, b)
    oo = b.out_offsets()
    good = np.ones(b.n, bool)
    good[bad_variant + sha3] = False
    for i in np.flatnonzero(~good):
        assert (got[int(oo[i]):int(oo[i]) + int(b.out_lens[i])] == 0xEE).all(), i
    ok = W.RaggedBatch(b.msgs, b.offsets[good], b.lens[good], b.variants[good], b.out_lens[good])
    want = _oracle(oracle_mod, ok)
    pieces = [got[int(oo[i]):int(oo[i]) + int(b.out_lens[i])] for i in np.flatnonzero(good)]
    assert np.array_equal(np.concatenate(pieces), want)


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
