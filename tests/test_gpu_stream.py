"""Streaming (incremental) hashing: messages fed in pieces over several
keccak_stream_absorb calls give exactly the one-shot digests (the sponge of
Section 3.2 paused between calls), checked against the oracle."""
import os

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint64): np.int64, np.dtype(np.uint32): np.int32}.get(a.dtype)
    return torch.from_numpy(a.view(view) if view is not None else a).cuda()


@pytest.mark.parametrize("seed,calls", [(301, 1), (302, 4), (303, 9)])
def test_stream_pieces_equal_one_shot(cuda_lib, oracle_mod, seed, calls):
    import torch

    b = W.ragged_batch(400, seed=seed, max_len=3000, gap=3)
    n = b.n
    states = torch.zeros(n * cuda_lib.KB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    d_msgs = _dev(torch, b.msgs)
    cuda_lib.keccak_stream_init(states, _dev(torch, b.variants), n)
    rng = np.random.default_rng(seed)
    cursor = np.zeros(n, dtype=np.uint64)
    keep = []
    for c in range(calls):
        remaining = b.lens - cursor
        if c == calls - 1:
            plen = remaining
        else:  # random pieces, often empty, often crossing block boundaries
            plen = (rng.random(n) * remaining.astype(np.float64) * rng.choice([0.0, 0.3, 1.0], size=n)).astype(
                np.uint64)
        offs, lens = _dev(torch, b.offsets + cursor), _dev(torch, plen)
        keep += [offs, lens]
        cuda_lib.keccak_stream_absorb(states, d_msgs, offs, lens, n)
        cursor += plen
    assert (cursor == b.lens).all()
    out = torch.full((b.total_out(),), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_stream_final(states, _dev(torch, b.out_lens), out, n)
    torch.cuda.synchronize()
    want = oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens, THREADS)
    assert np.array_equal(out.cpu().numpy(), want)
    assert cuda_lib.keccak_last_error() == 0
    # A finalised state refuses further pieces and a second final.
    cuda_lib.keccak_stream_absorb(states, d_msgs, _dev(torch, b.offsets), _dev(torch, b.lens), n)
    assert cuda_lib.keccak_last_error() != 0


def test_stream_matches_oracle_incremental_form(cuda_lib, oracle_mod):
    # One SHAKE128 message of 1000 bytes fed as 17, 0, 151, 832 bytes, output
    # 400 bytes (three squeeze blocks), against the oracle's incremental sponge.
    import torch

    msg = W.random_bytes(1000, seed=9)
    pieces = (17, 0, 151, 832)
    states = torch.zeros(cuda_lib.KB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    d_msg = torch.from_numpy(msg).cuda()
    cuda_lib.keccak_stream_init(states, torch.tensor([4], dtype=torch.uint8, device="cuda"), 1)
    inc = oracle_mod.Incremental(4)
    pos = 0
    for p in pieces:
        cuda_lib.keccak_stream_absorb(states, d_msg, torch.tensor([pos], dtype=torch.int64, device="cuda"),
                                      torch.tensor([p], dtype=torch.int64, device="cuda"), 1)
        inc.absorb(msg[pos:pos + p])
        pos += p
    out = torch.zeros(400, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_stream_final(states, torch.tensor([400], dtype=torch.int32, device="cuda"), out, 1)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tobytes() == inc.final(400) == oracle_mod.hash(4, msg.tobytes(), 400)


@pytest.mark.parametrize("seed,calls", [(311, 2), (312, 5)])
def test_fused_first_and_last_steps(cuda_lib, oracle_mod, seed, calls):
    # keccak_stream_init_absorb takes the first piece with the initialisation
    # and keccak_stream_absorb_final the last piece with the padding and
    # squeeze: the digests equal the one-shot hashes, pieces of any length
    # (empty ones, ones crossing block boundaries, unaligned starts).
    import torch

    b = W.ragged_batch(500, seed=seed, max_len=4000, gap=5)
    n = b.n
    states = torch.zeros(n * cuda_lib.KB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    d_msgs = _dev(torch, b.msgs)
    rng = np.random.default_rng(seed)
    cursor = np.zeros(n, dtype=np.uint64)
    keep = []
    out = torch.full((b.total_out(),), 0xEE, dtype=torch.uint8, device="cuda")
    for c in range(calls):
        remaining = b.lens - cursor
        if c == calls - 1:
            plen = remaining
        else:
            plen = (rng.random(n) * remaining.astype(np.float64) * rng.choice([0.0, 0.4, 1.0], size=n)).astype(
                np.uint64)
        offs, lens = _dev(torch, b.offsets + cursor), _dev(torch, plen)
        keep += [offs, lens]
        if c == 0:
            cuda_lib.keccak_stream_init_absorb(states, _dev(torch, b.variants), d_msgs, offs, lens, n)
        elif c == calls - 1:
            cuda_lib.keccak_stream_absorb_final(states, d_msgs, offs, lens, _dev(torch, b.out_lens), out, n)
        else:
            cuda_lib.keccak_stream_absorb(states, d_msgs, offs, lens, n)
        cursor += plen
    torch.cuda.synchronize()
    want = oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens, THREADS)
    assert np.array_equal(out.cpu().numpy(), want)
    assert cuda_lib.keccak_last_error() == 0
    # A finalised state refuses a further final step.
    cuda_lib.keccak_stream_absorb_final(states, d_msgs, _dev(torch, b.offsets), _dev(torch, b.lens),
                                        _dev(torch, b.out_lens), out, n)
    assert cuda_lib.keccak_last_error() != 0
