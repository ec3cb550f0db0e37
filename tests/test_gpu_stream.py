"""Streaming (incremental) hashing: messages fed in pieces over several
keccak_stream_absorb calls give exactly the one-shot digests (the sponge of
Section 3.2 paused between calls), checked against the oracle."""
import os

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))
RATES = (144, 136, 104, 72, 168, 136)


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


@pytest.mark.parametrize("seed", [321, 322])
def test_stream_pieces_at_many_block_offsets(cuda_lib, oracle_mod, seed):
    # Pieces are XORed into the lanes where they land, so the head of a piece
    # starts at any byte of the open block and at any address alignment.
    # Each call gives message i a piece of 0, 1, 2, 3 or 7 bytes, exactly the
    # bytes that close its open block, one rate, one rate plus one byte, a
    # random length below the rate, or all that is left; all six variants,
    # messages at odd offsets.
    import torch

    rng = np.random.default_rng(seed)
    n = 600
    variants = (np.arange(n) % 6).astype(np.uint8)
    rates = np.array(RATES, dtype=np.int64)[variants]
    lens = rng.integers(0, 4 * rates + 9).astype(np.uint64)
    offsets = np.zeros(n, dtype=np.uint64)
    pos = 0
    for i in range(n):
        pos += int(rng.integers(1, 8))  # odd gaps: pieces start at every alignment
        offsets[i] = pos
        pos += int(lens[i])
    msgs = W.random_bytes(pos + 8, seed=seed)
    out_lens = np.where(variants < 4, np.array([28, 32, 48, 64, 0, 0])[variants],
                        rng.integers(1, 400, size=n)).astype(np.uint32)
    states = torch.zeros(n * cuda_lib.KB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    d_msgs = _dev(torch, msgs)
    cuda_lib.keccak_stream_init(states, _dev(torch, variants), n)
    cursor = np.zeros(n, dtype=np.uint64)
    keep = []
    heads = set()
    calls = 0
    while (cursor < lens).any():
        remaining = (lens - cursor).astype(np.int64)
        close = rates - (cursor.astype(np.int64) % rates)
        choice = rng.integers(0, 10, size=n)
        plen = np.select([choice < 5, choice == 5, choice == 6, choice == 7, choice == 8],
                         [np.array([0, 1, 2, 3, 7])[np.minimum(choice, 4)], close, rates, rates + 1,
                          rng.integers(1, rates)], remaining)
        plen = np.minimum(plen, remaining).astype(np.uint64)
        heads.update(zip(variants[plen > 0].tolist(), (cursor % rates.astype(np.uint64))[plen > 0].tolist()))
        offs, pl = _dev(torch, offsets + cursor), _dev(torch, plen)
        keep += [offs, pl]
        cuda_lib.keccak_stream_absorb(states, d_msgs, offs, pl, n)
        cursor += plen
        calls += 1
    assert calls > 5
    assert len(heads) > 300  # distinct (variant, open-block offset) pairs a piece started at
    out = torch.full((int(out_lens.sum()),), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_stream_final(states, _dev(torch, out_lens), out, n)
    torch.cuda.synchronize()
    want = oracle_mod.hash_batch(msgs, offsets, lens, variants, out_lens, THREADS)
    assert np.array_equal(out.cpu().numpy(), want)
    assert cuda_lib.keccak_last_error() == 0
