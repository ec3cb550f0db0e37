"""GPU parity of the NEXT rows at the sizes and launch configurations the
benchmark times: streaming states fed in pieces, the tree of one long
message, many small trees and the bare permutation.  Expected values come
from the oracle (sampled outputs) and from hashlib, which is independent of
both the library and the oracle; every digest is exact, so every comparison
is bit for bit."""
import hashlib
import os

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))


def _sample(rng, n, k, extra=()):
    return sorted(set(int(i) for i in rng.choice(n, k, replace=False)) | set(extra))


def test_stream_2p20_states_four_2KiB_pieces(cuda_lib, oracle_mod):
    # The benchmark's streaming workload: 2^20 SHA3-256 states, four calls of
    # a 2 KiB piece each (never a whole number of blocks, so every call
    # completes an open block and opens the next), the first fused with the
    # initialisation and the last with the padding.  Message i is its piece
    # four times over.
    import torch

    n, piece, k = 1 << 20, 2048, 4
    buf_np = W.random_bytes(n * piece, seed=20)
    buf = torch.from_numpy(buf_np).cuda()
    offs = torch.arange(n, dtype=torch.int64, device="cuda") * piece
    lens = torch.full((n,), piece, dtype=torch.int64, device="cuda")
    states = torch.empty(n * cuda_lib.KB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    variants = torch.full((n,), 1, dtype=torch.uint8, device="cuda")
    out_lens = torch.full((n,), 32, dtype=torch.int32, device="cuda")
    dig = torch.full((n * 32,), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_stream_init_absorb(states, variants, buf, offs, lens, n)
    for _ in range(k - 2):
        cuda_lib.keccak_stream_absorb(states, buf, offs, lens, n)
    cuda_lib.keccak_stream_absorb_final(states, buf, offs, lens, out_lens, dig, n)
    got = dig.cpu().numpy().reshape(n, 32)
    assert cuda_lib.keccak_last_error() == 0
    # Sampled messages against the oracle and against hashlib.
    rng = np.random.default_rng(20)
    idx = _sample(rng, n, 64, (0, n - 1))
    for i in idx:
        m = buf_np[i * piece:(i + 1) * piece].tobytes() * k
        want = oracle_mod.hash(1, m, 32)
        assert got[i].tobytes() == want == hashlib.sha3_256(m).digest(), i
    for i in _sample(rng, n, 4096):
        m = buf_np[i * piece:(i + 1) * piece].tobytes() * k
        assert got[i].tobytes() == hashlib.sha3_256(m).digest(), i
    # Every message against the one-shot fixed-stride path over the
    # concatenated pieces (itself pinned to the oracle by the parity suite).
    one = buf.view(n, piece).repeat(1, k).contiguous()
    ref = torch.empty(n * 32, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch_uniform(one, piece * k, piece * k, 1, 32, ref, n)
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy().reshape(n, 32), got)


def test_merkle_message_1GiB_in_8KiB_chunks(cuda_lib):
    # The tree of one 1 GiB message in 8 KiB chunks (131,072 leaves, 17
    # levels above them: per-level launches, then the climbing launches),
    # against the level-by-level definition computed with hashlib.
    import torch

    length, chunk = 1 << 30, 8192
    msg = W.random_bytes(length, seed=22)
    got = cuda_lib.merkle_sha3_256_message(torch.from_numpy(msg).cuda(), length, chunk)
    mv = memoryview(msg)
    level = [hashlib.sha3_256(b"\x00" + mv[i:i + chunk]).digest() for i in range(0, length, chunk)]
    while len(level) > 1:
        nxt = [hashlib.sha3_256(b"\x01" + level[2 * j] + level[2 * j + 1]).digest() for j in range(len(level) // 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    assert got == level[0]


def test_merkle_many_2p18_trees_of_16_leaves(cuda_lib, oracle_mod):
    # 2^18 trees of 16 leaves of 256 B, one thread per tree: sampled roots
    # against the oracle, and against hashlib's level-by-level tree.
    import torch

    nt, lpt, lb = 1 << 18, 16, 256
    tree = lpt * lb
    buf = W.random_bytes(nt * tree, seed=21)
    roots = torch.full((nt * 32,), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.merkle_sha3_256_many(torch.from_numpy(buf).cuda(), nt, lpt, lb, roots)
    got = roots.cpu().numpy().reshape(nt, 32)
    rng = np.random.default_rng(21)
    for t in _sample(rng, nt, 256, (0, nt - 1)):
        tb = buf[t * tree:(t + 1) * tree]
        assert got[t].tobytes() == oracle_mod.merkle_root(tb, lpt, lb), t
        level = [hashlib.sha3_256(b"\x00" + tb[i * lb:(i + 1) * lb].tobytes()).digest() for i in range(lpt)]
        while len(level) > 1:
            level = [hashlib.sha3_256(b"\x01" + level[2 * j] + level[2 * j + 1]).digest()
                     for j in range(len(level) // 2)]
        assert got[t].tobytes() == level[0], t


def _lanes_to_bits(lanes: np.ndarray, w: int) -> np.ndarray:
    # Eq. 1: string bit w(5y+x)+z is bit z of lane x+5y.
    return np.array([(int(lanes[i]) >> z) & 1 for i in range(25) for z in range(w)], dtype=np.uint8)


@pytest.mark.parametrize("b,nr", [(1600, 24), (1600, 12), (200, 18)])
def test_keccak_p_2p24_states(cuda_lib, oracle_mod, b, nr):
    # 2^24 raw states in place, the benchmark's launch: sampled states against
    # the oracle's Keccak-p[b, n_r]; Keccak-f[1600] also against hashlib's
    # SHA3-256 of one-block messages (a state holding a padded block).
    import torch

    ns, w = 1 << 24, b // 25
    states = np.frombuffer(W.random_bytes(ns * 200, seed=23 + b + nr), dtype=np.uint64).reshape(ns, 25)
    states = states & np.uint64((1 << w) - 1) if w < 64 else states
    d = torch.from_numpy(states.view(np.int64).copy()).cuda()
    cuda_lib.keccak_p_batch(d, b, nr, ns)
    got = d.cpu().numpy().view(np.uint64).reshape(ns, 25)
    rng = np.random.default_rng(b * 100 + nr)
    for i in _sample(rng, ns, 48, (0, ns - 1)):
        want = oracle_mod.keccak_p(b, nr, _lanes_to_bits(states[i], w))
        assert np.array_equal(_lanes_to_bits(got[i], w), want), (b, nr, i)
    if b == 1600 and nr == 24:
        # SHA3-256 of a 100-byte message is Keccak-f[1600] of its padded
        # block: run the same launch on 2^24 such states, check samples.
        msgs = W.random_bytes(ns * 100, seed=24).reshape(ns, 100)
        block = np.zeros((ns, 200), dtype=np.uint8)
        block[:, :100] = msgs
        block[:, 100] ^= 0x06
        block[:, 135] ^= 0x80
        d = torch.from_numpy(block.view(np.int64).reshape(ns, 25).copy()).cuda()
        cuda_lib.keccak_p_batch(d, 1600, 24, ns)
        out = d.cpu().numpy().view(np.uint8).reshape(ns, 200)
        for i in _sample(rng, ns, 256, (0, ns - 1)):
            assert out[i, :32].tobytes() == hashlib.sha3_256(msgs[i].tobytes()).digest(), i
