"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Every digest is an exact function of its message (FIPS 202, which the paper
restates in Section 3), so the tolerance is zero everywhere.  Inputs come from
the seeded generators in paper_1902_05320_gb300.workloads; expected values only
from the oracle (or, for the 4 GiB Merkle root, from hashlib).
"""
import hashlib
import os

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RATES = (144, 136, 104, 72, 168, 136)
DIG = (28, 32, 48, 64, None, None)
THREADS = len(os.sched_getaffinity(0))


def _torch():
    import torch

    return torch


def dev(a: np.ndarray):
    torch = _torch()
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint64): np.int64, np.dtype(np.uint32): np.int32}.get(a.dtype)
    t = torch.from_numpy(a.view(view) if view is not None else a)
    return t.cuda()


def host(t) -> np.ndarray:
    _torch().cuda.synchronize()
    return t.cpu().numpy().view(np.uint8).reshape(-1)


def oracle_uniform(oracle_mod, msgs, stride, length, variant, out_len, n, idx=None):
    idx = np.arange(n) if idx is None else np.asarray(idx)
    offs = (idx.astype(np.uint64) * np.uint64(stride))
    k = idx.size
    return oracle_mod.hash_batch(msgs, offs, np.full(k, length, np.uint64), np.full(k, variant, np.uint8),
                                 np.full(k, out_len, np.uint32), THREADS).reshape(k, out_len)


def gpu_uniform(cuda_lib, msgs_np, stride, length, variant, out_len, n, base_shift=0):
    torch = _torch()
    buf = torch.zeros(msgs_np.size + base_shift + 16, dtype=torch.uint8, device="cuda")
    if msgs_np.size:
        buf[base_shift:base_shift + msgs_np.size] = dev(msgs_np)
    out = torch.full((max(n * out_len, 1),), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch_uniform(buf.data_ptr() + base_shift, stride, length, variant, out_len, out, n)
    return host(out)[: n * out_len].reshape(n, out_len)


# -- the 4096 x 64 B SHA3-256 batch, every digest ----------------------------------
def test_sha3_256_4096_messages_of_64_bytes(cuda_lib, oracle_mod):
    n, L = 4096, 64
    msgs = W.uniform_messages(n, L, seed=0)
    got = gpu_uniform(cuda_lib, msgs, L, L, 1, 32, n)
    want = oracle_uniform(oracle_mod, msgs, L, L, 1, 32, n)
    assert np.array_equal(got, want)


# -- fixed-stride batches: every variant, padding boundary and alignment ------------
@pytest.mark.parametrize("variant", range(6))
def test_uniform_lengths_and_alignments(cuda_lib, oracle_mod, variant):
    r = RATES[variant]
    rng = np.random.default_rng(100 + variant)
    n = 200  # spans two 128-thread blocks with a ragged tail
    for L in (0, 1, 7, 8, 63, 64, 65, r - 2, r - 1, r, r + 1, 2 * r + 3, 700):
        out_len = DIG[variant] or int(rng.choice([0, 1, 32, r - 1, r, r + 1, 2 * r + 5]))
        for stride, shift in ((-(-max(L, 1) // 16) * 16, 0), (L + 3, 1), (L, 2)):
            stride = max(stride, 1) if L == 0 else stride
            msgs = W.random_bytes((n - 1) * stride + L, seed=int(rng.integers(1 << 30)))
            got = gpu_uniform(cuda_lib, msgs, stride, L, variant, out_len, n, base_shift=shift)
            want = oracle_uniform(oracle_mod, msgs, stride, L, variant, out_len, n)
            assert np.array_equal(got, want), (variant, L, stride, shift, out_len)


@pytest.mark.parametrize("n", [1, 127, 128, 200, 4096 + 77, 152 * 6 * 128 * 2 + 5])
@pytest.mark.parametrize("variant", [1, 3, 5])
@pytest.mark.parametrize("staging", [0, 1])
def test_uniform_64_byte_staging(cuda_lib, oracle_mod, restore_tuning, n, variant, staging):
    # 64-byte messages back to back, loaded directly (0) and through the
    # bulk-copy staging kernel (1): partial last tiles, one tile, and more
    # tiles than the grid holds at once.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_STAGING, staging)
    out_len = DIG[variant] or 200
    msgs = W.uniform_messages(n, 64, seed=900 + n)
    got = gpu_uniform(cuda_lib, msgs, 64, 64, variant, out_len, n)
    want = oracle_uniform(oracle_mod, msgs, 64, 64, variant, out_len, n)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, (bad.size, bad[:16])
    assert cuda_lib.keccak_last_error() == 0


@pytest.mark.parametrize("out_len", [0, 1, 31, 168, 169, 337])
@pytest.mark.parametrize("staging", [0, 1])
def test_uniform_64_byte_shake_output_lengths(cuda_lib, oracle_mod, restore_tuning, out_len, staging):
    # SHAKE128 of 64-byte messages: empty, short, exactly one rate block and
    # just past it, two blocks; loaded directly and staged by bulk copies.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_STAGING, staging)
    n = 300
    msgs = W.uniform_messages(n, 64, seed=950 + out_len)
    if out_len == 0:
        torch = _torch()
        buf = dev(msgs)
        out = torch.full((16,), 0xEE, dtype=torch.uint8, device="cuda")
        cuda_lib.keccak_batch_uniform(buf, 64, 64, 4, 0, out, n)
        assert (host(out) == 0xEE).all()
        return
    got = gpu_uniform(cuda_lib, msgs, 64, 64, 4, out_len, n)
    want = oracle_uniform(oracle_mod, msgs, 64, 64, 4, out_len, n)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("staging", [0, 1])
def test_long_shake_outputs(cuda_lib, oracle_mod, restore_tuning, staging):
    # Outputs of hundreds of squeeze blocks, fixed-stride and ragged.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_STAGING, staging)
    msgs = W.uniform_messages(5, 64, seed=990)
    got = gpu_uniform(cuda_lib, msgs, 64, 64, 5, 70001, 5)
    want = oracle_uniform(oracle_mod, msgs, 64, 64, 5, 70001, 5)
    assert np.array_equal(got, want)
    b = W.ragged_batch(3, seed=991, lens=np.array([0, 300, 5000]), gap=3)
    b.variants = np.array([4, 5, 1], dtype=np.uint8)
    b.out_lens = np.array([100003, 1, 32], dtype=np.uint32)
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))


@pytest.mark.parametrize("n,length,variant", [(119040, 10, 1), (121601, 10, 1), (250000, 10, 1), (60000, 100, 5),
                                              (33, 7, 3)])
def test_uniform_one_block_batches_around_one_wave(cuda_lib, oracle_mod, n, length, variant):
    # One-block messages: a batch that one wave of single-warp blocks holds
    # runs as that wave (119,040 is the paper's largest batch); larger ones
    # take the grid-stride split.  Every digest against the oracle.
    msgs = W.uniform_messages(n, length, seed=n + length)
    out_len = 32 if variant == 5 else [28, 32, 48, 64][variant]
    got = gpu_uniform(cuda_lib, msgs, length, length, variant, out_len, n)
    want = oracle_uniform(oracle_mod, msgs, length, length, variant, out_len, n)
    assert np.array_equal(got, want)


def test_uniform_zero_stride_and_single_message(cuda_lib, oracle_mod):
    msgs = W.random_bytes(300, seed=5)
    got = gpu_uniform(cuda_lib, msgs, 0, 300, 3, 64, 37)
    want = oracle_mod.hash(3, msgs.tobytes())
    assert all(row.tobytes() == want for row in got)
    got1 = gpu_uniform(cuda_lib, msgs, 300, 300, 5, 1000, 1)
    assert got1[0].tobytes() == oracle_mod.hash(5, msgs.tobytes(), 1000)


# -- ragged, mixed-variant batches ----------------------------------------------------
def _run_ragged(cuda_lib, b: W.RaggedBatch, sentinel=0xEE):
    torch = _torch()
    out = torch.full((max(b.total_out(), 1),), sentinel, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch(dev(b.msgs), dev(b.offsets), dev(b.lens), dev(b.variants), dev(b.out_lens), out, b.n)
    return host(out)[: b.total_out()]


def _oracle_ragged(oracle_mod, b: W.RaggedBatch):
    return oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens, THREADS)


@pytest.mark.parametrize("seed,n,max_len,gap", [(11, 3000, 1500, 7), (12, 300, 65536, 3), (13, 1, 50, 0),
                                                (14, 129, 300, 0)])
def test_ragged_batch_matches_oracle(cuda_lib, oracle_mod, seed, n, max_len, gap):
    b = W.ragged_batch(n, seed=seed, max_len=max_len, gap=gap)
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))
    assert cuda_lib.keccak_last_error() == 0


def test_ragged_every_padding_case(cuda_lib, oracle_mod):
    # For each variant: len mod r in {0, 1, r-2, r-1} plus the empty message.
    lens, variants = [], []
    for v in range(6):
        r = RATES[v]
        for L in (0, 1, r - 2, r - 1, r, r + 1, 2 * r - 1, 2 * r):
            lens.append(L)
            variants.append(v)
    rng = np.random.default_rng(3)
    order = rng.permutation(len(lens))
    b = W.ragged_batch(len(lens), seed=21, lens=np.array(lens)[order], gap=5)
    b.variants = np.array(variants, dtype=np.uint8)[order]
    b.out_lens = np.array([DIG[v] or int(rng.integers(0, 600)) for v in b.variants], dtype=np.uint32)
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))


def test_ragged_shake_every_output_length(cuda_lib, oracle_mod):
    # SHAKE outputs of every length 0..520 (one, two, three and four squeeze
    # blocks), packed back to back so that the output starts fall on every
    # alignment; message lengths cover every alignment of the last block.
    n = 2 * 521
    rng = np.random.default_rng(44)
    b = W.ragged_batch(n, seed=44, lens=rng.integers(0, 400, size=n), gap=3)
    b.variants = np.array([4 + (i & 1) for i in range(n)], dtype=np.uint8)
    b.out_lens = np.array([i // 2 for i in range(n)], dtype=np.uint32)
    perm = rng.permutation(n)
    b = W.RaggedBatch(b.msgs, b.offsets[perm], b.lens[perm], b.variants[perm], b.out_lens[perm])
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))
    assert cuda_lib.keccak_last_error() == 0


def test_ragged_same_digest_alone_and_in_the_mix(cuda_lib):
    torch = _torch()
    b = W.ragged_batch(500, seed=31, max_len=4000, gap=3)
    mixed = _run_ragged(cuda_lib, b)
    oo = b.out_offsets()
    d_msgs = dev(b.msgs)
    for i in np.random.default_rng(0).choice(b.n, size=25, replace=False):
        out = torch.zeros(max(int(b.out_lens[i]), 1), dtype=torch.uint8, device="cuda")
        cuda_lib.keccak_batch(d_msgs, dev(b.offsets[i:i + 1]), dev(b.lens[i:i + 1]), dev(b.variants[i:i + 1]),
                              dev(b.out_lens[i:i + 1]), out, 1)
        alone = host(out)[: int(b.out_lens[i])]
        assert np.array_equal(alone, mixed[int(oo[i]):int(oo[i]) + int(b.out_lens[i])]), i


def test_ragged_bad_messages_are_flagged_and_skipped(cuda_lib, oracle_mod):
    b = W.ragged_batch(64, seed=41, max_len=500, variants=(1, 3))
    b.variants[5] = 9          # no such variant
    b.out_lens[7] = 31 if b.variants[7] == 1 else 63  # wrong SHA3 digest size
    assert cuda_lib.keccak_last_error() == 0
    got = _run_ragged(cuda_lib, b, sentinel=0xEE)
    status = cuda_lib.keccak_last_error()
    assert status & 0x1 and status & 0x2
    assert cuda_lib.keccak_last_error() == 0  # cleared by the read
    oo = b.out_offsets()
    for i in range(b.n):
        seg = got[int(oo[i]):int(oo[i]) + int(b.out_lens[i])]
        if i in (5, 7):
            assert (seg == 0xEE).all()
        else:
            want = oracle_mod.hash(int(b.variants[i]), b.msgs[int(b.offsets[i]):int(b.offsets[i] + b.lens[i])],
                                   int(b.out_lens[i]))
            assert seg.tobytes() == want


# -- Merkle trees ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_leaves,leaf_bytes", [(1, 8), (2, 64), (3, 135), (5, 136), (7, 1001), (8, 8192),
                                                 (9, 7), (33, 200), (100, 64), (1000, 32), (64, 8192),
                                                 (65, 16), (129, 8), (4097, 16), (10001, 8), (32769, 8),
                                                 (40001, 8), (98305, 8)])
def test_merkle_levels_and_root(cuda_lib, oracle_mod, n_leaves, leaf_bytes):
    torch = _torch()
    buf = W.merkle_buffer(n_leaves, leaf_bytes, seed=n_leaves * 1000 + leaf_bytes)
    want = oracle_mod.merkle_levels(buf, n_leaves, leaf_bytes)
    d_buf = dev(buf)
    total = cuda_lib.merkle_node_count(n_leaves)
    nodes = torch.zeros(32 * total, dtype=torch.uint8, device="cuda")
    cuda_lib.merkle_sha3_256_levels(d_buf, n_leaves, leaf_bytes, nodes)
    assert np.array_equal(host(nodes).reshape(total, 32), want)
    assert cuda_lib.merkle_sha3_256(d_buf, n_leaves, leaf_bytes) == want[-1].tobytes()


def test_merkle_unaligned_buffer(cuda_lib, oracle_mod):
    torch = _torch()
    n, lb = 17, 96
    buf = W.merkle_buffer(n, lb, seed=77)
    raw = torch.zeros(buf.size + 8, dtype=torch.uint8, device="cuda")
    raw[3:3 + buf.size] = dev(buf)
    assert cuda_lib.merkle_sha3_256(raw.data_ptr() + 3, n, lb) == oracle_mod.merkle_root(buf, n, lb)


# -- host-buffer pipeline ---------------------------------------------------------------------
@pytest.mark.parametrize("pinned,path", [(True, 0), (True, 1), (True, 2), (False, 0), (False, 1)])
def test_host_pipeline_matches_oracle(cuda_lib, oracle_mod, pinned, path):
    torch = _torch()
    saved = cuda_lib.keccak_tune_get(cuda_lib.KB_TUNE_HOST_PATH)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_HOST_PATH, path)
    n, L = 700_000, 64  # 44.8 MB of input: more than one 32 MiB chunk
    msgs = W.uniform_messages(n, L, seed=51)
    if pinned:
        h_in = torch.from_numpy(msgs).pin_memory()
        h_out = torch.zeros(n * 32, dtype=torch.uint8).pin_memory()
    else:
        h_in, h_out = msgs, np.zeros(n * 32, dtype=np.uint8)
    try:
        cuda_lib.keccak_batch_uniform_host(h_in, L, L, 1, 32, h_out, n)
    finally:
        cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_HOST_PATH, saved)
    got = (h_out.numpy() if pinned else h_out).reshape(n, 32)
    chunk = (32 << 20) // L
    idx = np.unique(np.concatenate([np.arange(5), np.arange(chunk - 3, chunk + 3), np.arange(n - 5, n),
                                    np.random.default_rng(1).choice(n, 2000, replace=False)]))
    want = oracle_uniform(oracle_mod, msgs, L, L, 1, 32, n, idx)
    assert np.array_equal(got[idx], want)


def test_host_path_trial_and_numa_buffers(cuda_lib, oracle_mod):
    # KB_HOST_PATH_AUTO on page-locked buffers from keccak_host_alloc: the first
    # call of a size class hashes a warm-up by each path, then two eighths of
    # the batch by each, alternating, then the rest by the faster; every
    # message must come out exactly once, across every boundary between the
    # parts, and later calls use the decision.
    cuda_lib.keccak_release()  # no earlier decision for this size class
    n, L = 700_000, 64
    assert cuda_lib.keccak_host_path_for(n) == cuda_lib.KB_HOST_PATH_AUTO
    msgs = W.uniform_messages(n, L, seed=52)
    h_in, h_out = cuda_lib.HostBuffer(n * L), cuda_lib.HostBuffer(n * 32)
    assert h_in.numa_node() >= -1 and h_out.numa_node() >= -1
    h_in.array[:] = msgs
    warm, eighth = n // 64, n // 8
    edges = [0, warm, 2 * warm] + [2 * warm + k * eighth for k in range(1, 5)] + [n]
    idx = np.unique(np.concatenate([np.arange(max(0, e - 3), min(n, e + 3)) for e in edges]
                                   + [np.random.default_rng(3).choice(n, 3000, replace=False)]))
    want = oracle_uniform(oracle_mod, msgs, L, L, 1, 32, n, idx)
    for call in range(2):
        h_out.array[:] = 0xEE
        cuda_lib.keccak_batch_uniform_host(h_in, L, L, 1, 32, h_out, n)
        assert np.array_equal(h_out.array.reshape(n, 32)[idx], want), call
        assert cuda_lib.keccak_host_path_for(n) in (cuda_lib.KB_HOST_PATH_STAGED, cuda_lib.KB_HOST_PATH_ZERO_COPY)
    h_in.free()
    h_out.free()
    cuda_lib.keccak_release()
    assert cuda_lib.keccak_host_path_for(n) == cuda_lib.KB_HOST_PATH_AUTO


def test_host_alloc_arguments(cuda_lib):
    import ctypes

    lib = cuda_lib.load()
    p = ctypes.c_void_p()
    assert lib.keccak_host_alloc(0, ctypes.addressof(p)) == cuda_lib.KB_ERR_INVALID
    assert lib.keccak_host_alloc(16, None) == cuda_lib.KB_ERR_INVALID
    assert lib.keccak_host_free(None) == cuda_lib.KB_OK
    local = np.zeros(64, np.uint8)
    assert lib.keccak_host_free(local.ctypes.data) == cuda_lib.KB_ERR_INVALID


# -- full benchmark sizes, sampled ---------------------------------------------------------------
def test_full_size_fixed_batches_sampled(cuda_lib, oracle_mod):
    torch = _torch()
    n, L = 1 << 24, 64
    msgs = W.uniform_messages(n, L, seed=1)
    d_msgs = dev(msgs)
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([np.arange(64), np.arange(n - 64, n), rng.choice(n, 4096, replace=False)]))
    for variant, dl in ((1, 32), (3, 64)):
        out = torch.zeros(n * dl, dtype=torch.uint8, device="cuda")
        cuda_lib.keccak_batch_uniform(d_msgs, L, L, variant, dl, out, n)
        got = host(out).reshape(n, dl)
        assert np.array_equal(got[idx], oracle_uniform(oracle_mod, msgs, L, L, variant, dl, n, idx)), variant
        del out
    del d_msgs
    n2, L2 = 1 << 22, 1024
    msgs2 = W.uniform_messages(n2, L2, seed=2)
    d2 = dev(msgs2)
    out2 = torch.zeros(n2 * 32, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch_uniform(d2, L2, L2, 1, 32, out2, n2)
    got2 = host(out2).reshape(n2, 32)
    idx2 = np.unique(np.concatenate([np.arange(16), np.arange(n2 - 16, n2), rng.choice(n2, 1024, replace=False)]))
    assert np.array_equal(got2[idx2], oracle_uniform(oracle_mod, msgs2, L2, L2, 1, 32, n2, idx2))


def test_full_size_ragged_batch_sampled(cuda_lib, oracle_mod):
    b = W.ragged_batch(1 << 20, seed=3, max_len=65536)
    got = _run_ragged(cuda_lib, b)
    oo = b.out_offsets()
    rng = np.random.default_rng(4)
    longest = np.argsort(b.lens)[-8:]
    idx = np.unique(np.concatenate([np.arange(32), np.arange(b.n - 32, b.n), longest,
                                    rng.choice(b.n, 400, replace=False)]))
    sub = W.RaggedBatch(b.msgs, b.offsets[idx], b.lens[idx], b.variants[idx], b.out_lens[idx])
    want = _oracle_ragged(oracle_mod, sub)
    pos = 0
    for i in idx:
        ln = int(b.out_lens[i])
        assert np.array_equal(got[int(oo[i]):int(oo[i]) + ln], want[pos:pos + ln]), i
        pos += ln
    assert cuda_lib.keccak_last_error() == 0


def test_full_size_ragged_batch_every_digest_against_hashlib(cuda_lib):
    # Beyond the oracle's sample: all 2^20 digests of the full-size mixed batch
    # against Python's hashlib (OpenSSL), hashed on host threads.
    import hashlib
    from concurrent.futures import ThreadPoolExecutor

    b = W.ragged_batch(1 << 20, seed=3, max_len=65536)
    got = _run_ragged(cuda_lib, b)
    fns = (hashlib.sha3_224, hashlib.sha3_256, hashlib.sha3_384, hashlib.sha3_512)

    def part(lo, hi):
        out = []
        for i in range(lo, hi):
            o, ln, v, d = int(b.offsets[i]), int(b.lens[i]), int(b.variants[i]), int(b.out_lens[i])
            m = b.msgs[o:o + ln]
            if v < 4:
                out.append(fns[v](m).digest())
            else:
                out.append((hashlib.shake_128 if v == 4 else hashlib.shake_256)(m).digest(d))
        return b"".join(out)

    step = 8192
    with ThreadPoolExecutor(THREADS) as ex:
        parts = list(ex.map(lambda lo: part(lo, min(b.n, lo + step)), range(0, b.n, step)))
    want = b"".join(parts)
    assert got.tobytes() == want
    # The configuration the autotuner picks for this batch, as the bench runs it.
    torch = _torch()
    d = [dev(x) for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.full((b.total_out(),), 0xEE, dtype=torch.uint8, device="cuda")
    cuda_lib.keccak_batch_autotune(*d, out, b.n)
    out.fill_(0xEE)
    cuda_lib.keccak_batch(*d, out, b.n)
    assert host(out).tobytes() == want
    torch.cuda.synchronize()
    cuda_lib.keccak_release()  # drops the tuned configuration with the cached scratch


def test_full_size_merkle_root(cuda_lib, oracle_mod):
    torch = _torch()
    n, lb = 524288, 8192
    buf = W.merkle_buffer(n, lb, seed=4)
    d_buf = dev(buf)
    total = cuda_lib.merkle_node_count(n)
    nodes = torch.zeros(32 * total, dtype=torch.uint8, device="cuda")
    cuda_lib.merkle_sha3_256_levels(d_buf, n, lb, nodes)
    got = host(nodes).reshape(total, 32)
    root = cuda_lib.merkle_sha3_256(d_buf, n, lb)
    assert root == got[-1].tobytes()
    # Sampled leaves against the oracle.
    for i in np.random.default_rng(5).choice(n, 16, replace=False):
        assert got[i].tobytes() == oracle_mod.hash(1, b"\x00" + buf[i * lb:(i + 1) * lb].tobytes())
    # Every level from its children, and the leaves, with hashlib (independent of both).
    leaves = [hashlib.sha3_256(b"\x00" + buf[i * lb:(i + 1) * lb].tobytes()).digest() for i in range(n)]
    assert all(got[i].tobytes() == leaves[i] for i in range(n))
    level, pos = leaves, n
    while len(level) > 1:
        nxt = [hashlib.sha3_256(b"\x01" + level[2 * j] + level[2 * j + 1]).digest() for j in range(len(level) // 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        assert all(got[pos + j].tobytes() == nxt[j] for j in range(len(nxt)))
        pos += len(nxt)
        level = nxt
    assert root == level[0]


def test_interleaved_control_matches_oracle(cuda_lib, oracle_mod):
    # The bit-interleaved state layout (tuning knob) gives the same digests.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_REPRESENTATION, cuda_lib.KB_REP_INTERLEAVED)
    try:
        for n, L in ((1000, 64), (300, 1000)):
            msgs = W.uniform_messages(n, L, seed=60 + L)
            got = gpu_uniform(cuda_lib, msgs, L, L, 1, 32, n)
            assert np.array_equal(got, oracle_uniform(oracle_mod, msgs, L, L, 1, 32, n)), L
    finally:
        cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_REPRESENTATION, cuda_lib.KB_REP_PLAIN)


# -- ragged schedules, graph replay, autotuner -------------------------------------------
@pytest.fixture
def restore_tuning(cuda_lib):
    keys = range(cuda_lib.KB_TUNE_KEYS)
    saved = [cuda_lib.keccak_tune_get(k) for k in keys]
    yield
    for k, v in zip(keys, saved):
        cuda_lib.keccak_tune_set(k, v)


@pytest.mark.parametrize("schedule", [0, 1, 2, 3])
@pytest.mark.parametrize("graphs", [0, 1])
def test_ragged_schedules_match_oracle(cuda_lib, oracle_mod, restore_tuning, schedule, graphs):
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_RAGGED_SCHEDULE, schedule)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_GRAPHS, graphs)
    b = W.ragged_batch(5000, seed=70 + schedule, max_len=5000, gap=4)
    want = _oracle_ragged(oracle_mod, b)
    assert np.array_equal(_run_ragged(cuda_lib, b), want)
    assert cuda_lib.keccak_last_error() == 0


QUEUE_KERNELS = ([(m, 1) for m in (2, 3, 4, 5, 6, 8)] + [(m, s) for s in (2, 3) for m in (2, 3, 4)]
                 + [(m, 4) for m in (2, 3)])


@pytest.mark.parametrize("min_blocks,staging", QUEUE_KERNELS)
def test_queue_register_budgets_match_oracle(cuda_lib, oracle_mod, restore_tuning, min_blocks, staging):
    # Every compiled queue kernel: register budget x how it reads message blocks.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_MIN_BLOCKS, min_blocks)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_BLOCKS_PER_SM, 2)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_STAGING, staging)
    assert cuda_lib.keccak_tuned_config(1500)["staging"] == cuda_lib.QUEUE_STAGING_NAMES[staging]
    b = W.ragged_batch(1500, seed=80 + min_blocks + 10 * staging, max_len=2000, gap=2)
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))
    assert cuda_lib.keccak_last_error() == 0


@pytest.mark.parametrize("staging", [1, 2, 3, 4])
def test_queue_staging_every_padding_case(cuda_lib, oracle_mod, restore_tuning, staging):
    # Every way the queue kernel reads blocks (direct, direct with the looped
    # permutation, cp.async into shared memory, registers loaded before the
    # permutation): every len mod r edge of every variant, multi-block
    # messages, starts at every byte alignment, SHAKE outputs across squeeze
    # blocks, in one batch so that warps mix rates at bucket boundaries.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_STAGING, staging)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_MIN_BLOCKS, 2)
    rng = np.random.default_rng(700 + staging)
    lens, var, ol = [], [], []
    for v in range(6):
        r = RATES[v]
        for L in (0, 1, 3, 4, 5, 7, 8, r - 9, r - 8, r - 2, r - 1, r, r + 1, r + 3, 2 * r - 1, 2 * r, 2 * r + 5,
                  5 * r + 7, 9 * r):
            for _ in range(3):
                lens.append(L)
                var.append(v)
                ol.append(DIG[v] if v < 4 else int(rng.choice((0, 1, r - 1, r, r + 1, 3 * r + 2, 512))))
    order = rng.permutation(len(lens))
    b = W.ragged_batch(len(lens), seed=710 + staging, gap=7, lens=np.asarray(lens, np.uint64)[order])
    b.variants = np.asarray(var, np.uint8)[order]
    b.out_lens = np.asarray(ol, np.uint32)[order]
    assert len(set(int(o) % 4 for o in b.offsets)) == 4
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))
    assert cuda_lib.keccak_last_error() == 0


@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("k", ["0", "1", "32", "all"])
def test_hybrid_threads_per_message_matches_oracle(cuda_lib, oracle_mod, restore_tuning, k, graphs):
    # Threads per message: the K costliest messages one warp each (on a side
    # stream, concurrently with the queue), the rest one thread each.  K = all
    # puts every message on the warp kernel and leaves the queue empty.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_GRAPHS, graphs)
    b = W.ragged_batch(3000, seed=720 + graphs, max_len=20000, gap=3)
    kk = b.n if k == "all" else int(k)
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_QUEUE_WARP_MESSAGES, kk)
    assert cuda_lib.keccak_tuned_config(b.n)["warp_messages"] == kk
    torch = _torch()
    s = torch.cuda.Stream()
    d = [dev(x) for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.full((b.total_out(),), 0xEE, dtype=torch.uint8, device="cuda")
    want = _oracle_ragged(oracle_mod, b)
    for _ in range(2):  # the second call replays the captured graph
        out.fill_(0xEE)
        torch.cuda.synchronize()
        cuda_lib.keccak_batch(*d, out, b.n, s)
        s.synchronize()
        assert np.array_equal(host(out), want)
    assert cuda_lib.keccak_last_error(s) == 0


def test_graph_replay_reads_current_bytes(cuda_lib, oracle_mod, restore_tuning):
    # A replayed graph holds pointers, not contents: new bytes in the same
    # buffers give the new digests, on a non-default stream.
    torch = _torch()
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_GRAPHS, 1)
    b = W.ragged_batch(2000, seed=90, max_len=3000, gap=1)
    s = torch.cuda.Stream()
    d = [dev(x) for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.zeros(b.total_out(), dtype=torch.uint8, device="cuda")
    for trial in range(3):
        fresh = W.random_bytes(b.msgs.size, seed=1000 + trial)
        d[0].copy_(torch.from_numpy(fresh))
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            cuda_lib.keccak_batch(*d, out, b.n, s)
        s.synchronize()
        want = oracle_mod.hash_batch(fresh, b.offsets, b.lens, b.variants, b.out_lens, THREADS)
        assert np.array_equal(out.cpu().numpy(), want), trial


def test_autotune_keeps_digests(cuda_lib, oracle_mod, restore_tuning):
    torch = _torch()
    b = W.ragged_batch(3000, seed=95, max_len=8000, gap=3)
    d = [dev(x) for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.zeros(b.total_out(), dtype=torch.uint8, device="cuda")
    chosen = cuda_lib.keccak_batch_autotune(*d, out, b.n)
    assert chosen["min_blocks"] in (2, 3, 4, 5, 6, 8) and chosen["blocks_per_sm"] >= 1 and chosen["ms"] > 0
    assert chosen["staging"] in ("direct", "direct_looped", "async", "regs") and chosen["warp_messages"] in (0, 32, 608)
    tuned = cuda_lib.keccak_tuned_config(b.n)
    assert all(tuned[key] == chosen[key] for key in tuned)
    want = _oracle_ragged(oracle_mod, b)
    assert np.array_equal(host(out)[: b.total_out()], want)
    out.zero_()
    cuda_lib.keccak_batch(*d, out, b.n)  # now runs with the tuned configuration
    assert np.array_equal(host(out)[: b.total_out()], want)


def test_lane_parallel_long_messages_every_variant(cuda_lib, oracle_mod, restore_tuning):
    # One warp per message: multi-block messages, every padding position of the
    # final block, SHAKE outputs across squeeze blocks, aligned and unaligned.
    cuda_lib.keccak_tune_set(cuda_lib.KB_TUNE_RAGGED_SCHEDULE, cuda_lib.KB_SCHEDULE_LANE_PARALLEL)
    lens, variants = [], []
    for v in range(6):
        r = RATES[v]
        for L in (0, 1, r - 1, r, r + 1, 5 * r + 3, 20_000):
            lens.append(L)
            variants.append(v)
    rng = np.random.default_rng(77)
    b = W.ragged_batch(len(lens), seed=78, lens=np.array(lens), gap=5)
    b.variants = np.array(variants, dtype=np.uint8)
    b.out_lens = np.array([DIG[v] or int(rng.choice([0, 1, 167, 168, 169, 500])) for v in b.variants],
                          dtype=np.uint32)
    assert np.array_equal(_run_ragged(cuda_lib, b), _oracle_ragged(oracle_mod, b))


@pytest.mark.parametrize("length,chunk,shift", [(0, 64, 0), (1, 64, 0), (64, 64, 0), (65, 64, 3), (1000, 136, 1),
                                                (4097, 128, 0), (3000, 999, 5), (10_000_000, 8192, 0),
                                                (10_000_001, 8192, 7)])
def test_merkle_message_tree(cuda_lib, oracle_mod, length, chunk, shift):
    torch = _torch()
    msg = W.random_bytes(length, seed=length % 1000 + chunk)
    raw = torch.zeros(length + shift + 8, dtype=torch.uint8, device="cuda")
    if length:
        raw[shift:shift + length] = dev(msg)
    got = cuda_lib.merkle_sha3_256_message(raw.data_ptr() + shift, length, chunk)
    assert got == oracle_mod.merkle_message_root(msg, chunk)


@pytest.mark.parametrize("n_trees,leaves,leaf_bytes,shift", [(1, 1, 1, 0), (300, 1, 64, 0), (300, 3, 135, 1),
                                                             (200, 7, 8, 0), (129, 13, 200, 3), (64, 33, 40, 0),
                                                             (16, 100, 17, 5), (32, 16, 256, 0),
                                                             (50, 5, 1000, 0), (40, 2, 136, 0)])
def test_merkle_many_small_trees(cuda_lib, oracle_mod, n_trees, leaves, leaf_bytes, shift):
    torch = _torch()
    buf = W.merkle_buffer(n_trees * leaves, leaf_bytes, seed=n_trees + leaves + leaf_bytes)
    raw = torch.zeros(buf.size + shift + 8, dtype=torch.uint8, device="cuda")
    raw[shift:shift + buf.size] = dev(buf)
    roots = torch.zeros(32 * n_trees, dtype=torch.uint8, device="cuda")
    cuda_lib.merkle_sha3_256_many(raw.data_ptr() + shift, n_trees, leaves, leaf_bytes, roots)
    got = host(roots).reshape(n_trees, 32)
    tree = leaves * leaf_bytes
    for t in range(n_trees):
        assert got[t].tobytes() == oracle_mod.merkle_root(buf[t * tree:(t + 1) * tree], leaves, leaf_bytes), t


# -- the permutation alone, every width (Keccak-p[b, n_r]) --------------------------------
def _lanes_to_bits(lanes: np.ndarray, w: int) -> np.ndarray:
    # Eq. 1: string bit w(5y+x)+z is bit z of lane x+5y.
    return np.array([(int(lanes[i]) >> z) & 1 for i in range(25) for z in range(w)], dtype=np.uint8)


@pytest.mark.parametrize("b,nr", [(200, 18), (1600, 24), (1600, 12)])
def test_keccak_p_several_tiles(cuda_lib, oracle_mod, b, nr):
    # 3 full tiles of 128 states and a partial one; the states after the n
    # given ones stay untouched.
    torch = _torch()
    w = b // 25
    n, extra = 128 * 3 + 77, 5
    rng = np.random.default_rng(b + nr)
    states = rng.integers(0, 2**64, size=(n + extra, 25), dtype=np.uint64) & np.uint64((1 << w) - 1)
    d = torch.from_numpy(states.view(np.int64).copy()).cuda()
    cuda_lib.keccak_p_batch(d, b, nr, n)
    got = d.cpu().numpy().view(np.uint64).reshape(n + extra, 25)
    assert np.array_equal(got[n:], states[n:])
    for i in list(range(0, n, 37)) + [127, 128, 383, 384, n - 1]:
        want = oracle_mod.keccak_p(b, nr, _lanes_to_bits(states[i], w))
        assert np.array_equal(_lanes_to_bits(got[i], w), want), (b, nr, i)


@pytest.mark.parametrize("b,nr", [(200, 18), (1600, 12), (25, 7), (800, 22)])
def test_keccak_p_many_tiles_per_block(cuda_lib, oracle_mod, b, nr):
    # Enough states that every block of the persistent grid runs several
    # tiles (its next tile's copies in flight while it permutes the current
    # one), with a partial last tile; sampled states against the oracle, the
    # states after the n given ones untouched.
    torch = _torch()
    w = b // 25
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, extra = 128 * 8 * sms * 3 + 77, 3
    rng = np.random.default_rng(b * 7 + nr)
    states = rng.integers(0, 2**64, size=(n + extra, 25), dtype=np.uint64) & np.uint64((1 << w) - 1)
    d = torch.from_numpy(states.view(np.int64).copy()).cuda()
    cuda_lib.keccak_p_batch(d, b, nr, n)
    got = d.cpu().numpy().view(np.uint64).reshape(n + extra, 25)
    assert np.array_equal(got[n:], states[n:])
    sample = list(rng.choice(n, 150, replace=False)) + [0, 127, 128, n - 78, n - 77, n - 1]
    for i in sample:
        want = oracle_mod.keccak_p(b, nr, _lanes_to_bits(states[i], w))
        assert np.array_equal(_lanes_to_bits(got[i], w), want), (b, nr, i)


@pytest.mark.parametrize("b", [25, 50, 100, 200, 400, 800, 1600])
def test_keccak_p_every_width_and_round_count(cuda_lib, oracle_mod, b):
    torch = _torch()
    w = b // 25
    l = int(np.log2(w))
    rng = np.random.default_rng(b)
    n = 64
    for nr in sorted({1, 3, 12 + 2 * l, 12 + 2 * l + 5}):
        mask = (1 << w) - 1
        states = rng.integers(0, 2**63, size=(n, 25), dtype=np.uint64) & np.uint64(mask)
        d = torch.from_numpy(states.view(np.int64).copy()).cuda()
        cuda_lib.keccak_p_batch(d, b, nr, n)
        got = d.cpu().numpy().view(np.uint64)
        for i in range(n):
            want = oracle_mod.keccak_p(b, nr, _lanes_to_bits(states[i], w))
            assert np.array_equal(_lanes_to_bits(got[i], w), want), (b, nr, i)


# -- the binding's byte-string convenience call --------------------------------------------
def test_hash_many_byte_strings(cuda_lib, oracle_mod):
    rng = np.random.default_rng(123)
    lens = [0, 1, 71, 72, 135, 136, 137, 168, 1000, 5000] + list(rng.integers(0, 3000, size=90))
    messages = [rng.integers(0, 256, size=int(k), dtype=np.uint8).tobytes() for k in lens]
    variants = [int(v) for v in rng.integers(0, 6, size=len(messages))]
    out_lens = [W.DIGEST_BYTES[v] if W.DIGEST_BYTES[v] is not None else int(rng.integers(0, 400))
                for v in variants]
    got = cuda_lib.hash_many(messages, variants, out_lens)
    assert got == [oracle_mod.hash(v, m, o) for m, v, o in zip(messages, variants, out_lens)]
    # One SHA3 function for all, default output sizes.
    assert cuda_lib.hash_many(messages[:10]) == [oracle_mod.hash(1, m, 32) for m in messages[:10]]
    assert cuda_lib.hash_many([]) == []
