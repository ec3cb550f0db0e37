"""Seeded synthetic inputs shared by the tests and the benchmark.

Only input generation lives here: random bytes, lengths, variants and output
sizes drawn from numpy's PCG64 (``default_rng(seed)``).  No hashing
arithmetic.  The shapes follow the paper's many-small-messages workload
(Section 4.3: a large number of same-length messages) and its
generalisations:

* uniform batches: n messages of one length, bytes uniform on 0..255;
* ragged batches: lengths log-uniform over 0..max_len, drawn as
  floor(exp(U[0, ln(max_len + 1)))) - 1, a variant uniform over the six
  functions and, for SHAKE, an output length uniform over 16..512 bytes;
* Merkle buffers: uniform random bytes split into fixed-size leaves.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DIGEST_BYTES = (28, 32, 48, 64, None, None)


def random_bytes(nbytes: int, seed: int) -> np.ndarray:
    """nbytes uniform random bytes (uint8 array) from seed."""
    rng = np.random.default_rng(seed)
    out = np.empty(nbytes, dtype=np.uint8)
    chunk = 1 << 28
    for s in range(0, nbytes, chunk):
        e = min(nbytes, s + chunk)
        out[s:e] = np.frombuffer(rng.bytes(e - s), dtype=np.uint8)
    return out


def uniform_messages(n: int, length: int, seed: int) -> np.ndarray:
    """n back-to-back messages of `length` bytes (stride = length)."""
    return random_bytes(n * length, seed)


@dataclass
class RaggedBatch:
    msgs: np.ndarray       # uint8, all messages (with gaps)
    offsets: np.ndarray    # uint64[n]
    lens: np.ndarray       # uint64[n]
    variants: np.ndarray   # uint8[n]
    out_lens: np.ndarray   # uint32[n]

    @property
    def n(self) -> int:
        return int(self.offsets.size)

    def out_offsets(self) -> np.ndarray:
        o = np.zeros(self.n, dtype=np.uint64)
        if self.n > 1:
            np.cumsum(self.out_lens[:-1], dtype=np.uint64, out=o[1:])
        return o

    def total_out(self) -> int:
        return int(self.out_lens.sum(dtype=np.uint64))


def log_uniform_lengths(rng: np.random.Generator, n: int, max_len: int, min_len: int = 0) -> np.ndarray:
    """Lengths in [min_len, max_len], log-uniform (0 allowed when min_len = 0)."""
    lo, hi = np.log(min_len + 1), np.log(max_len + 1)
    lens = np.floor(np.exp(rng.uniform(lo, hi, size=n))).astype(np.int64) - 1
    return np.clip(lens, min_len, max_len).astype(np.uint64)


def ragged_batch(n: int, seed: int, max_len: int = 65536, min_len: int = 0,
                 variants=(0, 1, 2, 3, 4, 5), shake_out=(16, 512), gap: int = 0,
                 lens: np.ndarray | None = None) -> RaggedBatch:
    """A ragged, mixed-variant batch.  gap > 0 leaves 0..gap random bytes between
    messages, so message starts fall on every alignment."""
    rng = np.random.default_rng(seed)
    if lens is None:
        lens = log_uniform_lengths(rng, n, max_len, min_len)
    lens = np.asarray(lens, dtype=np.uint64)
    var = rng.choice(np.asarray(variants, dtype=np.uint8), size=n).astype(np.uint8)
    out_lens = np.empty(n, dtype=np.uint32)
    for v in range(6):
        sel = var == v
        if DIGEST_BYTES[v] is not None:
            out_lens[sel] = DIGEST_BYTES[v]
        else:
            out_lens[sel] = rng.integers(shake_out[0], shake_out[1] + 1, size=int(sel.sum()))
    gaps = rng.integers(0, gap + 1, size=n).astype(np.uint64) if gap else np.zeros(n, dtype=np.uint64)
    offsets = np.zeros(n, dtype=np.uint64)
    if n:
        ends = np.cumsum(lens + gaps, dtype=np.uint64)
        offsets = ends - lens
        total = int(ends[-1])
    else:
        total = 0
    msgs = random_bytes(max(total, 1), seed + 1_000_003)
    return RaggedBatch(msgs, offsets, lens, var, out_lens)


def merkle_buffer(n_leaves: int, leaf_bytes: int, seed: int) -> np.ndarray:
    return random_bytes(n_leaves * leaf_bytes, seed)


@dataclass
class ServingWorkload:
    pool: np.ndarray        # uint8 message pool
    offsets: np.ndarray     # uint64[n]: request i's message starts at pool[offsets[i]]
    lens: np.ndarray        # uint64[n]
    variants: np.ndarray    # uint8[n]
    out_lens: np.ndarray    # uint32[n]
    arrival_ns: np.ndarray  # int64[n], non-decreasing

    @property
    def n(self) -> int:
        return int(self.offsets.size)


def serving_workload(rate_per_s: float, seconds: float, seed: int, min_len: int = 32, max_len: int = 1 << 20,
                     pool_bytes: int = 1 << 30, variants=(0, 1, 2, 3, 4, 5), shake_out=(16, 512)) -> ServingWorkload:
    """Poisson arrivals at rate_per_s for `seconds`; each request one message of
    log-uniform length in [min_len, max_len] taken at a seeded offset of a
    random pool, a uniform variant and (SHAKE) a uniform output length."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate_per_s * seconds))
    gaps = rng.exponential(1e9 / rate_per_s, size=n)
    arrival = np.floor(np.cumsum(gaps)).astype(np.int64)
    lo, hi = np.log(min_len), np.log(max_len + 1)
    lens = np.clip(np.floor(np.exp(rng.uniform(lo, hi, size=n))), min_len, max_len).astype(np.uint64)
    offsets = (rng.integers(0, 2**63, size=n, dtype=np.uint64) % (np.uint64(pool_bytes) - lens + np.uint64(1)))
    var = rng.choice(np.asarray(variants, dtype=np.uint8), size=n).astype(np.uint8)
    out_lens = np.empty(n, dtype=np.uint32)
    for v in range(6):
        sel = var == v
        if DIGEST_BYTES[v] is not None:
            out_lens[sel] = DIGEST_BYTES[v]
        else:
            out_lens[sel] = rng.integers(shake_out[0], shake_out[1] + 1, size=int(sel.sum()))
    pool = random_bytes(pool_bytes, seed + 7_000_003)
    return ServingWorkload(pool, offsets.astype(np.uint64), lens, var, out_lens, arrival)
