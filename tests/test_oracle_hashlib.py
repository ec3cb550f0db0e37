"""Pins the oracle's six functions against an independent implementation.

Python's hashlib (OpenSSL) computes SHA3-224/256/384/512 and SHAKE128/256 of
FIPS 202, the standard the paper restates in Eq. 12-18.  It is not used by the
oracle; any dropped term, wrong rotation, index, constant, padding or bit order
in the oracle changes these digests.
"""
import hashlib

import numpy as np
import pytest

RATES = (144, 136, 104, 72, 168, 136)  # bytes, r = 1600 - c (Eq. 12-18)
NAMES = ("sha3_224", "sha3_256", "sha3_384", "sha3_512", "shake_128", "shake_256")


def _ref(variant, msg, out_len=None):
    h = getattr(hashlib, NAMES[variant])(msg)
    return h.digest(out_len) if variant >= 4 else h.digest()


def _lengths(r, rng):
    # Every padding case of Eq. 11: len mod r in {0, 1, r-2, r-1}, the empty
    # message, a few multi-block lengths, and random lengths up to 3r+1.
    fixed = {0, 1, r - 2, r - 1, r, r + 1, 2 * r - 1, 2 * r, 2 * r + 1, 3 * r, 3 * r + 1}
    return sorted(fixed | set(int(x) for x in rng.integers(0, 3 * r + 2, size=24)))


@pytest.mark.parametrize("variant", range(6))
def test_oracle_matches_hashlib(oracle_mod, variant):
    rng = np.random.default_rng(1000 + variant)
    r = RATES[variant]
    for L in _lengths(r, rng):
        msg = rng.integers(0, 256, size=L, dtype=np.uint8).tobytes()
        if variant < 4:
            assert oracle_mod.hash(variant, msg) == _ref(variant, msg), (variant, L)
        else:
            d = int(rng.integers(16, 513))
            assert oracle_mod.hash(variant, msg, d) == _ref(variant, msg, d), (variant, L, d)


@pytest.mark.parametrize("variant", (4, 5))
def test_oracle_shake_output_lengths(oracle_mod, variant):
    # Squeeze across output-block boundaries (FIPS 202 Algorithm 8: f is
    # applied between output blocks): d in {0, 1, r-1, r, r+1, 3r+5, 512}.
    r = RATES[variant]
    msg = bytes(range(100))
    for d in (0, 1, r - 1, r, r + 1, 3 * r + 5, 512):
        assert oracle_mod.hash(variant, msg, d) == _ref(variant, msg, d), d


def test_oracle_shared_padding_byte(oracle_mod):
    # len mod r = r-1: suffix and final padding bit land in one byte.
    for variant in range(6):
        r = RATES[variant]
        msg = bytes((7 * i) & 0xFF for i in range(r - 1))
        d = None if variant < 4 else 64
        assert oracle_mod.hash(variant, msg, d) == _ref(variant, msg, d)


def test_oracle_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.hash(6, b"abc", 32)
    with pytest.raises(ValueError):
        oracle_mod.hash(1, b"abc", 31)  # SHA3-256 output must be 32 bytes


def _mixed_batch():
    """A CSR batch that exercises every layout case of the batch harness: all
    six functions, the empty message, every len mod r edge, multi-block
    messages, SHAKE outputs of 0 bytes and of more than one rate block, and
    random gaps so that message starts fall on every alignment."""
    from paper_1902_05320_gb300 import workloads

    rng = np.random.default_rng(77)
    lens, variants, out_lens = [], [], []
    for v in range(6):
        r = RATES[v]
        for L in (0, 1, r - 2, r - 1, r, r + 1, 2 * r - 1, 2 * r, 3 * r + 7):
            lens.append(L)
            variants.append(v)
            if v < 4:
                out_lens.append((28, 32, 48, 64)[v])
            else:
                out_lens.append(int(rng.choice((0, 1, r - 1, r, r + 1, 2 * r + 3, 512))))
    order = rng.permutation(len(lens))
    lens = np.asarray(lens, np.uint64)[order]
    b = workloads.ragged_batch(len(lens), seed=78, gap=13, lens=lens)
    b.variants = np.asarray(variants, np.uint8)[order]
    b.out_lens = np.asarray(out_lens, np.uint32)[order]
    return b


@pytest.mark.parametrize("nthreads", (1, 3, None))
def test_oracle_hash_batch_layout(oracle_mod, nthreads):
    # The batch harness of Section 4's batch mode: message i's output must sit
    # at the exclusive scan of the output sizes, whatever the thread split.
    # Checked byte for byte against per-message oracle.hash and against
    # hashlib, so a slip in the scan, the offsets or the thread hand-out fails.
    b = _mixed_batch()
    got = oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens,
                                nthreads=nthreads)
    assert got.size == b.total_out()
    out_off = b.out_offsets()
    for i in range(b.n):
        o, L, d = int(out_off[i]), int(b.lens[i]), int(b.out_lens[i])
        msg = b.msgs[int(b.offsets[i]): int(b.offsets[i]) + L].tobytes()
        v = int(b.variants[i])
        piece = got[o: o + d].tobytes()
        assert piece == oracle_mod.hash(v, msg, d), (i, v, L, d)
        assert piece == _ref(v, msg, d), (i, v, L, d)


def test_oracle_hash_batch_rejects_bad_descriptors(oracle_mod):
    b = _mixed_batch()
    bad = b.variants.copy()
    bad[3] = 6
    with pytest.raises(ValueError):
        oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, bad, b.out_lens)
    empty = oracle_mod.hash_batch(np.zeros(0, np.uint8), np.zeros(0, np.uint64),
                                  np.zeros(0, np.uint64), np.zeros(0, np.uint8),
                                  np.zeros(0, np.uint32))
    assert empty.size == 0
