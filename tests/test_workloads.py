"""The seeded synthetic inputs (paper_1902_05320_gb300/workloads.py): the
recipe the benchmark and the tests share -- deterministic per seed, inside
their bounds, and with the stated distributions (log-uniform lengths,
Poisson arrivals, uniform variants and SHAKE output sizes)."""
import math

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W


def test_random_bytes_are_seeded_and_uniform():
    a, b, c = W.random_bytes(1 << 20, 1), W.random_bytes(1 << 20, 1), W.random_bytes(1 << 20, 2)
    assert a.dtype == np.uint8 and a.size == 1 << 20
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    counts = np.bincount(a, minlength=256)
    assert counts.min() > 0.9 * (1 << 12) and counts.max() < 1.1 * (1 << 12)  # 4096 expected per value
    assert W.uniform_messages(4096, 64, seed=0).size == 4096 * 64


@pytest.mark.parametrize("max_len,min_len", [(65536, 0), (1 << 20, 32), (300, 0)])
def test_log_uniform_lengths(max_len, min_len):
    rng = np.random.default_rng(5)
    n = 200_000
    lens = W.log_uniform_lengths(rng, n, max_len, min_len).astype(np.int64)
    assert lens.min() >= min_len and lens.max() <= max_len
    # P(len <= k) = ln((k+1)/(min+1)) / ln((max+1)/(min+1)) for the floor(exp(U)) - 1 recipe.
    for k in (min_len, 10 * (min_len + 1), max_len // 2):
        want = math.log((k + 1 + 1) / (min_len + 1)) / math.log((max_len + 1) / (min_len + 1))
        got = float((lens <= k).mean())
        assert abs(got - min(want, 1.0)) < 0.01, (k, got, want)
    if min_len == 0:
        assert (lens == 0).any()


def test_ragged_batch_layout():
    b = W.ragged_batch(20_000, seed=3, max_len=4096, gap=7)
    ends = b.offsets + b.lens
    assert int(ends.max()) <= b.msgs.size
    starts_after = b.offsets[1:] - ends[:-1]  # the random gap between messages
    assert starts_after.min() >= 0 and starts_after.max() <= 7
    assert set(np.unique(b.variants).tolist()) == {0, 1, 2, 3, 4, 5}
    sha3 = b.variants < 4
    assert np.array_equal(b.out_lens[sha3], np.array(W.DIGEST_BYTES[:4], dtype=np.uint32)[b.variants[sha3]])
    shake = b.out_lens[~sha3]
    assert shake.min() >= 16 and shake.max() <= 512
    assert b.total_out() == int(b.out_lens.sum()) and b.out_offsets()[-1] == b.total_out() - b.out_lens[-1]
    again = W.ragged_batch(20_000, seed=3, max_len=4096, gap=7)
    assert np.array_equal(again.msgs, b.msgs) and np.array_equal(again.lens, b.lens)
    packed = W.ragged_batch(1000, seed=4, max_len=100)
    assert np.array_equal(packed.offsets[1:], (packed.offsets + packed.lens)[:-1])  # no gaps by default


def test_serving_workload_is_a_poisson_stream():
    rate, seconds = 50_000, 2.0
    wl = W.serving_workload(rate, seconds, seed=9, max_len=1 << 16, pool_bytes=8 << 20)
    n = wl.n
    assert abs(n - rate * seconds) < 5 * math.sqrt(rate * seconds)
    gaps = np.diff(wl.arrival_ns)
    assert gaps.min() >= 0
    assert abs(gaps.mean() - 1e9 / rate) < 0.02 * 1e9 / rate
    # Exponential gaps: the coefficient of variation is 1.
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03
    assert wl.lens.min() >= 32 and wl.lens.max() <= 1 << 16
    assert int((wl.offsets + wl.lens).max()) <= wl.pool.size
    assert set(np.unique(wl.variants).tolist()) == {0, 1, 2, 3, 4, 5}
