"""The serving loop (kb_server_*): continuous batching of requests that arrive
one by one, admitted against a device-memory budget.  Outputs are checked
against the CPU oracle (all of them at small loads, a sample at the full
bench load), and each result must be the same when the message is hashed
alone as when it went through the server mixed with others."""
import os

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))


def _pinned(torch, arr: np.ndarray):
    t = torch.empty(max(arr.size, 1), dtype=torch.uint8, pin_memory=True)
    if arr.size:
        t[: arr.size] = torch.from_numpy(arr)
    return t


def _replay(server, torch, wl):
    pool = _pinned(torch, wl.pool)
    total = int(wl.out_lens.sum(dtype=np.uint64))
    outputs = torch.full((max(total, 1),), 0xEE, dtype=torch.uint8, pin_memory=True)
    lat = np.zeros(wl.n, dtype=np.int64)
    stats = server.replay(pool, wl.offsets, wl.lens, wl.variants, wl.out_lens, wl.arrival_ns, outputs, lat)
    return outputs.numpy()[:total].copy(), lat, stats, pool


@pytest.mark.parametrize("long_lane_parallel", [True, False])
def test_server_replay_matches_oracle(cuda_lib, oracle_mod, long_lane_parallel):
    import torch

    from paper_1902_05320_gb300.serve import Server

    wl = W.serving_workload(50_000, 0.05, seed=501, max_len=65536, pool_bytes=64 << 20)
    with Server(hbm_budget_bytes=256 << 20, max_inflight=8, max_batch_requests=1024,
                long_lane_parallel=long_lane_parallel) as srv:
        got, lat, stats, _ = _replay(srv, torch, wl)
    assert stats["requests"] == wl.n and (lat > 0).all()
    assert stats["lat_p50_us"] <= stats["lat_p99_us"] <= stats["lat_max_us"]
    # The latency's parts: each request is submitted no earlier than its
    # arrival, launched after it is submitted and completed after its launch.
    assert 0 <= stats["submit_lag_p50_us"] <= stats["submit_lag_p99_us"] <= stats["lat_max_us"]
    assert 0 <= stats["queue_wait_p50_us"] <= stats["queue_wait_p99_us"] <= stats["lat_max_us"]
    assert 0 < stats["service_p50_us"] <= stats["service_p99_us"] <= stats["lat_max_us"]
    want = oracle_mod.hash_batch(wl.pool, wl.offsets, wl.lens, wl.variants, wl.out_lens, THREADS)
    assert np.array_equal(got, want)


def test_server_result_alone_equals_result_in_the_mix(cuda_lib):
    import torch

    from paper_1902_05320_gb300.serve import Server

    wl = W.serving_workload(100_000, 0.02, seed=502, max_len=200_000, pool_bytes=32 << 20)
    with Server(hbm_budget_bytes=128 << 20, max_inflight=16, max_batch_requests=256) as srv:
        mixed, _, stats, _ = _replay(srv, torch, wl)
    assert stats["batches"] > 1  # the requests really were batched while others ran
    pos = np.concatenate([[0], np.cumsum(wl.out_lens[:-1], dtype=np.uint64)])
    d_pool = torch.from_numpy(wl.pool).cuda()
    for i in np.random.default_rng(1).choice(wl.n, size=min(80, wl.n), replace=False):
        out = torch.zeros(int(wl.out_lens[i]), dtype=torch.uint8, device="cuda")
        one = lambda a, dt: torch.tensor([int(a)], dtype=dt, device="cuda")  # noqa: E731
        offs, lens = one(wl.offsets[i], torch.int64), one(wl.lens[i], torch.int64)
        var, ol = one(wl.variants[i], torch.uint8), one(wl.out_lens[i], torch.int32)
        cuda_lib.keccak_batch(d_pool, offs, lens, var, ol, out, 1)
        torch.cuda.synchronize()
        alone = out.cpu().numpy()
        assert np.array_equal(alone, mixed[int(pos[i]):int(pos[i]) + int(wl.out_lens[i])]), i


def test_server_admission_under_a_small_budget(cuda_lib, oracle_mod):
    import torch

    from paper_1902_05320_gb300 import binding
    from paper_1902_05320_gb300.serve import Server

    budget = 192 << 10
    wl = W.serving_workload(20_000, 0.02, seed=503, max_len=64 << 10, pool_bytes=4 << 20)
    with Server(hbm_budget_bytes=budget, max_inflight=4, max_batch_requests=64) as srv:
        got, _, stats, pool = _replay(srv, torch, wl)
        assert stats["peak_arena_bytes"] <= budget
        # A message that can never fit the budget is refused at once.
        out = Server.pinned(32)
        with pytest.raises(binding.Sha3gbError) as e:
            srv.submit(pool.data_ptr(), budget + 1, 1, 32, out.data_ptr())
        assert e.value.status == binding.KB_ERR_TOO_LARGE
    want = oracle_mod.hash_batch(wl.pool, wl.offsets, wl.lens, wl.variants, wl.out_lens, THREADS)
    assert np.array_equal(got, want)


def test_server_submit_and_wait(cuda_lib, oracle_mod):
    import torch

    from paper_1902_05320_gb300.serve import Server

    msgs = [W.random_bytes(n, seed=600 + n) for n in (0, 1, 135, 136, 5000, 300_000)]
    with Server(hbm_budget_bytes=64 << 20) as srv:
        bufs, outs, tickets = [], [], []
        for k, m in enumerate(msgs):
            variant, out_len = (k % 6, (28, 32, 48, 64, 100, 700)[k % 6])
            b = _pinned(torch, m)
            o = Server.pinned(out_len)
            tickets.append((srv.submit(b.data_ptr(), m.size, variant, out_len, o.data_ptr()), variant, out_len))
            bufs.append(b)
            outs.append(o)
        for (t, variant, out_len), o, m in zip(tickets, outs, msgs):
            srv.wait(t, timeout_ms=20_000)
            assert o.numpy()[:out_len].tobytes() == oracle_mod.hash(variant, m.tobytes(), out_len)


def test_full_size_serving_run_sampled(cuda_lib, oracle_mod):
    # The bench's serving load in full (Poisson 200k req/s for 10 s, 32 B..1 MiB,
    # a 4 GiB pool, a 2 GiB budget): every request completes, 300 sampled
    # outputs equal the oracle's and 20,000 equal hashlib's.
    import hashlib
    from concurrent.futures import ThreadPoolExecutor

    import torch

    from paper_1902_05320_gb300.serve import Server

    wl = W.serving_workload(200_000, 10.0, seed=5, pool_bytes=4 << 30)
    with Server(hbm_budget_bytes=2 << 30, max_inflight=48, max_batch_requests=4096) as srv:
        got, lat, stats, _ = _replay(srv, torch, wl)
    assert stats["requests"] == wl.n and (lat > 0).all()
    pos = np.concatenate([[0], np.cumsum(wl.out_lens[:-1], dtype=np.uint64)])
    rng = np.random.default_rng(55)
    idx = rng.choice(wl.n, size=300, replace=False)
    want = oracle_mod.hash_batch(wl.pool, wl.offsets[idx], wl.lens[idx], wl.variants[idx], wl.out_lens[idx], THREADS)
    at = 0
    for i in idx:
        ln = int(wl.out_lens[i])
        assert np.array_equal(got[int(pos[i]):int(pos[i]) + ln], want[at:at + ln]), i
        at += ln
    fns = (hashlib.sha3_224, hashlib.sha3_256, hashlib.sha3_384, hashlib.sha3_512)

    def check(i):
        o, ln, v, d = int(wl.offsets[i]), int(wl.lens[i]), int(wl.variants[i]), int(wl.out_lens[i])
        m = wl.pool[o:o + ln]
        h = fns[v](m).digest() if v < 4 else (hashlib.shake_128 if v == 4 else hashlib.shake_256)(m).digest(d)
        return h == got[int(pos[i]):int(pos[i]) + d].tobytes()

    with ThreadPoolExecutor(THREADS) as ex:
        assert all(ex.map(check, rng.choice(wl.n, size=20_000, replace=False)))
