"""The N>1 path of bench.py on CPU: two gloo ranks, each with its own seeded
inputs (weak scaling, no collective on the data), the step time reduced to the
slowest rank and the value counting the messages of every rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1902_05320_gb300 import workloads

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        msgs = workloads.uniform_messages(64, 64, seed=bench.rank_seed(1, rank))
        ms = bench.max_over_ranks(1.0 + rank, world)   # ranks report 1 ms and 2 ms
        value = bench.whole_job_mhash_s(1 << 24, world, ms)
        out[rank] = (ms, value, msgs[:16].tobytes())
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_reduce_time_and_count_all_messages():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (ms0, v0, m0), (ms1, v1, m1) = out[0], out[1]
    assert ms0 == ms1 == 2.0                       # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * (1 << 24) / 2e-3 / 1e6)
    assert m0 != m1                                 # each rank hashes its own messages
    np.testing.assert_equal(len(m0), 16)
