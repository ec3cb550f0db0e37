"""Host logic of keccak_batch_uniform_host: how a batch is cut into pipeline
chunks (csrc/host_chunks.h).  Compiled with g++ into a small driver that
prints the chunk sizes; no GPU involved."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "host_chunks.h"
int main(int argc, char **argv) {
    const unsigned long long n = strtoull(argv[1], 0, 10), chunk = strtoull(argv[2], 0, 10);
    for (unsigned long long c : kb::pipeline_chunks(n, chunk)) printf("%llu\n", c);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("chunks")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1902_05320_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return str(exe)


def chunks(driver, n, chunk):
    out = subprocess.run([driver, str(n), str(chunk)], capture_output=True, text=True, check=True).stdout
    return [int(v) for v in out.split()]


@pytest.mark.parametrize("n,chunk", [(1, 1), (1, 524288), (7, 3), (100, 32), (1000, 16), (1 << 24, 524288),
                                     ((1 << 24) + 12345, 524288), (524288, 524288), (524289, 524288),
                                     (600000, 524288), (31, 17), (10**6, 1)])
def test_chunks_cover_the_batch_and_ramp(driver, n, chunk):
    c = chunks(driver, n, chunk)
    cap = max(1, min(chunk, n))
    assert sum(c) == n and all(0 < v <= cap for v in c)
    base = max(1, cap // 16)
    assert c[0] == min(base, n)
    if len(c) > 1:
        assert c[-1] <= base  # the last copy out is short too
    # A ramp doubles from chunk/16 on each side, so it has at most four steps.
    up = 0
    while up < len(c) - 1 and up < 4 and c[up + 1] == 2 * c[up] and c[up + 1] < cap:
        up += 1
    middle = c[up + 1:len(c) - up - 1] if len(c) > 2 * (up + 1) else []
    if middle:
        # Full chunks, then the remainder.
        assert all(v == cap for v in middle[:-1]) and 0 < middle[-1] <= cap


def test_no_chunks_for_an_empty_batch(driver):
    assert chunks(driver, 0, 100) == []


def test_headline_batch_chunking(driver):
    # 2^24 messages of 64 bytes in 32 MiB chunks: a ramp of 2, 4, 8 and 16 MiB
    # each way around 30 full chunks.
    c = chunks(driver, 1 << 24, 524288)
    assert c[:4] == [32768, 65536, 131072, 262144] and c[-4:] == [262144, 131072, 65536, 32768]
    assert c[4:-4] == [524288] * 30 + [65536]
