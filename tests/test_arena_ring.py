"""Host logic of the serving loop's admission: the ring allocator over the
device arena (csrc/arena_ring.h) never hands out overlapping or out-of-range
regions, frees in any order, and refuses what does not fit.  Compiled with g++
into a small test driver; no GPU involved."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include "arena_ring.h"
int main(int argc, char **argv) {
    unsigned long long seed = strtoull(argv[1], 0, 10);
    auto rnd = [&]() { seed ^= seed << 13; seed ^= seed >> 7; seed ^= seed << 17; return seed; };
    const uint64_t size = 1 + rnd() % 5000;
    kb::ArenaRing ring(size);
    struct Live { uint64_t s, b; };
    std::vector<Live> live;
    for (int step = 0; step < 20000; ++step) {
        if (live.empty() || rnd() % 3) {
            uint64_t b = 1 + rnd() % (size / 3 + 1), s;
            if (ring.alloc(b, &s)) {
                if (s + b > size) { printf("out of range\n"); return 1; }
                for (auto &l : live)
                    if (s < l.s + l.b && l.s < s + b) { printf("overlap\n"); return 1; }
                live.push_back({s, b});
            } else {
                uint64_t total = 0;
                for (auto &l : live) total += l.b;
                if (live.empty()) { printf("refused on empty arena\n"); return 1; }
            }
        } else {
            size_t k = rnd() % live.size();
            ring.free(live[k].s);
            live.erase(live.begin() + k);
        }
        if (ring.used() > size) { printf("used exceeds size\n"); return 1; }
    }
    for (auto &l : live) ring.free(l.s);
    if (ring.used() != 0 || ring.live() != 0) { printf("leak\n"); return 1; }
    uint64_t s;
    if (!ring.alloc(size, &s) || s != 0) { printf("empty arena refused a full-size region\n"); return 1; }
    printf("ok\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("arena")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1902_05320_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("seed", range(1, 41))
def test_arena_ring_random_sequences(driver, seed):
    r = subprocess.run([driver, str(seed * 7919)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
