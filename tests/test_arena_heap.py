"""Host logic of the serving loop's admission: the best-fit allocator over the
device arena (csrc/arena_heap.h) never hands out overlapping or out-of-range
regions, frees in any order, refuses a request only when no free stretch of
its length exists (checked against a byte map of the arena), and merges free
space back into one run.  Compiled with g++ into a small test driver; no GPU
involved."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "arena_heap.h"
int main(int argc, char **argv) {
    unsigned long long seed = strtoull(argv[1], 0, 10);
    auto rnd = [&]() { seed ^= seed << 13; seed ^= seed >> 7; seed ^= seed << 17; return seed; };
    const uint64_t size = 1 + rnd() % 5000;
    kb::ArenaHeap heap(size);
    std::vector<unsigned char> used(size, 0);  // byte map: 1 = inside a live region
    struct Live { uint64_t s, b; };
    std::vector<Live> live;
    uint64_t live_bytes = 0, peak = 0;
    auto longest_free = [&]() {
        uint64_t best = 0, run = 0;
        for (uint64_t i = 0; i < size; ++i) { run = used[i] ? 0 : run + 1; if (run > best) best = run; }
        return best;
    };
    for (int step = 0; step < 20000; ++step) {
        if (live.empty() || rnd() % 3) {
            uint64_t b = 1 + rnd() % (size / 3 + 1), s;
            if (heap.alloc(b, &s)) {
                if (s + b > size) { printf("out of range\n"); return 1; }
                for (uint64_t i = s; i < s + b; ++i)
                    if (used[i]) { printf("overlap\n"); return 1; }
                for (uint64_t i = s; i < s + b; ++i) used[i] = 1;
                live.push_back({s, b});
                live_bytes += b;
                if (live_bytes > peak) peak = live_bytes;
            } else if (longest_free() >= b) {
                printf("refused %llu bytes with a free stretch of %llu\n", (unsigned long long)b,
                       (unsigned long long)longest_free());
                return 1;
            }
        } else {
            size_t k = rnd() % live.size();
            heap.free(live[k].s);
            for (uint64_t i = live[k].s; i < live[k].s + live[k].b; ++i) used[i] = 0;
            live_bytes -= live[k].b;
            live.erase(live.begin() + k);
        }
        if (heap.used() != live_bytes) { printf("used %llu != live bytes\n", (unsigned long long)heap.used()); return 1; }
        if (heap.largest_free() != longest_free()) { printf("largest free run disagrees\n"); return 1; }
        heap.free(size + 7);  // not a live region: no effect
    }
    if (heap.peak() != peak) { printf("peak disagrees\n"); return 1; }
    for (auto &l : live) heap.free(l.s);
    if (heap.used() != 0 || heap.live() != 0 || heap.free_runs() != 1) { printf("leak or unmerged runs\n"); return 1; }
    uint64_t s;
    if (!heap.alloc(size, &s) || s != 0) { printf("empty arena refused a full-size region\n"); return 1; }
    if (heap.alloc(1, &s)) { printf("full arena gave out a byte\n"); return 1; }
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
def test_arena_heap_random_sequences(driver, seed):
    r = subprocess.run([driver, str(seed * 7919)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
