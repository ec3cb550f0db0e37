// host_chunks.h -- how the host-buffer pipeline cuts a batch of n messages
// into chunks (plain C++, no CUDA; unit-tested on the CPU).
//
// Chunks hold at most `chunk` messages.  Their sizes ramp up from chunk/16,
// doubling, at the start and mirror that ramp at the end, so that the first
// copy in and the last copy out, which nothing overlaps, are short.  What
// lies between is cut into full chunks and, last, the remainder, so that
// the full chunks start at whole multiples of the chunk after the ramp (cut
// into equal sizes instead, one end-to-end run measured 2616 against
// 2723-2747 Mhash/s).  The sizes add up to n; none is empty.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace kb {

inline std::vector<uint64_t> pipeline_chunks(uint64_t n, uint64_t chunk) {
    std::vector<uint64_t> counts;
    if (n == 0) return counts;
    chunk = std::max<uint64_t>(1, std::min(chunk, n));
    const uint64_t base = std::max<uint64_t>(1, chunk / 16);
    uint64_t remaining = n;
    std::vector<uint64_t> tail;
    for (uint64_t c = base; c < chunk && remaining; c *= 2) {
        const uint64_t take = std::min(c, remaining);
        counts.push_back(take);
        remaining -= take;
        if (!remaining) break;
        const uint64_t take_tail = std::min(c, remaining);
        tail.push_back(take_tail);
        remaining -= take_tail;
    }
    for (; remaining; remaining -= std::min(chunk, remaining)) counts.push_back(std::min(chunk, remaining));
    counts.insert(counts.end(), tail.rbegin(), tail.rend());
    return counts;
}

}  // namespace kb
