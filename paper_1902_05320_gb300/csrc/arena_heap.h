// arena_heap.h -- best-fit allocator over a fixed device arena (host-side
// logic of the serving loop's admission by device-memory budget).  Plain C++,
// no CUDA: it hands out offsets, the caller owns the memory.
//
// Free space is kept as maximal runs (adjacent free runs are merged when a
// region is freed), indexed both by offset and by (length, offset).  An
// allocation takes the shortest run that fits, at its start (lowest offset
// among equally short runs).  A region holds its bytes only while it is
// live: freeing it makes them available at once, whatever the order of
// frees, so a long-lived region does not hold back the space of the regions
// allocated after it.  Since runs are maximal, an allocation fails only when
// no contiguous free stretch of that length exists.
#pragma once

#include <algorithm>
#include <cstdint>
#include <map>
#include <set>
#include <utility>

namespace kb {

class ArenaHeap {
  public:
    explicit ArenaHeap(uint64_t size = 0) { reset(size); }

    void reset(uint64_t size) {
        size_ = size;
        used_ = peak_ = 0;
        by_start_.clear();
        by_len_.clear();
        live_.clear();
        if (size_) add_run(0, size_);
    }

    // Allocates `bytes` (> 0); returns false when no free run is that long.
    bool alloc(uint64_t bytes, uint64_t *start) {
        if (bytes == 0 || bytes > size_) return false;
        const auto it = by_len_.lower_bound({bytes, 0});
        if (it == by_len_.end()) return false;
        const uint64_t len = it->first, s = it->second;
        drop_run(s, len);
        if (len > bytes) add_run(s + bytes, len - bytes);
        live_.emplace(s, bytes);
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        *start = s;
        return true;
    }

    // Frees the live region that starts at `start` (no effect otherwise).
    void free(uint64_t start) {
        const auto it = live_.find(start);
        if (it == live_.end()) return;
        uint64_t s = start, len = it->second;
        live_.erase(it);
        used_ -= len;
        const auto next = by_start_.find(s + len);
        if (next != by_start_.end()) {
            const uint64_t nl = next->second;
            drop_run(s + len, nl);
            len += nl;
        }
        auto prev = by_start_.lower_bound(s);
        if (prev != by_start_.begin()) {
            --prev;
            if (prev->first + prev->second == s) {
                const uint64_t ps = prev->first, pl = prev->second;
                drop_run(ps, pl);
                s = ps;
                len += pl;
            }
        }
        add_run(s, len);
    }

    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }  // bytes in live regions
    uint64_t peak() const { return peak_; }
    size_t live() const { return live_.size(); }
    size_t free_runs() const { return by_start_.size(); }
    uint64_t largest_free() const { return by_len_.empty() ? 0 : by_len_.rbegin()->first; }

  private:
    void add_run(uint64_t s, uint64_t len) {
        by_start_.emplace(s, len);
        by_len_.emplace(len, s);
    }
    void drop_run(uint64_t s, uint64_t len) {
        by_start_.erase(s);
        by_len_.erase({len, s});
    }

    uint64_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<uint64_t, uint64_t> by_start_;          // free run: start -> length
    std::set<std::pair<uint64_t, uint64_t>> by_len_;  // free run: (length, start)
    std::map<uint64_t, uint64_t> live_;               // live region: start -> length
};

}  // namespace kb
