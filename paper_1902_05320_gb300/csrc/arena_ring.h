// arena_ring.h -- ring allocator over a fixed device arena (host-side logic of
// the serving loop's admission by device-memory budget).  Plain C++, no CUDA:
// it hands out offsets, the caller owns the memory.
//
// Regions are allocated in FIFO order at the head and may be freed in any
// order; space is reclaimed from the oldest live region forward.  Live data
// occupies [tail, head) when not wrapped, [tail, size) + [0, head) when
// wrapped.  A region never straddles the end of the arena: when the space up
// to the end is too small, the allocation restarts at 0 and the skipped bytes
// count as used until that region is reclaimed.
#pragma once

#include <cstdint>
#include <deque>

namespace kb {

class ArenaRing {
  public:
    explicit ArenaRing(uint64_t size = 0) : size_(size) {}

    void reset(uint64_t size) {
        size_ = size;
        head_ = tail_ = used_ = peak_ = 0;
        live_.clear();
    }

    // Allocates `bytes` (> 0); returns false when they do not fit now.
    bool alloc(uint64_t bytes, uint64_t *start) {
        if (bytes == 0 || bytes > size_) return false;
        if (live_.empty()) head_ = tail_ = 0;
        const bool wrapped = !live_.empty() && head_ <= tail_;
        uint64_t s, waste = 0;
        if (!wrapped) {
            if (size_ - head_ >= bytes) {
                s = head_;
            } else if (tail_ >= bytes) {
                s = 0;
                waste = size_ - head_;
            } else {
                return false;
            }
        } else {
            if (tail_ - head_ < bytes) return false;
            s = head_;
        }
        live_.push_back(Region{s, bytes, waste, false});
        head_ = s + bytes;
        used_ += bytes + waste;
        if (used_ > peak_) peak_ = used_;
        *start = s;
        return true;
    }

    // Frees the live region that starts at `start`.
    void free(uint64_t start) {
        for (auto &r : live_)
            if (r.start == start && !r.freed) {
                r.freed = true;
                break;
            }
        while (!live_.empty() && live_.front().freed) {
            used_ -= live_.front().bytes + live_.front().waste;
            live_.pop_front();
        }
        if (live_.empty()) {
            head_ = tail_ = 0;
            return;
        }
        tail_ = live_.front().start;
        // Once the region that wrapped to 0 is the oldest, the bytes it skipped
        // at the end of the arena are free space again.
        used_ -= live_.front().waste;
        live_.front().waste = 0;
    }

    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }
    size_t live() const { return live_.size(); }

  private:
    struct Region {
        uint64_t start, bytes, waste;
        bool freed;
    };
    uint64_t size_ = 0, head_ = 0, tail_ = 0, used_ = 0, peak_ = 0;
    std::deque<Region> live_;
};

}  // namespace kb
