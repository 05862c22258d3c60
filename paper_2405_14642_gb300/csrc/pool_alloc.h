// First-fit allocator over the offsets [0, size) of the serving loop's device
// result pool, with coalescing frees.  Host code only (it hands out offsets;
// the caller owns the memory).  Free blocks are kept in address order, so
// alloc() returns the lowest offset whose free block is large enough.
#pragma once
#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>

namespace bn {

class PoolAllocator {
  public:
    explicit PoolAllocator(uint64_t size) : size_(size) {
        if (size) free_[0] = size;
    }
    // Reserves `bytes` (> 0) at the lowest fitting offset; false if none fits.
    bool alloc(uint64_t bytes, uint64_t *off) {
        if (bytes == 0) return false;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes;
            const uint64_t start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            high_ = std::max(high_, used_);
            return true;
        }
        return false;
    }
    // Returns a block obtained from alloc(); merges it with free neighbours.
    void release(uint64_t off, uint64_t bytes) {
        auto next = free_.lower_bound(off);
        uint64_t start = off, len = bytes;
        if (next != free_.end() && next->first == off + bytes) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        used_ -= bytes;
    }
    uint64_t used() const { return used_; }
    uint64_t high_water() const { return high_; }
    uint64_t size() const { return size_; }
    size_t free_blocks() const { return free_.size(); }

  private:
    uint64_t size_, used_ = 0, high_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

}  // namespace bn
