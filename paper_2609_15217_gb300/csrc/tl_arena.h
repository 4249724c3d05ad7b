// tl_arena.h -- host-side bookkeeping of one device memory block (the
// request server's budget): first-fit allocation of 256-byte aligned
// ranges, coalescing on free.  Pure C++, no CUDA: the server owns the
// device block and asks this class for offsets into it.
#pragma once
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace tl {

class Arena {
public:
    static constexpr size_t kAlign = 256;

    explicit Arena(size_t bytes = 0) { reset(bytes); }

    void reset(size_t bytes)
    {
        free_.clear();
        capacity_ = bytes / kAlign * kAlign;
        used_ = 0;
        high_ = 0;
        if (capacity_) free_[0] = capacity_;
    }

    static size_t round_up(size_t bytes) { return (bytes + kAlign - 1) / kAlign * kAlign; }

    // Offset of a free range of at least `bytes` (rounded up to kAlign), or
    // SIZE_MAX when no free range is large enough.  Zero bytes take kAlign.
    size_t alloc(size_t bytes)
    {
        const size_t need = round_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first;
            const size_t rest = it->second - need;
            free_.erase(it);
            if (rest) free_[off + need] = rest;
            used_ += need;
            if (used_ > high_) high_ = used_;
            return off;
        }
        return SIZE_MAX;
    }

    // Return a range obtained from alloc(bytes) with the same `bytes`.
    void release(size_t off, size_t bytes)
    {
        const size_t len = round_up(bytes ? bytes : 1);
        used_ -= len;
        auto next = free_.lower_bound(off);
        size_t start = off, size = len;
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                size += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + len == next->first) {
            size += next->second;
            free_.erase(next);
        }
        free_[start] = size;
    }

    size_t capacity() const { return capacity_; }
    size_t used() const { return used_; }
    size_t high_water() const { return high_; }
    size_t free_ranges() const { return free_.size(); }
    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    std::map<size_t, size_t> free_;  // offset -> length, disjoint, non-adjacent
    size_t capacity_ = 0, used_ = 0, high_ = 0;
};

}  // namespace tl
