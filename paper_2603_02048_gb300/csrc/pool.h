// First-fit allocator over a fixed byte range, in offsets (host logic only:
// the server maps offsets into one device allocation of its memory budget).
// Free blocks are kept coalesced; every block starts on an `align` boundary.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace hh {

class OffsetPool {
   public:
    explicit OffsetPool(size_t capacity = 0, size_t align = 256) { reset(capacity, align); }

    void reset(size_t capacity, size_t align = 256) {
        align_ = align ? align : 1;
        cap_ = capacity - capacity % align_;
        used_ = 0;
        free_.clear();
        live_.clear();
        if (cap_) free_[0] = cap_;
    }

    // Reserves `bytes` (rounded up to the alignment; 0 counts as one unit).
    // Returns false when no free block is large enough.
    bool alloc(size_t bytes, size_t* off) {
        const size_t need = round_up(bytes ? bytes : 1);
        if (need == 0 || need > cap_) return false;  // 0: rounding overflowed
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t o = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest) free_[o + need] = rest;
            live_[o] = need;
            used_ += need;
            *off = o;
            return true;
        }
        return false;
    }

    // Returns a block; false for an offset that is not a live block.
    bool release(size_t off) {
        auto it = live_.find(off);
        if (it == live_.end()) return false;
        size_t o = it->first, n = it->second;
        live_.erase(it);
        used_ -= n;
        auto next = free_.lower_bound(o);
        if (next != free_.end() && o + n == next->first) {  // merge with the following block
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {  // merge with the preceding block
            auto prev = std::prev(next);
            if (prev->first + prev->second == o) {
                prev->second += n;
                return true;
            }
        }
        free_[o] = n;
        return true;
    }

    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t live_blocks() const { return live_.size(); }
    size_t free_blocks() const { return free_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    // Bytes one allocation of `bytes` occupies.
    size_t footprint(size_t bytes) const { return round_up(bytes ? bytes : 1); }

   private:
    size_t round_up(size_t b) const {
        const size_t r = b % align_;
        return r ? (b > SIZE_MAX - (align_ - r) ? 0 : b + (align_ - r)) : b;
    }

    size_t cap_ = 0, align_ = 256, used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> size, coalesced
    std::map<size_t, size_t> live_;  // offset -> size
};

}  // namespace hh
