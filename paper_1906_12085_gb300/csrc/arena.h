// First-fit allocator over one contiguous range [0, size) (offsets only; the
// serving loop maps them onto its device arena).  Blocks are rounded up to 256
// bytes; freed blocks merge with free neighbours.  Host-only C++, no CUDA.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace gbr {

class Arena {
  public:
    static constexpr size_t kAlign = 256;
    static size_t round(size_t bytes) { return (bytes + kAlign - 1) & ~(kAlign - 1); }

    void init(size_t size) {
        size_ = size & ~(kAlign - 1);
        used_ = 0;
        free_.clear();
        if (size_) free_[0] = size_;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t largest_free() const {
        size_t b = 0;
        for (const auto &f : free_) b = f.second > b ? f.second : b;
        return b;
    }
    size_t free_blocks() const { return free_.size(); }

    // Lowest-offset free block that fits; false when none does.
    bool alloc(size_t bytes, size_t *off) {
        bytes = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t o = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[o + bytes] = rest;
            used_ += bytes;
            *off = o;
            return true;
        }
        return false;
    }

    // Returns a block obtained from alloc (same byte count).
    void release(size_t off, size_t bytes) {
        bytes = round(bytes ? bytes : 1);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
};

}  // namespace gbr
