// heget_arena.h -- first-fit allocator of byte ranges, used by the request
// server to place each admitted request's tile partials and result in its
// device arena.  Host code only: it hands out offsets, never touches memory.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace heget {

// Offsets and lengths in bytes; every range is rounded up to 256 bytes, so
// offsets stay 256-aligned.  Freed ranges merge with free neighbours.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;      // offset -> length of each free range
    void init(size_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    // The lowest free range that fits n bytes; false if none does.
    bool alloc(size_t n, size_t* off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    // Returns a range obtained from alloc(n) (same n).
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
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
};

}  // namespace heget
