// First-fit allocator over a byte range, used by the server to admit
// requests by device memory (include/permx.h, serve_*): offsets and sizes are
// rounded up to 256 bytes (a zero-byte request takes 256, so every block
// holds space and the free list never carries empty entries), freed blocks
// merge with free neighbours.  Host only; the server owns the device range
// the offsets point into.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <iterator>
#include <map>

namespace permx {

inline size_t arena_round(size_t x) { return x == 0 ? 256 : (x + 255) & ~size_t(255); }

class Arena {
public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
        used_ = 0;
    }
    // offset of a block of at least `bytes` (rounded up), or -1 if none fits
    int64_t alloc(size_t bytes) {
        bytes = arena_round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return (int64_t)off;
            }
        }
        return -1;
    }
    // return a block that alloc(bytes) gave at `off`
    void release(size_t off, size_t bytes) {
        bytes = arena_round(bytes);
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
    size_t used() const { return used_; }
    size_t free_blocks() const { return free_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    std::map<size_t, size_t> free_;   // offset -> length of each free block
    size_t used_ = 0;
};

}  // namespace permx
