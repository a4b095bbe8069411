// cvs_arena.h - first-fit allocator over one pre-allocated device region.
//
// The serving loop reserves all of its frame and map memory at start-up as one
// cudaMalloc and carves requests out of it with this allocator, so admitting a
// request never calls cudaMalloc (which would synchronise the whole device and
// serialise the streams that are meant to overlap).  Host-only bookkeeping:
// offsets, never dereferenced here.  Not thread-safe (the server locks it).
#pragma once
#include <cstdint>
#include <iterator>
#include <map>

namespace cvs {

class Arena {
  public:
    static constexpr int64_t kAlign = 256;

    explicit Arena(int64_t size = 0) { reset(size); }

    void reset(int64_t size) {
        free_.clear();
        used_.clear();
        size_ = size - size % kAlign;
        if (size_ > 0) free_[0] = size_;
        in_use_ = 0;
        peak_ = 0;
    }

    // Offset of a block of at least `bytes` (rounded up to kAlign), or -1.
    int64_t alloc(int64_t bytes) {
        if (bytes <= 0) bytes = 1;
        const int64_t need = (bytes + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const int64_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[off + need] = len - need;
            used_[off] = need;
            in_use_ += need;
            if (in_use_ > peak_) peak_ = in_use_;
            return off;
        }
        return -1;
    }

    // Return a block; adjacent free blocks are merged.  False if `off` is not
    // the start of a live block.
    bool release(int64_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        int64_t start = off, len = u->second;
        in_use_ -= len;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        return true;
    }

    int64_t size() const { return size_; }
    int64_t in_use() const { return in_use_; }
    int64_t peak() const { return peak_; }
    int64_t largest_free() const {
        int64_t m = 0;
        for (const auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    int64_t free_blocks() const { return (int64_t)free_.size(); }

  private:
    std::map<int64_t, int64_t> free_;  // offset -> length
    std::map<int64_t, int64_t> used_;  // offset -> length
    int64_t size_ = 0, in_use_ = 0, peak_ = 0;
};

}  // namespace cvs
