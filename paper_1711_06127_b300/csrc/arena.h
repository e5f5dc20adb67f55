// arena.h -- first-fit allocator over an offset range (host-side bookkeeping
// only; the server maps offsets onto one device allocation).  Blocks are
// multiples of kAlign bytes; freed blocks coalesce with free neighbours.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <unordered_map>

namespace supra {

class OffsetArena {
   public:
    static constexpr size_t kAlign = 256;
    static constexpr size_t kNone = SIZE_MAX;

    void reset(size_t bytes) {
        size_ = bytes / kAlign * kAlign;
        used_ = peak_ = 0;
        free_.clear();
        sizes_.clear();
        if (size_) free_[0] = size_;
    }
    // Offset of a new block of at least `bytes` (lowest fitting address), or kNone.
    size_t alloc(size_t bytes) {
        bytes = (std::max<size_t>(bytes, 1) + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            sizes_[off] = bytes;
            return off;
        }
        return kNone;
    }
    // Frees a block returned by alloc (unknown offsets are ignored).
    void free(size_t off) {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + len) {
            len += next->second;
            free_.erase(next);
        }
        auto it = free_.emplace(off, len).first;
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == off) {
                prev->second += len;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t free_blocks() const { return free_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }

   private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;            // offset -> length
    std::unordered_map<size_t, size_t> sizes_; // allocated offset -> length
};

}  // namespace supra
