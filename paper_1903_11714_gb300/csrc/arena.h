// Offset bookkeeping of a batch's arena (the HBM budget a batch admits lattices
// against): first-fit placement in 256-byte granules over one region of `size`
// bytes, with the free blocks kept by offset and merged with their neighbours on
// release, so that free space is always a list of maximal gaps.  Host code only
// (the region itself is allocated by the caller).
#pragma once
#include <cstdint>
#include <iterator>
#include <map>

namespace ising {

struct FreeList {
    static constexpr int64_t kGranule = 256;
    int64_t size = 0;
    int64_t used = 0;
    std::map<int64_t, int64_t> free_;  // offset -> length

    static int64_t round_up(int64_t bytes) { return (bytes + kGranule - 1) / kGranule * kGranule; }

    void reset(int64_t bytes)
    {
        size = round_up(bytes);
        used = 0;
        free_.clear();
        free_[0] = size;
    }
    // offset of a block of at least `bytes` (rounded up to granules), the free
    // block with the lowest offset that fits; -1 when none does
    int64_t alloc(int64_t bytes)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used += bytes;
                return off;
            }
        }
        return -1;
    }
    // returns a block that alloc gave out (same offset and byte count)
    void release(int64_t off, int64_t bytes)
    {
        bytes = round_up(bytes);
        used -= bytes;
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
};

}  // namespace ising
