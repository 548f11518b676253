// Host-side policies of the server, free of CUDA so that they can be tested
// on their own: the first-fit arena allocator that hands out the server's
// device (and pinned staging) memory, and the rule that merges the crops of
// queries on the same frame into shared integral-histogram regions.
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace swih {

// First-fit allocator over [0, size) with 256-byte granules. Free blocks are
// kept by offset and coalesced with their neighbours on release.
class Arena {
  public:
    static constexpr uint64_t kAlign = 256;

    explicit Arena(uint64_t size = 0) { reset(size); }

    void reset(uint64_t size)
    {
        size_ = size / kAlign * kAlign;
        free_.clear();
        if (size_) free_[0] = size_;
        used_ = 0;
    }

    static uint64_t granules(uint64_t bytes) { return (bytes + kAlign - 1) / kAlign * kAlign; }

    // first free block that holds the request; false when none does
    bool alloc(uint64_t bytes, uint64_t &off)
    {
        const uint64_t need = granules(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            off = it->first;
            const uint64_t rest = it->second - need;
            free_.erase(it);
            if (rest) free_[off + need] = rest;
            used_ += need;
            return true;
        }
        return false;
    }

    void release(uint64_t off, uint64_t bytes)
    {
        uint64_t len = granules(bytes ? bytes : 1);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            free_.erase(next);
        }
        free_[off] = len;
    }

    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    uint64_t largest_free() const
    {
        uint64_t m = 0;
        for (const auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t free_blocks() const { return free_.size(); }
    const std::map<uint64_t, uint64_t> &free_map() const { return free_; }

  private:
    uint64_t size_ = 0, used_ = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
};

struct Rect {
    int x0 = 0, y0 = 0, w = 0, h = 0;
    int64_t area() const { return (int64_t)w * h; }
};

inline Rect bounding(const Rect &a, const Rect &b)
{
    const int x0 = std::min(a.x0, b.x0), y0 = std::min(a.y0, b.y0);
    const int x1 = std::max(a.x0 + a.w, b.x0 + b.w), y1 = std::max(a.y0 + a.h, b.y0 + b.h);
    return Rect{x0, y0, x1 - x0, y1 - y0};
}

// Crops of queries that share a frame, bin count and kernel are merged into
// regions whose integral histograms serve all of them. Visiting the crops in
// order, a crop joins the first region whose bounding box, grown to cover it,
// has no more pixels than the region and the crop had apart (so a merge
// never adds quantisation or scan work) and no wider than max_w; otherwise
// it opens a region. Regions are merged the same way until none changes.
// Returns each crop's region index; regions receives the bounding boxes.
inline std::vector<int> merge_crops(const std::vector<Rect> &crops, std::vector<Rect> &regions, int max_w)
{
    std::vector<int> of(crops.size(), -1);
    regions.clear();
    for (size_t i = 0; i < crops.size(); ++i) {
        int dst = -1;
        for (size_t r = 0; r < regions.size(); ++r) {
            const Rect b = bounding(regions[r], crops[i]);
            if (b.w <= max_w && b.area() <= regions[r].area() + crops[i].area()) {
                dst = (int)r;
                regions[r] = b;
                break;
            }
        }
        if (dst < 0) {
            dst = (int)regions.size();
            regions.push_back(crops[i]);
        }
        of[i] = dst;
    }
    // regions that grew may now overlap: merge pairs under the same rule
    bool changed = true;
    while (changed) {
        changed = false;
        for (size_t a = 0; a < regions.size() && !changed; ++a)
            for (size_t b = a + 1; b < regions.size() && !changed; ++b) {
                const Rect u = bounding(regions[a], regions[b]);
                if (u.w <= max_w && u.area() <= regions[a].area() + regions[b].area()) {
                    regions[a] = u;
                    regions.erase(regions.begin() + (long)b);
                    for (int &o : of) {
                        if (o == (int)b) o = (int)a;
                        else if (o > (int)b) --o;
                    }
                    changed = true;
                }
            }
    }
    return of;
}

}  // namespace swih
