// Host-side policies of the server, free of CUDA so that they can be tested
// on their own: the first-fit arena allocator that hands out the server's
// device (and pinned staging) memory, the rule that merges the crops of
// queries on the same frame into shared integral-histogram regions, and the
// bookkeeping of integral histograms kept resident between micro-batches.
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>
#include <string>
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

// Integral histograms kept resident in the server's arena after the
// micro-batch that built them, for later queries on the same frame. A block is
// one arena allocation (the memory of one build); it holds one or more
// entries, each a rectangle of one frame built with a given key (pixel type,
// bit depth, bins, term set and ring: integral histograms are reusable only
// by queries with the same key). A block in use by running micro-batches
// (users > 0) is never evicted; the others go least recently used first.
// Invalidating a frame drops its entries at once; a block without entries is
// freed as soon as no micro-batch uses it.
class ResidentCache {
  public:
    struct Entry {
        int frame = 0;
        Rect rect;
        std::string key;
        int block = 0;
        int region = 0;  // region index within the block's build
    };
    struct Block {
        uint64_t off = 0, bytes = 0;
        int users = 0;
        uint64_t last_use = 0;
        int entries = 0;
    };

    // a new block of arena memory [off, off + bytes) with no entries yet
    int add_block(uint64_t off, uint64_t bytes)
    {
        const int id = next_++;
        Block b;
        b.off = off;
        b.bytes = bytes;
        b.last_use = ++clock_;
        blocks_[id] = b;
        bytes_ += bytes;
        return id;
    }

    void add_entry(int block, int frame, const Rect &r, const std::string &key, int region)
    {
        Entry e;
        e.frame = frame;
        e.rect = r;
        e.key = key;
        e.block = block;
        e.region = region;
        entries_.push_back(e);
        ++blocks_[block].entries;
    }

    // the entry whose rectangle of this frame holds crop c under this key
    // (the smallest such), or -1
    int find(int frame, const std::string &key, const Rect &c) const
    {
        int best = -1;
        for (size_t i = 0; i < entries_.size(); ++i) {
            const Entry &e = entries_[i];
            if (e.frame != frame || e.key != key) continue;
            if (c.x0 < e.rect.x0 || c.y0 < e.rect.y0 || c.x0 + c.w > e.rect.x0 + e.rect.w ||
                c.y0 + c.h > e.rect.y0 + e.rect.h)
                continue;
            if (best < 0 || e.rect.area() < entries_[best].rect.area()) best = (int)i;
        }
        return best;
    }

    const Entry &entry(int i) const { return entries_[i]; }
    const Block &block(int id) const { return blocks_.at(id); }

    void acquire(int block)
    {
        Block &b = blocks_.at(block);
        ++b.users;
        b.last_use = ++clock_;
    }

    // one use ends; returns true (and forgets the block) when it must be
    // freed now: no user and no entry left
    bool release(int block, uint64_t &off, uint64_t &bytes)
    {
        Block &b = blocks_.at(block);
        --b.users;
        b.last_use = ++clock_;
        return drop_if_empty(block, off, bytes);
    }

    // drop every entry of the frame; the blocks to free now are appended
    // (ids to freed_ids when given)
    void invalidate_frame(int frame, std::vector<std::pair<uint64_t, uint64_t>> &to_free,
                          std::vector<int> *freed_ids = nullptr)
    {
        std::vector<int> touched;
        for (size_t i = 0; i < entries_.size();) {
            if (entries_[i].frame == frame) {
                --blocks_[entries_[i].block].entries;
                touched.push_back(entries_[i].block);
                entries_.erase(entries_.begin() + (long)i);
            } else {
                ++i;
            }
        }
        for (int id : touched) {
            uint64_t off = 0, bytes = 0;
            if (blocks_.count(id) && drop_if_empty(id, off, bytes)) {
                to_free.push_back({off, bytes});
                if (freed_ids) freed_ids->push_back(id);
            }
        }
    }

    // the least recently used block nobody uses: its entries are dropped and
    // it is forgotten; false when every block is in use
    bool evict_one(uint64_t &off, uint64_t &bytes, int *evicted = nullptr)
    {
        int victim = -1;
        for (auto &kv : blocks_)
            if (kv.second.users == 0 && (victim < 0 || kv.second.last_use < blocks_[victim].last_use))
                victim = kv.first;
        if (victim < 0) return false;
        for (size_t i = 0; i < entries_.size();) {
            if (entries_[i].block == victim) entries_.erase(entries_.begin() + (long)i);
            else ++i;
        }
        off = blocks_[victim].off;
        bytes = blocks_[victim].bytes;
        bytes_ -= bytes;
        blocks_.erase(victim);
        ++evictions_;
        if (evicted) *evicted = victim;
        return true;
    }

    uint64_t resident_bytes() const { return bytes_; }
    uint64_t evictions() const { return evictions_; }
    size_t n_entries() const { return entries_.size(); }
    size_t n_blocks() const { return blocks_.size(); }

  private:
    bool drop_if_empty(int id, uint64_t &off, uint64_t &bytes)
    {
        Block &b = blocks_.at(id);
        if (b.users > 0 || b.entries > 0) return false;
        off = b.off;
        bytes = b.bytes;
        bytes_ -= b.bytes;
        blocks_.erase(id);
        return true;
    }

    std::vector<Entry> entries_;
    std::map<int, Block> blocks_;
    int next_ = 0;
    uint64_t clock_ = 0, bytes_ = 0, evictions_ = 0;
};

}  // namespace swih
