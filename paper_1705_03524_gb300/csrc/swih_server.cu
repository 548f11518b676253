// Server (swih_server_*): continuous batching of tracking queries.
//
// A scheduler thread owns a device arena and a pinned staging arena. Waiting
// queries are admitted, oldest first, in micro-batches whenever a stream slot
// is free and their work fits in the arena; a micro-batch that does not fit
// is halved until it does, and when even one query does not fit the
// scheduler waits for running micro-batches to finish. A micro-batch groups
// its queries by (pixel type, bit depth, B, kernel); each group is one work
// set whose regions are the queries' crops, merged per frame where that adds
// no pixels, so queries on the same frame share integral histograms. Each
// micro-batch runs on its own stream (table upload, K1, K2, K3 groups, status
// read-back, host callback), so micro-batches overlap on the device.
//
// Locking: the queue, the completions and the per-slot "done" flags are
// guarded by the server mutex; the arenas and the slots' contents are the
// scheduler thread's alone. No CUDA call is made while the mutex is held
// (the completion callback takes it).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "serve_policy.h"
#include "swih_host.h"

using namespace swih;

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

swih_status sfail(swih_status st, const std::string &msg)
{
    thread_error() = msg;
    return st;
}

struct Query {
    swih_query q;
    swih_frame_desc f;  // copied at submission
    uint64_t id = 0;
    uint64_t submit_ns = 0;
    uint64_t start_ns = 0;
    bool admitting = false;  // copied by the scheduler for a micro-batch being built
};

struct MicroBatch {
    swih_server_s *srv = nullptr;
    int slot = 0;
    std::vector<Query> queries;
    std::vector<std::unique_ptr<WorkSet>> sets;  // build sets (K1, K2) first, then gather sets (K3)
    std::vector<std::vector<int>> set_queries;  // queries whose work is in each set
    std::vector<std::pair<uint64_t, uint64_t>> dev_blocks;  // gather sets' memory: freed at retirement
    // build sets: their memory becomes resident integral histograms at
    // retirement (keep_ih), else it is freed; one block per build set
    struct Built {
        uint64_t off = 0, bytes = 0;
        int set = 0;                    // index into sets
        std::vector<int> frames;        // per region of the set
        std::vector<Rect> rects;
        std::string key;                // pixel type, bit depth, bins, term set and ring
    };
    std::vector<Built> built;
    std::vector<int> held;              // resident blocks this micro-batch reads (one use each)
    std::vector<char> reused;           // per query: its integral histograms were resident
    uint64_t host_off = 0, host_bytes = 0;
    uint32_t *h_status = nullptr;  // pinned, one word per set
    cudaEvent_t ev = nullptr;      // recorded after the status read-back
    bool done = false;             // set by the completion callback (or an event error)
    bool fired = false;            // the completion callback ran
    bool hostfn = false;           // the completion callback was enqueued
    swih_status launch_status = SWIH_OK;
};

// offset (in floats) of map (t, s) in a query's d_out, and the total
uint64_t map_offset(const swih_query &q, int t, int s)
{
    uint64_t per_target = 0, within = 0;
    for (int k = 0; k < q.n_scales; ++k) {
        const uint64_t n = (uint64_t)(q.height - q.win_h[k] + 1) * (uint64_t)(q.width - q.win_w[k] + 1);
        if (k < s) within += n;
        per_target += n;
    }
    return (uint64_t)t * per_target + within;
}

swih_status check_query(const swih_query *q, const swih_frame_desc *f)
{
    if (!q) return sfail(SWIH_ERR_INVALID_ARG, "query is NULL");
    if (q->width < 3 || q->height < 3) return sfail(SWIH_ERR_INVALID_ARG, "crop must be at least 3 x 3");
    if (f && (q->x0 < 0 || q->y0 < 0 || (int64_t)q->x0 + q->width > f->width ||
              (int64_t)q->y0 + q->height > f->height))
        return sfail(SWIH_ERR_INVALID_ARG, "crop is not inside the frame");
    if (q->bins < 1 || q->bins > 256) return sfail(SWIH_ERR_INVALID_ARG, "bins must be in [1, 256]");
    if (q->kernel < SWIH_KERNEL_PLAIN || q->kernel > SWIH_KERNEL_GAUSSIAN)
        return sfail(SWIH_ERR_INVALID_ARG, "unknown kernel");
    if (q->n_targets < 1 || q->n_targets > SWIH_MAX_TARGETS)
        return sfail(SWIH_ERR_INVALID_ARG, "n_targets out of range");
    if (q->n_scales < 1 || q->n_scales > SWIH_MAX_SCALES) return sfail(SWIH_ERR_INVALID_ARG, "n_scales out of range");
    for (int k = 0; k < q->n_scales; ++k)
        if (!odd_window(q->win_w[k]) || !odd_window(q->win_h[k]) || q->win_w[k] > q->width ||
            q->win_h[k] > q->height)
            return sfail(SWIH_ERR_INVALID_ARG, "window sides must be odd, >= 3 and fit the crop");
    return SWIH_OK;
}

WorkSpec spec_of(const swih_server_desc &d, const Query &qr)
{
    WorkSpec sp;
    sp.pixel_type = qr.f.pixel_type;
    sp.bitdepth = qr.f.bitdepth;
    sp.bins = qr.q.bins;
    sp.kernel_mask = SWIH_KERNEL_BIT(qr.q.kernel);
    sp.gauss_degree = d.gauss_degree;
    sp.gauss_sigma_frac = d.gauss_sigma_frac;
    return sp;
}

// Regions of the crops of queries qs[idx] (merge: overlapping crops of one
// frame share a region where that adds no pixels): regions (image rectangles),
// their frame rectangles, and each query's region (region_of, indexed like qs).
void crop_regions(const std::vector<Query> &qs, const std::vector<int> &idx, bool merge,
                  std::vector<WorkRegion> &regions, std::vector<Rect> &rects, std::vector<int> &frames,
                  std::vector<int> &region_of)
{
    regions.clear();
    rects.clear();
    frames.clear();
    region_of.assign(qs.size(), -1);
    std::map<int, std::vector<int>> by_frame;
    for (int i : idx) by_frame[qs[i].q.frame].push_back(i);
    for (auto &kv : by_frame) {
        std::vector<Rect> crops, merged;
        for (int i : kv.second) crops.push_back(Rect{qs[i].q.x0, qs[i].q.y0, qs[i].q.width, qs[i].q.height});
        std::vector<int> of;
        if (merge) {
            of = merge_crops(crops, merged, 8192);
        } else {
            merged = crops;
            of.resize(crops.size());
            for (size_t c = 0; c < crops.size(); ++c) of[c] = (int)c;
        }
        const int base = (int)regions.size();
        const Query &q0 = qs[kv.second[0]];
        const int pb = q0.f.pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
        for (const Rect &r : merged) {
            WorkRegion wr;
            wr.image = static_cast<const uint8_t *>(q0.f.d_pixels) + (int64_t)r.y0 * q0.f.pitch_bytes + (int64_t)r.x0 * pb;
            wr.pitch = q0.f.pitch_bytes;
            wr.H = r.h;
            wr.W = r.w;
            regions.push_back(wr);
            rects.push_back(r);
            frames.push_back(kv.first);
        }
        for (size_t c = 0; c < kv.second.size(); ++c) region_of[kv.second[c]] = base + of[c];
    }
}

// One job per window of each query qs[i], i in idx, over region region_of[i]
// whose frame rectangle is rects[region_of[i]]: its histograms are scored
// against every target of the query.
void query_jobs(const std::vector<Query> &qs, const std::vector<int> &idx, const std::vector<Rect> &rects,
                const std::vector<int> &region_of, std::vector<WorkJob> &jobs)
{
    jobs.clear();
    for (int i : idx) {
        const swih_query &q = qs[i].q;
        const int r = region_of[i];
        const Rect &R = rects[r];
        for (int s = 0; s < q.n_scales; ++s) {
            WorkJob jb;
            jb.region = r;
            jb.kernel = q.kernel;
            jb.w = q.win_w[s];
            jb.h = q.win_h[s];
            jb.cx0 = q.x0 - R.x0 + (jb.w - 1) / 2;
            jb.cy0 = q.y0 - R.y0 + (jb.h - 1) / 2;
            jb.ncx = q.width - jb.w + 1;
            jb.ncy = q.height - jb.h + 1;
            jb.target = q.d_targets;
            jb.map = q.d_out + map_offset(q, 0, s);
            jb.n_targets = q.n_targets;
            jb.target_stride = q.bins;
            jb.map_stride = (int64_t)map_offset(q, 1, 0);  // floats per target
            jobs.push_back(jb);
        }
    }
}

// regions and jobs of a group of queries (indices into qs) in one set
void group_work(const std::vector<Query> &qs, const std::vector<int> &idx, bool merge,
                std::vector<WorkRegion> &regions, std::vector<WorkJob> &jobs)
{
    std::vector<Rect> rects;
    std::vector<int> frames, region_of;
    crop_regions(qs, idx, merge, regions, rects, frames, region_of);
    query_jobs(qs, idx, rects, region_of, jobs);
}

}  // namespace

struct swih_server_s {
    swih_server_desc desc{};
    int device = 0;
    char *d_arena = nullptr;
    char *h_staging = nullptr;
    Arena dev, host;
    std::vector<cudaStream_t> streams;
    std::vector<MicroBatch *> slot;

    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Query> queue;
    std::deque<swih_completion> completions;
    std::vector<swih_frame_desc> frames;
    uint64_t outstanding = 0;
    uint64_t next_id = 1;
    bool stop = false;
    bool mem_blocked = false;
    std::vector<MicroBatch *> zombies;  // failed micro-batches whose callback never ran
    std::thread th;

    // resident integral histograms (keep_ih): the policy, and where each
    // resident (block, region) lives; scheduler thread only
    ResidentCache cache;
    std::map<std::pair<int, int>, WorkRegion> resident_where;
    std::vector<int> pending_invalidate;  // frames whose pixels changed (guarded by mu)
    swih_server_stats stats{};            // guarded by mu

    void run();
    MicroBatch *try_build(const std::vector<Query> &qs, int si, bool &fatal, std::string &err);
    int plan_part(MicroBatch *mb, const std::vector<int> &part, std::string &err);
    bool alloc_dev(uint64_t bytes, uint64_t &off);
    void free_block(int id, uint64_t off, uint64_t bytes);
    void release(MicroBatch *mb);
    void launch(MicroBatch *mb);
    void retire(MicroBatch *mb, std::vector<swih_completion> &out);
};

namespace {

void CUDART_CB on_done(void *p)
{
    MicroBatch *mb = static_cast<MicroBatch *>(p);
    {
        std::lock_guard<std::mutex> lk(mb->srv->mu);
        mb->done = true;
        mb->fired = true;
    }
    mb->srv->cv.notify_all();
}

}  // namespace

void swih_server_s::free_block(int id, uint64_t off, uint64_t bytes)
{
    for (auto it = resident_where.begin(); it != resident_where.end();)
        it = it->first.first == id ? resident_where.erase(it) : std::next(it);
    dev.release(off, bytes);
}

// arena memory, evicting resident integral histograms nobody uses (least
// recently used first) until it fits
bool swih_server_s::alloc_dev(uint64_t bytes, uint64_t &off)
{
    for (;;) {
        if (dev.alloc(bytes, off)) return true;
        uint64_t o = 0, b = 0;
        int id = -1;
        if (!cache.evict_one(o, b, &id)) return false;
        free_block(id, o, b);
    }
}

void swih_server_s::release(MicroBatch *mb)
{
    for (auto &b : mb->dev_blocks) dev.release(b.first, b.second);
    mb->dev_blocks.clear();
    for (auto &b : mb->built) dev.release(b.off, b.bytes);
    mb->built.clear();
    for (int id : mb->held) {
        uint64_t off = 0, bytes = 0;
        if (cache.release(id, off, bytes)) free_block(id, off, bytes);
    }
    mb->held.clear();
    if (mb->host_bytes) host.release(mb->host_off, mb->host_bytes);
    mb->host_bytes = 0;
}

enum { kPartOk = 0, kPartNoRoom = 1, kPartLayout = 2, kPartFail = 3 };

// The work of queries `part` (same pixel type, bit depth, bins and kernel):
// a build set (K1, K2) over the crops whose integral histograms are not
// resident, then a gather set (K3 only) whose regions are all prebuilt: the
// build set's and the resident ones. kPartLayout when the part's term set and
// ring cannot be laid out (the caller splits it), kPartNoRoom when the arena
// is full even after evicting what nobody uses.
int swih_server_s::plan_part(MicroBatch *mb, const std::vector<int> &part, std::string &err)
{
    const std::vector<Query> &qs = mb->queries;
    WorkSpec spec = spec_of(desc, qs[part[0]]);
    for (int i : part)
        for (int k = 0; k < qs[i].q.n_scales; ++k) {
            spec.want_win_w = std::max(spec.want_win_w, qs[i].q.win_w[k]);
            spec.want_win_h = std::max(spec.want_win_h, qs[i].q.win_h[k]);
        }
    // the part's term set and ring: a layout of its crops and jobs in one set
    std::vector<WorkRegion> regions;
    std::vector<WorkJob> jobs;
    std::vector<Rect> rects;
    std::vector<int> frames, region_of;
    crop_regions(qs, part, false, regions, rects, frames, region_of);
    query_jobs(qs, part, rects, region_of, jobs);
    WorkSet dry;
    if (dry.plan(spec, regions, jobs, err) != SWIH_OK) return kPartLayout;
    const Query &q0 = qs[part[0]];
    const std::string tail = "p" + std::to_string(q0.f.pixel_type) + "d" + std::to_string(q0.f.bitdepth);
    const std::string key = dry.signature() + tail;
    // resident hits; their blocks are taken before any allocation, so that
    // making room for this part never evicts what it is about to read
    std::vector<int> hit(qs.size(), -1), miss;
    std::vector<ResidentCache::Entry> hit_entry(qs.size());
    for (int i : part) {
        const Rect c{qs[i].q.x0, qs[i].q.y0, qs[i].q.width, qs[i].q.height};
        hit[i] = desc.keep_ih ? cache.find(qs[i].q.frame, key, c) : -1;
        if (hit[i] < 0) {
            miss.push_back(i);
            continue;
        }
        hit_entry[i] = cache.entry(hit[i]);
        if (std::find(mb->held.begin(), mb->held.end(), hit_entry[i].block) == mb->held.end()) {
            cache.acquire(hit_entry[i].block);
            mb->held.push_back(hit_entry[i].block);
        }
    }
    std::vector<WorkRegion> pre;
    std::vector<Rect> pre_rect;
    std::vector<int> pre_of(qs.size(), -1);
    if (!miss.empty()) {
        std::vector<WorkRegion> br;
        std::vector<Rect> brect;
        std::vector<int> bframe, bof;
        crop_regions(qs, miss, desc.merge_regions != 0, br, brect, bframe, bof);
        std::unique_ptr<WorkSet> bs(new WorkSet());
        if (bs->plan(spec, br, {}, err) != SWIH_OK) return kPartFail;
        if (bs->signature() + tail != key) {
            err = "internal: the build's term set differs from the gather's";
            return kPartFail;
        }
        uint64_t off = 0;
        if (!alloc_dev(bs->bytes(), off)) return kPartNoRoom;
        MicroBatch::Built b;
        b.off = off;
        b.bytes = bs->bytes();
        b.set = (int)mb->sets.size();
        b.frames = bframe;
        b.rects = brect;
        b.key = key;
        mb->built.push_back(b);
        if (bs->bind(d_arena + off, err) != SWIH_OK) return kPartFail;
        const int base = (int)pre.size();
        for (int k = 0; k < (int)br.size(); ++k) {
            pre.push_back(bs->region_as_prebuilt(k));
            pre_rect.push_back(brect[k]);
        }
        for (int i : miss) pre_of[i] = base + bof[i];
        mb->sets.push_back(std::move(bs));
        mb->set_queries.push_back(miss);
    }
    std::map<std::pair<int, int>, int> entry_region;  // (block, region) -> gather-set region
    for (int i : part) {
        if (hit[i] < 0) continue;
        const ResidentCache::Entry &E = hit_entry[i];
        const std::pair<int, int> at{E.block, E.region};
        if (!entry_region.count(at)) {
            entry_region[at] = (int)pre.size();
            pre.push_back(resident_where.at(at));
            pre_rect.push_back(E.rect);
        }
        pre_of[i] = entry_region[at];
        mb->reused[i] = 1;
    }
    std::vector<WorkJob> gj;
    query_jobs(qs, part, pre_rect, pre_of, gj);
    std::unique_ptr<WorkSet> gs(new WorkSet());
    if (gs->plan(spec, pre, gj, err) != SWIH_OK) return kPartFail;
    uint64_t off = 0;
    if (!alloc_dev(gs->bytes(), off)) return kPartNoRoom;
    mb->dev_blocks.push_back({off, gs->bytes()});
    if (gs->bind(d_arena + off, err) != SWIH_OK) return kPartFail;
    mb->sets.push_back(std::move(gs));
    mb->set_queries.push_back(part);
    return kPartOk;
}

// Lay out the micro-batch of queries qs and take its memory; nullptr when the
// memory is not free now (fatal = false) or the work cannot be built (fatal).
MicroBatch *swih_server_s::try_build(const std::vector<Query> &qs, int si, bool &fatal, std::string &err)
{
    fatal = false;
    std::unique_ptr<MicroBatch> mb(new MicroBatch());
    mb->srv = this;
    mb->slot = si;
    mb->queries = qs;
    mb->reused.assign(qs.size(), 0);
    // groups: queries that can share integral histograms
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < (int)qs.size(); ++i)
        groups[std::make_tuple(qs[i].f.pixel_type, qs[i].f.bitdepth, qs[i].q.bins, qs[i].q.kernel)].push_back(i);
    for (auto &kv : groups) {
        // a group whose combined windows leave the exact ring (the largest
        // window of one query with the largest of another) runs one part per query
        int r = plan_part(mb.get(), kv.second, err);
        if (r == kPartLayout && kv.second.size() > 1) {
            r = kPartOk;
            for (int i : kv.second) {
                r = plan_part(mb.get(), {i}, err);
                if (r != kPartOk) break;
            }
        }
        if (r != kPartOk) {
            release(mb.get());
            fatal = r != kPartNoRoom;
            return nullptr;
        }
    }
    // one staging block for the tables and the status words
    uint64_t staging = 0;
    for (auto &ws : mb->sets) staging += Arena::granules(ws->tables_bytes());
    staging += Arena::granules(sizeof(uint32_t) * mb->sets.size());
    if (!host.alloc(staging, mb->host_off)) {
        release(mb.get());
        return nullptr;
    }
    mb->host_bytes = staging;
    return mb.release();
}

void swih_server_s::launch(MicroBatch *mb)
{
    cudaStream_t s = streams[mb->slot];
    char *stage = h_staging + mb->host_off;
    uint64_t o = 0;
    cudaError_t e = cudaSuccess;
    for (auto &ws : mb->sets) {
        std::memcpy(stage + o, ws->tables(), ws->tables_bytes());
        e = cudaMemcpyAsync(ws->tables_device(), stage + o, ws->tables_bytes(), cudaMemcpyHostToDevice, s);
        o += Arena::granules(ws->tables_bytes());
        if (e != cudaSuccess) break;
    }
    mb->h_status = reinterpret_cast<uint32_t *>(stage + o);
    for (size_t i = 0; i < mb->sets.size(); ++i) mb->h_status[i] = 0;
    const uint64_t t0 = now_ns();
    for (auto &q : mb->queries) q.start_ns = t0;
    for (size_t i = 0; i < mb->sets.size() && e == cudaSuccess; ++i) {
        e = mb->sets[i]->enqueue(s, true);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&mb->h_status[i], mb->sets[i]->status_device(), sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mb->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(mb->ev, s);
    if (e == cudaSuccess) {
        e = cudaLaunchHostFunc(s, on_done, mb);
        mb->hostfn = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        // nothing more is enqueued: finish the micro-batch once its stream drains
        cudaGetLastError();
        mb->launch_status = SWIH_ERR_CUDA;
        cudaStreamSynchronize(s);
        std::lock_guard<std::mutex> lk(mu);
        mb->done = true;
    }
}

void swih_server_s::retire(MicroBatch *mb, std::vector<swih_completion> &out)
{
    const uint64_t t = now_ns();
    std::vector<int32_t> st(mb->queries.size(), mb->launch_status);
    if (mb->launch_status == SWIH_OK)
        for (size_t i = 0; i < mb->sets.size(); ++i)
            if (mb->h_status[i] & kStatusTimeout)
                for (int qi : mb->set_queries[i]) st[qi] = SWIH_ERR_TIMEOUT;
    for (size_t i = 0; i < mb->queries.size(); ++i) {
        swih_completion c;
        c.id = mb->queries[i].id;
        c.user_tag = mb->queries[i].q.user_tag;
        c.status = st[i];
        c.batch_queries = (int32_t)mb->queries.size();
        c.submit_ns = mb->queries[i].submit_ns;
        c.start_ns = mb->queries[i].start_ns;
        c.done_ns = t;
        c.ih_reused = mb->reused[i];
        c.reserved = 0;
        out.push_back(c);
    }
    if (mb->hostfn && !mb->fired) {
        // failed through its event while its callback is still enqueued: the
        // stream may yet touch its memory and the callback its object, so both
        // are kept until the server is destroyed
        zombies.push_back(mb);
        return;
    }
    if (mb->ev) cudaEventDestroy(mb->ev);
    // integral histograms built without error stay resident (keep_ih) until
    // their memory is needed or their frame changes
    for (auto &b : mb->built) {
        const bool ok = mb->launch_status == SWIH_OK && !(mb->h_status[b.set] & kStatusTimeout);
        if (!desc.keep_ih || !ok) {
            dev.release(b.off, b.bytes);
            continue;
        }
        const int id = cache.add_block(b.off, b.bytes);
        for (int k = 0; k < (int)b.rects.size(); ++k) {
            cache.add_entry(id, b.frames[k], b.rects[k], b.key, k);
            resident_where[{id, k}] = mb->sets[b.set]->region_as_prebuilt(k);
        }
    }
    uint64_t n_built = 0, n_reused = 0;
    for (auto &b : mb->built) n_built += b.rects.size();
    for (char r : mb->reused) n_reused += r ? 1 : 0;
    mb->built.clear();
    release(mb);
    {
        std::lock_guard<std::mutex> lk(mu);
        stats.queries += mb->queries.size();
        stats.ih_reused += n_reused;
        stats.regions_built += n_built;
        stats.evictions = cache.evictions();
        stats.resident_bytes = cache.resident_bytes();
    }
    delete mb;
}

void swih_server_s::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        auto any_done = [&] {
            for (MicroBatch *mb : slot)
                if (mb && mb->done) return true;
            return false;
        };
        auto free_slot = [&] {
            for (size_t i = 0; i < slot.size(); ++i)
                if (!slot[i]) return (int)i;
            return -1;
        };
        auto idle = [&] {
            for (MicroBatch *mb : slot)
                if (mb) return false;
            return true;
        };
        const bool woke = cv.wait_for(lk, std::chrono::milliseconds(20), [&] {
            return any_done() || (!mem_blocked && !queue.empty() && free_slot() >= 0) || !pending_invalidate.empty() ||
                   (stop && queue.empty() && idle());
        });
        if (stop && queue.empty() && idle()) break;
        if (!woke) {
            // nothing new for a while: a micro-batch whose stream hit a CUDA
            // error never runs its completion callback; its event reports it
            std::vector<MicroBatch *> running;
            for (MicroBatch *mb : slot)
                if (mb && !mb->done && mb->ev) running.push_back(mb);
            lk.unlock();
            std::vector<MicroBatch *> failed_mb;
            for (MicroBatch *mb : running) {
                const cudaError_t e = cudaEventQuery(mb->ev);
                if (e != cudaSuccess && e != cudaErrorNotReady) failed_mb.push_back(mb);
            }
            lk.lock();
            for (MicroBatch *mb : failed_mb) {
                mb->launch_status = SWIH_ERR_CUDA;
                mb->done = true;
            }
            if (failed_mb.empty()) continue;
        }
        // retire finished micro-batches
        std::vector<MicroBatch *> fin;
        for (auto &mb : slot)
            if (mb && mb->done) {
                fin.push_back(mb);
                mb = nullptr;
            }
        if (!fin.empty()) {
            lk.unlock();
            std::vector<swih_completion> out;
            for (MicroBatch *mb : fin) retire(mb, out);
            lk.lock();
            for (auto &c : out) completions.push_back(c);
            outstanding -= out.size();
            mem_blocked = false;
            cv_done.notify_all();
        }
        // frames whose pixels changed: their resident integral histograms go
        // before anything newer is admitted
        if (!pending_invalidate.empty()) {
            std::vector<int> frames;
            frames.swap(pending_invalidate);
            lk.unlock();
            for (int f : frames) {
                std::vector<std::pair<uint64_t, uint64_t>> blocks;
                std::vector<int> ids;
                cache.invalidate_frame(f, blocks, &ids);
                for (size_t k = 0; k < ids.size(); ++k) free_block(ids[k], blocks[k].first, blocks[k].second);
            }
            lk.lock();
            stats.resident_bytes = cache.resident_bytes();
            mem_blocked = false;
        }
        // admit, oldest first
        int si;
        while (!mem_blocked && !queue.empty() && (si = free_slot()) >= 0) {
            const size_t k = std::min<size_t>((size_t)std::max(1, desc.max_batch_queries), queue.size());
            for (size_t i = 0; i < k; ++i) queue[i].admitting = true;  // cancel leaves these alone
            std::vector<Query> cand(queue.begin(), queue.begin() + (long)k);
            lk.unlock();
            MicroBatch *mb = nullptr;
            size_t take = k;
            bool fatal = false;
            std::string err;
            for (;;) {
                std::vector<Query> part(cand.begin(), cand.begin() + (long)take);
                mb = try_build(part, si, fatal, err);
                if (mb || fatal || take == 1) break;
                take = (take + 1) / 2;
            }
            std::vector<swih_completion> failed;
            if (!mb && fatal) {
                // a query whose work cannot be laid out: fail it, keep serving
                swih_completion c;
                c.id = cand[0].id;
                c.user_tag = cand[0].q.user_tag;
                c.status = SWIH_ERR_UNSUPPORTED;
                c.batch_queries = 1;
                c.submit_ns = cand[0].submit_ns;
                c.start_ns = c.done_ns = now_ns();
                failed.push_back(c);
                take = 1;
            }
            lk.lock();
            // the candidates are still the queue's first k entries: cancel skips
            // them and submissions only append
            for (size_t i = 0; i < k; ++i) queue[i].admitting = false;
            if (!mb && !fatal) {
                if (take > 1 || !idle()) {
                    mem_blocked = true;  // wait for a retirement
                    break;
                }
                // one query, nothing running, and still no room (staging too
                // small for its tables): it can never run
                swih_completion c;
                c.id = cand[0].id;
                c.user_tag = cand[0].q.user_tag;
                c.status = SWIH_ERR_BUDGET;
                c.batch_queries = 1;
                c.submit_ns = cand[0].submit_ns;
                c.start_ns = c.done_ns = now_ns();
                failed.push_back(c);
            }
            for (size_t i = 0; i < take; ++i) queue.pop_front();
            if (!mb) {
                for (auto &c : failed) completions.push_back(c);
                outstanding -= failed.size();
                cv_done.notify_all();
                continue;
            }
            slot[si] = mb;
            lk.unlock();
            launch(mb);
            lk.lock();
        }
    }
}

extern "C" {

swih_status swih_query_out_elems(const swih_query *q, uint64_t *elems)
{
    if (!elems) return sfail(SWIH_ERR_INVALID_ARG, "elems is NULL");
    const swih_status st = check_query(q, nullptr);
    if (st != SWIH_OK) return st;
    *elems = map_offset(*q, q->n_targets, 0);
    return SWIH_OK;
}

swih_status swih_server_create(const swih_server_desc *desc, swih_server_t *out)
{
    if (!out) return sfail(SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return sfail(SWIH_ERR_INVALID_ARG, "desc is NULL");
    if (desc->hbm_budget_bytes < (1u << 20)) return sfail(SWIH_ERR_INVALID_ARG, "hbm_budget_bytes below 1 MiB");
    if (desc->max_inflight < 1 || desc->max_inflight > 32)
        return sfail(SWIH_ERR_INVALID_ARG, "max_inflight must be in [1, 32]");
    if (desc->max_batch_queries < 1) return sfail(SWIH_ERR_INVALID_ARG, "max_batch_queries must be >= 1");
    if (desc->gauss_degree < 0 || desc->gauss_degree > 2)
        return sfail(SWIH_ERR_UNSUPPORTED, "gauss_degree must be 0 (default), 1 or 2");
    std::unique_ptr<swih_server_s> S(new swih_server_s());
    S->desc = *desc;
    if (!S->desc.staging_bytes) S->desc.staging_bytes = 64ull << 20;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->d_arena), S->desc.hbm_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(nullptr, "cudaMalloc(server arena)", e);
    }
    e = cudaMallocHost(reinterpret_cast<void **>(&S->h_staging), S->desc.staging_bytes);
    if (e != cudaSuccess) {
        cudaFree(S->d_arena);
        return cuda_fail(nullptr, "cudaMallocHost(server staging)", e);
    }
    S->dev.reset(S->desc.hbm_budget_bytes);
    S->host.reset(S->desc.staging_bytes);
    S->streams.resize(S->desc.max_inflight, nullptr);
    S->slot.assign(S->desc.max_inflight, nullptr);
    for (auto &s : S->streams) {
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto &s2 : S->streams)
                if (s2) cudaStreamDestroy(s2);
            cudaFree(S->d_arena);
            cudaFreeHost(S->h_staging);
            return cuda_fail(nullptr, "cudaStreamCreate", e);
        }
    }
    swih_server_s *raw = S.release();
    raw->th = std::thread([raw] { raw->run(); });
    *out = raw;
    return SWIH_OK;
}

swih_status swih_server_add_frame(swih_server_t S, const swih_frame_desc *f, int32_t *frame_id)
{
    if (!S || !f || !frame_id) return sfail(SWIH_ERR_INVALID_ARG, "server, frame and frame_id are required");
    if (!f->d_pixels) return sfail(SWIH_ERR_INVALID_ARG, "d_pixels is NULL");
    if (f->pixel_type != SWIH_PIXEL_U8 && f->pixel_type != SWIH_PIXEL_U16)
        return sfail(SWIH_ERR_INVALID_ARG, "pixel_type must be U8 or U16");
    const int pb = f->pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    if (f->height < 3 || f->width < 3) return sfail(SWIH_ERR_INVALID_ARG, "frame must be at least 3 x 3");
    if (f->pitch_bytes < (int64_t)f->width * pb) return sfail(SWIH_ERR_INVALID_ARG, "pitch_bytes smaller than a row");
    if (pb == 2 && ((f->pitch_bytes & 1) || (reinterpret_cast<uintptr_t>(f->d_pixels) & 1)))
        return sfail(SWIH_ERR_INVALID_ARG, "16-bit frames need an even pitch and address");
    if (f->bitdepth < 1 || f->bitdepth > 8 * pb) return sfail(SWIH_ERR_INVALID_ARG, "bitdepth out of range");
    std::lock_guard<std::mutex> lk(S->mu);
    *frame_id = (int32_t)S->frames.size();
    S->frames.push_back(*f);
    return SWIH_OK;
}

swih_status swih_server_query_bytes(swih_server_t S, const swih_query *q, uint64_t *bytes)
{
    if (!S || !bytes) return sfail(SWIH_ERR_INVALID_ARG, "server and bytes are required");
    swih_frame_desc f;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!q || q->frame < 0 || q->frame >= (int)S->frames.size()) return sfail(SWIH_ERR_INVALID_ARG, "no such frame");
        f = S->frames[q->frame];
    }
    swih_status st = check_query(q, &f);
    if (st != SWIH_OK) return st;
    Query qr;
    qr.q = *q;
    qr.f = f;
    if (!qr.q.d_targets) qr.q.d_targets = reinterpret_cast<const float *>(256);
    if (!qr.q.d_out) qr.q.d_out = reinterpret_cast<float *>(256);
    std::vector<Query> one{qr};
    std::vector<WorkRegion> regions;
    std::vector<WorkJob> jobs;
    group_work(one, {0}, false, regions, jobs);
    WorkSet ws;
    std::string err;
    st = ws.plan(spec_of(S->desc, qr), regions, jobs, err);
    if (st != SWIH_OK) return sfail(st, err);
    *bytes = ws.bytes();
    return SWIH_OK;
}

swih_status swih_server_submit(swih_server_t S, const swih_query *q, uint64_t *id)
{
    if (!S) return sfail(SWIH_ERR_INVALID_ARG, "server is NULL");
    if (!q || !q->d_targets || !q->d_out) return sfail(SWIH_ERR_INVALID_ARG, "query, d_targets and d_out are required");
    uint64_t need = 0;
    swih_status st = swih_server_query_bytes(S, q, &need);
    if (st != SWIH_OK) return st;
    if (need > S->dev.size()) {
        char m[160];
        std::snprintf(m, sizeof m, "query needs %llu bytes of work memory, the arena holds %llu",
                      (unsigned long long)need, (unsigned long long)S->dev.size());
        return sfail(SWIH_ERR_BUDGET, m);
    }
    Query qr;
    qr.q = *q;
    qr.submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return sfail(SWIH_ERR_INVALID_ARG, "server is stopping");
        qr.f = S->frames[q->frame];
        qr.id = S->next_id++;
        S->queue.push_back(qr);
        ++S->outstanding;
    }
    S->cv.notify_all();
    if (id) *id = qr.id;
    return SWIH_OK;
}

swih_status swih_server_poll(swih_server_t S, swih_completion *out, int32_t max, int32_t *n, int32_t wait_us)
{
    if (!S || !n || (max > 0 && !out)) return sfail(SWIH_ERR_INVALID_ARG, "server, out and n are required");
    *n = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->completions.empty() && wait_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !S->completions.empty(); });
    while (*n < max && !S->completions.empty()) {
        out[(*n)++] = S->completions.front();
        S->completions.pop_front();
    }
    return SWIH_OK;
}

swih_status swih_server_cancel(swih_server_t S, uint64_t id)
{
    if (!S) return sfail(SWIH_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
            if (it->id != id) continue;
            if (it->admitting) return sfail(SWIH_ERR_INVALID_ARG, "query is being admitted");
            swih_completion c;
            c.id = it->id;
            c.user_tag = it->q.user_tag;
            c.status = SWIH_ERR_CANCELLED;
            c.batch_queries = 0;
            c.submit_ns = it->submit_ns;
            c.start_ns = c.done_ns = now_ns();
            S->queue.erase(it);
            S->completions.push_back(c);
            --S->outstanding;
            S->cv_done.notify_all();
            return SWIH_OK;
        }
    }
    return sfail(SWIH_ERR_INVALID_ARG, "query " + std::to_string(id) + " is not waiting for admission");
}

swih_status swih_server_frame_changed(swih_server_t S, int32_t frame_id)
{
    if (!S) return sfail(SWIH_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (frame_id < 0 || frame_id >= (int)S->frames.size()) return sfail(SWIH_ERR_INVALID_ARG, "no such frame");
        S->pending_invalidate.push_back(frame_id);
    }
    S->cv.notify_all();
    return SWIH_OK;
}

swih_status swih_server_get_stats(swih_server_t S, swih_server_stats *out)
{
    if (!S || !out) return sfail(SWIH_ERR_INVALID_ARG, "server and out are required");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return SWIH_OK;
}

swih_status swih_server_drain(swih_server_t S)
{
    if (!S) return sfail(SWIH_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->outstanding == 0; });
    return SWIH_OK;
}

swih_status swih_server_destroy(swih_server_t S)
{
    if (!S) return SWIH_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    if (!S->zombies.empty()) {
        // a stream failed with work still enqueued: the context is unusable and
        // that work may never finish, so its memory and objects are left alone
        thread_error() = "server destroyed after a CUDA error; its device memory was not freed";
        return SWIH_ERR_CUDA;
    }
    for (auto &s : S->streams)
        if (s) cudaStreamDestroy(s);
    cudaError_t e = cudaFree(S->d_arena);
    cudaFreeHost(S->h_staging);
    delete S;
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaFree", e);
    return SWIH_OK;
}

}  // extern "C"
