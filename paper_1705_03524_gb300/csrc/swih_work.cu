// Work sets: many image regions and likelihood jobs laid out in one block of
// device memory and run by three table-driven launches (K1 and K2 over every
// region, K3 once per group of jobs sharing a kernel and fitted degrees).
// Used by the batch API and by the server. Host code only.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "swih_host.h"

namespace swih {

namespace {

constexpr uint64_t kStatusBytes = 256;

uint64_t align256(uint64_t v) { return (v + 255) / 256 * 256; }

}  // namespace

swih_status WorkSet::plan(const WorkSpec &spec, const std::vector<WorkRegion> &regions,
                          const std::vector<WorkJob> &jobs, std::string &err)
{
    auto bad = [&](swih_status st, const std::string &m) {
        err = m;
        return st;
    };
    if (regions.empty()) return bad(SWIH_ERR_INVALID_ARG, "no regions");
    if (regions.size() > (1u << 20)) return bad(SWIH_ERR_UNSUPPORTED, "more than 2^20 regions");
    if (spec.band_rows < 0) return bad(SWIH_ERR_INVALID_ARG, "band_rows must be >= 0");
    const int pb = spec.pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    int maxH = 3, maxW = 3, mw = 3, mh = 3;
    for (size_t i = 0; i < regions.size(); ++i) {
        const WorkRegion &r = regions[i];
        const std::string tag = "region " + std::to_string(i);
        if (r.H < 3 || r.W < 3) return bad(SWIH_ERR_INVALID_ARG, tag + " must be at least 3 x 3");
        if (r.pre_ih) {
            if (r.pre_ih_pitch < r.W || r.pre_plane < (int64_t)r.H * r.pre_ih_pitch || (r.pre_ih_pitch & 31))
                return bad(SWIH_ERR_INVALID_ARG, tag + ": prebuilt layout too small");
            maxH = std::max(maxH, r.H);
            maxW = std::max(maxW, r.W);
            continue;
        }
        if (!r.image) return bad(SWIH_ERR_INVALID_ARG, tag + ": image is NULL");
        if (r.pitch < (int64_t)r.W * pb) return bad(SWIH_ERR_INVALID_ARG, tag + ": pitch smaller than a row");
        if (pb == 2 && ((r.pitch & 1) || (reinterpret_cast<uintptr_t>(r.image) & 1)))
            return bad(SWIH_ERR_INVALID_ARG, tag + ": 16-bit pixels need an even pitch and address");
        maxH = std::max(maxH, r.H);
        maxW = std::max(maxW, r.W);
    }
    for (size_t j = 0; j < jobs.size(); ++j) {
        const WorkJob &jb = jobs[j];
        const std::string tag = "job " + std::to_string(j);
        if (jb.region < 0 || jb.region >= (int)regions.size()) return bad(SWIH_ERR_INVALID_ARG, tag + ": no such region");
        const WorkRegion &r = regions[jb.region];
        if (jb.kernel < SWIH_KERNEL_PLAIN || jb.kernel > SWIH_KERNEL_GAUSSIAN ||
            !(spec.kernel_mask & SWIH_KERNEL_BIT(jb.kernel)))
            return bad(SWIH_ERR_INVALID_ARG, tag + ": kernel not in kernel_mask");
        if (!odd_window(jb.w) || !odd_window(jb.h) || jb.w > r.W || jb.h > r.H)
            return bad(SWIH_ERR_INVALID_ARG, tag + ": window sides must be odd, >= 3 and fit the region");
        if (!jb.target || !jb.map) return bad(SWIH_ERR_INVALID_ARG, tag + ": target or map is NULL");
        if (jb.n_targets < 1 || jb.n_targets > kMaxTargets)
            return bad(SWIH_ERR_INVALID_ARG, tag + ": n_targets out of range");
        if (jb.n_targets > 1 && (jb.target_stride < spec.bins || jb.map_stride < 1))
            return bad(SWIH_ERR_INVALID_ARG, tag + ": target or map stride too small");
        const int rx = (jb.w - 1) / 2, ry = (jb.h - 1) / 2;
        if (jb.ncx == 0 && jb.ncy == 0) {
            // whole valid rectangle
        } else if (jb.ncx < 1 || jb.ncy < 1 || jb.cx0 < rx || jb.cy0 < ry ||
                   (int64_t)jb.cx0 + jb.ncx > r.W - rx || (int64_t)jb.cy0 + jb.ncy > r.H - ry) {
            return bad(SWIH_ERR_INVALID_ARG, tag + ": centre rectangle leaves the valid centres");
        }
        mw = std::max(mw, jb.w);
        mh = std::max(mh, jb.h);
    }
    spec_ = spec;
    in_jobs_ = jobs;
    for (auto &jb : in_jobs_)
        if (jb.ncx == 0 && jb.ncy == 0) {
            const WorkRegion &r = regions[jb.region];
            jb.cx0 = (jb.w - 1) / 2;
            jb.cy0 = (jb.h - 1) / 2;
            jb.ncx = r.W - jb.w + 1;
            jb.ncy = r.H - jb.h + 1;
        }
    n_centres_ = 0;
    for (auto &jb : in_jobs_) n_centres_ += (uint64_t)jb.ncx * jb.ncy * (uint64_t)jb.n_targets;

    // template: term set, ring and scan launch shape for the largest region and window
    swih_plan_desc pd;
    std::memset(&pd, 0, sizeof pd);
    pd.height = maxH;
    pd.width = maxW;
    pd.pitch_bytes = (int64_t)maxW * pb;
    pd.pixel_type = spec.pixel_type;
    pd.bitdepth = spec.bitdepth;
    pd.bins = spec.bins;
    pd.kernel_mask = spec.kernel_mask;
    pd.gauss_degree = spec.gauss_degree;
    pd.gauss_sigma_frac = spec.gauss_sigma_frac;
    pd.max_win_w = std::min(maxW, std::max(mw, spec.want_win_w));
    pd.max_win_h = std::min(maxH, std::max(mh, spec.want_win_h));
    if (pd.max_win_w % 2 == 0) --pd.max_win_w;
    if (pd.max_win_h % 2 == 0) --pd.max_win_h;
    pd.max_win_w = std::max(pd.max_win_w, mw);
    pd.max_win_h = std::max(pd.max_win_h, mh);
    pd.precision = spec.precision;
    tmpl_ = swih_plan_s();
    const swih_status st = build_layout(&pd, &tmpl_);
    if (st != SWIH_OK) return bad(st, thread_error());
    if (tmpl_.elem_bytes > 8 || (tmpl_.desc.kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_GAUSSIAN) &&
                                 (gauss_is_wide(&tmpl_, pd.max_win_w, pd.max_win_h))))
        return bad(SWIH_ERR_UNSUPPORTED, "batches, the server and streamed frames serve the Gaussian up to degree 2 "
                                         "in the 64-bit ring (use a plan for larger windows or degrees)");
    scan_E_ = tmpl_.scan_E;
    scan_threads_ = tmpl_.scan_threads;
    band_rows_ = spec.band_rows > 0 ? spec.band_rows : 32;

    // memory: status | scan flags + ticket | tables | per region: bins, IH, scan state
    const uint64_t es = (uint64_t)tmpl_.elem_bytes;
    const uint64_t n_chains = (uint64_t)spec.bins * tmpl_.n_q;
    const size_t nR = regions.size(), nJ = in_jobs_.size();
    regions_.assign(nR, Region());
    built_.clear();
    long long ticket = 0, chunk = 0;
    uint64_t flag_ints = 0;
    for (size_t i = 0; i < nR; ++i) {
        Region &R = regions_[i];
        R.in = regions[i];
        if (R.in.pre_ih) {  // read in place: no bins, scan state or tickets here
            R.prebuilt = true;
            R.ih_pitch = R.in.pre_ih_pitch;
            R.plane = R.in.pre_plane;
            continue;
        }
        built_.push_back((int)i);
        R.n_bands = (R.in.H + band_rows_ - 1) / band_rows_;
        R.bins_pitch = round_up(R.in.W, 128);
        R.ih_pitch = round_up(R.in.W, 32);
        R.plane = (int64_t)R.in.H * R.ih_pitch;
        R.off_flags = flag_ints;
        flag_ints += n_chains * R.n_bands;
        R.ticket0 = (int)ticket;
        ticket += (long long)(n_chains * R.n_bands);
        R.chunk0 = chunk;
        chunk += (long long)((R.in.W + 15) / 16) * R.in.H;
        if (ticket > (1LL << 30)) return bad(SWIH_ERR_UNSUPPORTED, "too many scan tiles in one work set");
    }
    scan_tiles_ = ticket;
    quant_chunks_ = chunk;
    flags_ints_ = flag_ints + 1;  // + the ticket counter
    tab_quant_ = 0;
    tab_scan_ = align256(tab_quant_ + sizeof(QuantRoi) * nR);
    tab_jobs_ = align256(tab_scan_ + sizeof(ScanRoi) * nR);
    tab_items_ = align256(tab_jobs_ + sizeof(GatherParams) * nJ);
    const uint64_t tables = align256(tab_items_ + sizeof(int) * (2 * nJ + 1));
    off_status_ = 0;
    off_flags_ = kStatusBytes;  // directly after the status word: one memset clears both
    off_tables_ = align256(off_flags_ + flags_ints_ * sizeof(int));
    uint64_t off = off_tables_ + tables;
    // rows that hold no pixel of a bin are not stored (bands of at most 64 rows,
    // regions below 32768 rows: the gathers keep stored rows as int16)
    sparse_ = band_rows_ <= 64;
    for (const auto &R : regions_) sparse_ = sparse_ && (R.prebuilt || R.in.H <= 32767);
    for (auto &R : regions_) {
        if (R.prebuilt) continue;
        R.off_bins = off;
        off = align256(off + (uint64_t)R.in.H * R.bins_pitch);
        R.off_ih = off;
        off = align256(off + (uint64_t)tmpl_.n_terms * spec.bins * R.plane * es);
        R.off_agg = off;
        off = align256(off + n_chains * R.n_bands * R.ih_pitch * es);
        R.off_incl = off;
        off = align256(off + n_chains * R.n_bands * R.ih_pitch * es);
        if (sparse_) {
            R.off_occ = off;
            off = align256(off + (uint64_t)spec.bins * R.n_bands * sizeof(unsigned long long));
            R.off_row_map = off;
            off = align256(off + (uint64_t)spec.bins * R.in.H * sizeof(int));
        }
    }
    total_ = off;
    d_mem_ = nullptr;
    groups_.clear();
    return SWIH_OK;
}

swih_status WorkSet::bind(char *d_mem, std::string &err)
{
    if (!d_mem || (reinterpret_cast<uintptr_t>(d_mem) & 255)) {
        err = "work set memory must be 256-byte aligned";
        return SWIH_ERR_INVALID_ARG;
    }
    d_mem_ = d_mem;
    return rebuild(err);
}

void WorkSet::set_group_want(int g, int tx, int stages, int bb)
{
    groups_[g].want_tx = tx;
    groups_[g].want_stages = stages;
    groups_[g].want_bb = bb;
}

void WorkSet::group_want(int g, int &tx, int &stages, int &bb) const
{
    tx = groups_[g].want_tx;
    stages = groups_[g].want_stages;
    bb = groups_[g].want_bb;
}

swih_status WorkSet::rebuild(std::string &err)
{
    const swih_status st = build_jobs(err);
    if (st != SWIH_OK) return st;
    build_blob();
    return SWIH_OK;
}

swih_status WorkSet::build_jobs(std::string &err)
{
    std::vector<GatherParams> jobs;
    std::vector<int> kinds;
    jobs.reserve(in_jobs_.size());
    for (size_t j = 0; j < in_jobs_.size(); ++j) {
        const WorkJob &jb = in_jobs_[j];
        const Region &R = regions_[jb.region];
        swih_plan_s view = tmpl_;  // term indices, ring and Gaussian settings, over this region
        view.desc.height = R.in.H;
        view.desc.width = R.in.W;
        view.plane = R.plane;
        view.ih_pitch = R.ih_pitch;
        view.d_mem = R.prebuilt ? static_cast<char *>(const_cast<void *>(R.in.pre_ih)) : d_mem_ + R.off_ih;
        view.off_ih = 0;
        view.d_status = status_device();
        GatherParams g;
        int kind = 0;
        const swih_status st = make_gather(&view, jb.kernel, jb.w, jb.h, g, kind);
        if (st != SWIH_OK) {
            err = "job " + std::to_string(j) + ": " + view.err;
            return st;
        }
        g.cx0 = jb.cx0;
        g.cy0 = jb.cy0;
        g.ncx = jb.ncx;
        g.ncy = jb.ncy;
        g.target = jb.target;
        g.map = jb.map;
        g.hist = nullptr;
        g.row_map = R.prebuilt ? R.in.pre_row_map
                    : sparse_  ? reinterpret_cast<const int *>(d_mem_ + R.off_row_map)
                               : nullptr;
        g.nbg = 1;  // table launches span many waves already; no split-gather scratch here
        // bytes the tiled gathers request, one counter per kind in the status block
        g.load_bytes = reinterpret_cast<unsigned long long *>(d_mem_ + off_status_) + 1 + kind;
        g.partial = nullptr;
        g.partial_cap = 0;
        g.n_targets = jb.n_targets;
        g.target_stride = jb.n_targets > 1 ? jb.target_stride : spec_.bins;
        g.map_stride = jb.n_targets > 1 ? jb.map_stride : 0;
        jobs.push_back(g);
        kinds.push_back(kind);
    }
    // group by (kind, fitted degrees), keeping each group's launch-shape wants
    const std::vector<Group> old = groups_;
    groups_.clear();
    jobs_.clear();
    std::vector<int> order(jobs.size());
    for (size_t j = 0; j < jobs.size(); ++j) order[j] = (int)j;
    auto key = [&](int j) { return kinds[j] * 16 + jobs[j].gdx * 4 + jobs[j].gdy; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
    for (int j : order) {
        const GatherParams &g = jobs[j];
        if (groups_.empty() || groups_.back().kind != kinds[j] || groups_.back().gdx != g.gdx ||
            groups_.back().gdy != g.gdy) {
            Group G;
            G.kind = kinds[j];
            G.gdx = g.gdx;
            G.gdy = g.gdy;
            G.job_begin = G.job_end = (int)jobs_.size();
            for (const Group &o : old)
                if (o.kind == G.kind && o.gdx == G.gdx && o.gdy == G.gdy) {
                    G.want_tx = o.want_tx;
                    G.want_stages = o.want_stages;
                    G.want_bb = o.want_bb;
                }
            groups_.push_back(G);
        }
        jobs_.push_back(g);
        groups_.back().job_end = (int)jobs_.size();
    }
    // launch shape and work items per group
    items_.clear();
    for (Group &G : groups_) {
        int max_w = 3, max_t = 1, max_h = 3;
        for (int j = G.job_begin; j < G.job_end; ++j) {
            max_w = std::max(max_w, 2 * jobs_[j].rx + 1);
            max_t = std::max(max_t, jobs_[j].n_targets);
            max_h = std::max(max_h, jobs_[j].H);
        }
        const GatherParams &g0 = jobs_[G.job_begin];
        // regions taller than the tiled gather's row range take the direct gather
        G.tiled = max_h <= kTiledMaxRows &&
                  tiled_shape(G.kind, tmpl_.elem_bytes, G.gdx, G.gdy, max_w, spec_.bins, g0.nl, max_t, G.want_tx,
                              G.want_stages, G.want_bb, true, &G.shape) == cudaSuccess;
        G.items_off = (int)items_.size();
        long long items = 0;
        for (int j = G.job_begin; j < G.job_end; ++j) {
            items_.push_back((int)items);
            if (G.tiled) items += tiled_items(&jobs_[j], G.shape);
            if (items > (1LL << 30)) {
                err = "too many gather work items in one work set";
                return SWIH_ERR_UNSUPPORTED;
            }
        }
        items_.push_back((int)items);
        G.n_items = (int)items;
    }
    return SWIH_OK;
}

void WorkSet::build_blob()
{
    const size_t nR = regions_.size();
    blob_.assign(tab_items_ + sizeof(int) * (2 * jobs_.size() + 1), 0);
    QuantRoi *qt = reinterpret_cast<QuantRoi *>(blob_.data() + tab_quant_);
    ScanRoi *stt = reinterpret_cast<ScanRoi *>(blob_.data() + tab_scan_);
    int *flags = reinterpret_cast<int *>(d_mem_ + off_flags_);
    (void)nR;
    for (size_t i = 0; i < built_.size(); ++i) {  // quantisation and scan tables: the regions built here
        const Region &R = regions_[built_[i]];
        qt[i].image = static_cast<const uint8_t *>(R.in.image);
        qt[i].pitch = R.in.pitch;
        qt[i].H = R.in.H;
        qt[i].W = R.in.W;
        qt[i].bins = reinterpret_cast<uint8_t *>(d_mem_ + R.off_bins);
        qt[i].bins_pitch = R.bins_pitch;
        qt[i].chunk0 = R.chunk0;
        qt[i].vec = (R.in.pitch % 16 == 0) && (reinterpret_cast<uintptr_t>(R.in.image) % 16 == 0);
        stt[i].bins = qt[i].bins;
        stt[i].bins_pitch = R.bins_pitch;
        stt[i].ih = d_mem_ + R.off_ih;
        stt[i].ih_pitch = R.ih_pitch;
        stt[i].plane = R.plane;
        stt[i].agg = d_mem_ + R.off_agg;
        stt[i].incl = d_mem_ + R.off_incl;
        stt[i].flags = flags + R.off_flags;
        stt[i].H = R.in.H;
        stt[i].W = R.in.W;
        stt[i].n_bands = R.n_bands;
        stt[i].ticket0 = R.ticket0;
        stt[i].occ = sparse_ ? reinterpret_cast<unsigned long long *>(d_mem_ + R.off_occ) : nullptr;
        stt[i].row_map = sparse_ ? reinterpret_cast<int *>(d_mem_ + R.off_row_map) : nullptr;
    }
    if (!jobs_.empty()) std::memcpy(blob_.data() + tab_jobs_, jobs_.data(), sizeof(GatherParams) * jobs_.size());
    if (!items_.empty()) std::memcpy(blob_.data() + tab_items_, items_.data(), sizeof(int) * items_.size());
}

cudaError_t WorkSet::enqueue_group(int gi, cudaStream_t s) const
{
    const Group &G = groups_[gi];
    if (G.tiled) {
        const GatherParams *d_jobs = reinterpret_cast<const GatherParams *>(tables_device() + tab_jobs_) + G.job_begin;
        const int *d_items = reinterpret_cast<const int *>(tables_device() + tab_items_) + G.items_off;
        return launch_gather_table(d_jobs, d_items, G.job_end - G.job_begin, G.n_items, jobs_[G.job_begin], G.kind,
                                   tmpl_.elem_bytes, G.gdx, G.gdy, G.shape, s);
    }
    for (int j = G.job_begin; j < G.job_end; ++j) {
        const cudaError_t e = launch_gather(jobs_[j], G.kind, tmpl_.elem_bytes, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t WorkSet::enqueue(cudaStream_t s, bool zero_status, cudaEvent_t const *ev) const
{
    const uint64_t from = zero_status ? off_status_ : off_flags_;
    cudaError_t e = cudaMemsetAsync(d_mem_ + from, 0, off_flags_ + flags_ints_ * sizeof(int) - from, s);
    if (e != cudaSuccess) return e;
    if (built_.empty()) {  // every region prebuilt: the gathers alone
        if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
        for (int g = 0; g < (int)groups_.size(); ++g) {
            e = enqueue_group(g, s);
            if (e != cudaSuccess) return e;
            if (ev && (e = cudaEventRecord(ev[1 + g], s)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    e = launch_quantize_table(reinterpret_cast<const QuantRoi *>(tables_device() + tab_quant_), (int)built_.size(),
                              quant_chunks_, spec_.bins, spec_.bitdepth, spec_.pixel_type == SWIH_PIXEL_U16 ? 2 : 1,
                              s);
    if (e != cudaSuccess) return e;
    ScanParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.B = spec_.bins;
    sp.band_rows = band_rows_;
    sp.n_q = tmpl_.n_q;
    for (int i = 0; i < tmpl_.n_q; ++i) {
        sp.q_val[i] = tmpl_.q_val[i];
        sp.p_count[i] = tmpl_.p_count[i];
        for (int k = 0; k < tmpl_.p_count[i]; ++k) {
            sp.p_val[i][k] = tmpl_.p_val[i][k];
            sp.term[i][k] = tmpl_.term_index[tmpl_.p_val[i][k]][tmpl_.q_val[i]];
        }
    }
    sp.ticket = reinterpret_cast<int *>(d_mem_ + off_flags_) + (flags_ints_ - 1);
    sp.status = status_device();
    sp.spin_limit = 1LL << 22;  // with 64 ns sleeps: well under a few seconds
    sp.stall_tile = -1;
    // a table launch only tests occ for non-NULL; each region writes its own
    sp.occ = sparse_ ? reinterpret_cast<unsigned long long *>(d_mem_ + regions_[built_[0]].off_occ) : nullptr;
    const ScanRoi *d_scan = reinterpret_cast<const ScanRoi *>(tables_device() + tab_scan_);
    e = launch_ih_scan_table(sp, d_scan, (int)built_.size(), scan_tiles_, tmpl_.elem_bytes, scan_E_, scan_threads_,
                             s);
    if (e != cudaSuccess) return e;
    if (sparse_) {
        e = launch_row_map_table(d_scan, (int)built_.size(), spec_.bins, band_rows_, s);
        if (e != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    for (int g = 0; g < (int)groups_.size(); ++g) {
        e = enqueue_group(g, s);
        if (e != cudaSuccess) return e;
        if (ev && (e = cudaEventRecord(ev[1 + g], s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

std::string WorkSet::signature() const
{
    std::string sig = "e" + std::to_string(tmpl_.elem_bytes) + "b" + std::to_string(spec_.bins) + "r" +
                      std::to_string(band_rows_) + (sparse_ ? "s" : "d") + "t";
    for (int t = 0; t < tmpl_.n_terms; ++t)
        sig += std::to_string(tmpl_.term_p[t]) + std::to_string(tmpl_.term_q[t]);
    return sig;
}

WorkRegion WorkSet::region_as_prebuilt(int i) const
{
    const Region &R = regions_[i];
    if (R.prebuilt) return R.in;
    WorkRegion out = R.in;
    out.pre_ih = d_mem_ + R.off_ih;
    out.pre_row_map = sparse_ ? reinterpret_cast<const int *>(d_mem_ + R.off_row_map) : nullptr;
    out.pre_ih_pitch = R.ih_pitch;
    out.pre_plane = R.plane;
    return out;
}

}  // namespace swih
