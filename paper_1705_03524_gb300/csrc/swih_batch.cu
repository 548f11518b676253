// Batches (swih_batch_*): regions of interest of one frame as work sets (one
// per bin count among the ROIs) in memory of their own, enqueued by replaying
// a CUDA graph captured once.
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "swih_host.h"

using namespace swih;

struct swih_batch_s {
    swih_batch_desc desc;
    std::vector<std::unique_ptr<WorkSet>> sets;  // one per bin count
    std::vector<uint64_t> offs;                  // each set's offset in d_mem
    char *d_mem = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

swih_status bfail(swih_status st, const std::string &msg)
{
    thread_error() = msg;
    return st;
}

swih_status bcuda(const char *what, cudaError_t e)
{
    return cuda_fail(nullptr, what, e);
}

// The work sets of a batch: ROIs grouped by bin count (ro.bins, 0: the
// batch's); in each set one region per ROI (a view into the frame) and one job
// per ROI and window over every valid centre. bytes = the sets' memory, each
// set at a 256-byte aligned offset (offs).
swih_status batch_work(const swih_batch_desc *d, const swih_roi_desc *rois, int n, const void *d_frame,
                       std::vector<std::unique_ptr<WorkSet>> &sets, std::vector<uint64_t> &offs, uint64_t &bytes)
{
    if (!d || !rois || n < 1) return bfail(SWIH_ERR_INVALID_ARG, "desc, rois and n_rois >= 1 required");
    if (n > (1 << 20)) return bfail(SWIH_ERR_UNSUPPORTED, "more than 2^20 ROIs in one batch");
    if (d->height < 3 || d->width < 3) return bfail(SWIH_ERR_INVALID_ARG, "frame must be at least 3 x 3");
    const int pb = d->pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    if (d->pitch_bytes < (int64_t)d->width * pb)
        return bfail(SWIH_ERR_INVALID_ARG, "pitch_bytes smaller than a frame row");
    // layout only needs non-NULL addresses; swih_batch_plan passes the frame
    const uint8_t *frame = static_cast<const uint8_t *>(d_frame ? d_frame : reinterpret_cast<const void *>(256));
    std::map<int, std::vector<int>> by_bins;
    for (int i = 0; i < n; ++i) {
        const int B = rois[i].bins > 0 ? rois[i].bins : d->bins;
        if (rois[i].bins < 0 || B > 256)
            return bfail(SWIH_ERR_INVALID_ARG, "ROI " + std::to_string(i) + ": bins must be in [0, 256]");
        by_bins[B].push_back(i);
    }
    sets.clear();
    offs.clear();
    bytes = 0;
    for (auto &kv : by_bins) {
        WorkSpec spec;
        spec.pixel_type = d->pixel_type;
        spec.bitdepth = d->bitdepth;
        spec.bins = kv.first;
        spec.kernel_mask = d->kernel_mask;
        spec.gauss_degree = d->gauss_degree;
        spec.gauss_sigma_frac = d->gauss_sigma_frac;
        spec.precision = d->precision;
        spec.band_rows = d->band_rows;
        std::vector<WorkRegion> regions;
        std::vector<WorkJob> jobs;
        for (int i : kv.second) {
            const swih_roi_desc &ro = rois[i];
            const std::string tag = "ROI " + std::to_string(i);
            if (ro.width < 3 || ro.height < 3 || ro.x0 < 0 || ro.y0 < 0 ||
                (int64_t)ro.x0 + ro.width > d->width || (int64_t)ro.y0 + ro.height > d->height)
                return bfail(SWIH_ERR_INVALID_ARG, tag + " is not inside the frame");
            if (ro.n_windows < 1 || ro.n_windows > SWIH_MAX_SCALES)
                return bfail(SWIH_ERR_INVALID_ARG, tag + ": n_windows out of range");
            if (!ro.d_target) return bfail(SWIH_ERR_INVALID_ARG, tag + ": d_target is NULL");
            WorkRegion reg;
            reg.image = frame + (int64_t)ro.y0 * d->pitch_bytes + (int64_t)ro.x0 * pb;
            reg.pitch = d->pitch_bytes;
            reg.H = ro.height;
            reg.W = ro.width;
            for (int k = 0; k < ro.n_windows; ++k) {
                WorkJob jb;
                jb.region = (int)regions.size();
                jb.kernel = ro.kernel;
                jb.w = ro.win_w[k];
                jb.h = ro.win_h[k];
                jb.target = ro.d_target;
                jb.map = ro.d_map[k];
                if (!jb.map) return bfail(SWIH_ERR_INVALID_ARG, tag + ": window " + std::to_string(k) + " map is NULL");
                jobs.push_back(jb);
            }
            regions.push_back(reg);
        }
        std::unique_ptr<WorkSet> w(new WorkSet());
        std::string err;
        const swih_status st = w->plan(spec, regions, jobs, err);
        if (st != SWIH_OK) return bfail(st, err);
        offs.push_back(bytes);
        bytes += (w->bytes() + 255) / 256 * 256;
        sets.push_back(std::move(w));
    }
    if (d->hbm_budget_bytes && bytes > d->hbm_budget_bytes) {
        char m[160];
        std::snprintf(m, sizeof m, "batch workspace %llu bytes exceeds the budget of %llu bytes",
                      (unsigned long long)bytes, (unsigned long long)d->hbm_budget_bytes);
        return bfail(SWIH_ERR_BUDGET, m);
    }
    return SWIH_OK;
}

swih_status upload_tables(swih_batch_s *b)
{
    for (auto &w : b->sets) {
        const cudaError_t e = cudaMemcpy(w->tables_device(), w->tables(), w->tables_bytes(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bcuda("cudaMemcpy(batch tables)", e);
    }
    return SWIH_OK;
}

swih_status capture(swih_batch_s *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda("cudaStreamBeginCapture", e);
    cudaError_t le = cudaSuccess;
    for (size_t k = 0; k < b->sets.size() && le == cudaSuccess; ++k) le = b->sets[k]->enqueue(b->cap, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda("batch launch (capture)", le);
    }
    if (e != cudaSuccess) return bcuda("cudaStreamEndCapture", e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return bcuda("cudaGraphInstantiate", e);
    return SWIH_OK;
}

}  // namespace

extern "C" {

swih_status swih_batch_workspace_bytes(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois,
                                       uint64_t *bytes)
{
    if (!bytes) return bfail(SWIH_ERR_INVALID_ARG, "bytes is NULL");
    std::vector<std::unique_ptr<WorkSet>> sets;
    std::vector<uint64_t> offs;
    swih_batch_desc d2;
    if (desc) {
        d2 = *desc;
        d2.hbm_budget_bytes = 0;
    }
    return batch_work(desc ? &d2 : nullptr, rois, n_rois, nullptr, sets, offs, *bytes);
}

swih_status swih_batch_plan(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois, const void *d_frame,
                            swih_batch_t *out)
{
    if (!out) return bfail(SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d_frame) return bfail(SWIH_ERR_INVALID_ARG, "d_frame is NULL");
    if (desc && desc->pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_frame) & 1))
        return bfail(SWIH_ERR_INVALID_ARG, "a U16 frame must be 2-byte aligned");
    swih_batch_s *b = new swih_batch_s();
    uint64_t bytes = 0;
    swih_status st = batch_work(desc, rois, n_rois, d_frame, b->sets, b->offs, bytes);
    if (st != SWIH_OK) {
        delete b;
        return st;
    }
    b->desc = *desc;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_mem), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bcuda("cudaMalloc(batch workspace)", e);
    }
    for (size_t k = 0; k < b->offs.size() && e == cudaSuccess; ++k)
        e = cudaMemset(b->d_mem + b->offs[k], 0, 256);  // each set's status block
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(b->d_mem);
        delete b;
        return bcuda("batch set-up", e);
    }
    std::string err;
    for (size_t k = 0; k < b->sets.size(); ++k) {
        st = b->sets[k]->bind(b->d_mem + b->offs[k], err);
        if (st != SWIH_OK) {
            swih_batch_destroy(b);
            return bfail(st, err);
        }
    }
    st = upload_tables(b);
    if (st != SWIH_OK) {
        swih_batch_destroy(b);
        return st;
    }
    *out = b;
    return SWIH_OK;
}

swih_status swih_batch_run(swih_batch_t b, void *stream)
{
    if (!b) return bfail(SWIH_ERR_INVALID_ARG, "batch is NULL");
    if (!b->exec) {
        const swih_status st = capture(b);
        if (st != SWIH_OK) return st;
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return bcuda("cudaGraphLaunch", e);
    return SWIH_OK;
}

swih_status swih_batch_autotune(swih_batch_t b, void *stream)
{
    if (!b) return bfail(SWIH_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // earlier replays may still read the tables that are rewritten below
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bcuda("cudaDeviceSynchronize", e);
    // integral histograms of the current frame, for the timings
    for (auto &ws : b->sets) {
        e = ws->enqueue(s, false);
        if (e != cudaSuccess) return bcuda("batch launch", e);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    swih_status st = SWIH_OK;
    std::string err;
    for (size_t wi = 0; wi < b->sets.size() && st == SWIH_OK; ++wi) {
        WorkSet &w = *b->sets[wi];
        for (int gi = 0; gi < w.n_groups() && st == SWIH_OK; ++gi) {
            const bool gau = w.group_kind(gi) == kGatherGaussian;
            float best = 1e30f;
            int bt = 0, bs = 0, bbb = 0;
            const int txs[2] = {128, 256};
            const int stages[4] = {2, 3, 4, 6};
            // bins per step: 2 exists only with 256 columns and 32-bit elements
            const int bbs[3] = {4, 8, 2};
            for (int ti = 0; ti < 2 && st == SWIH_OK; ++ti)
                for (int si = 0; si < 4 && st == SWIH_OK; ++si)
                    for (int bi = 0; bi < (gau ? 1 : 3) && st == SWIH_OK; ++bi) {
                        if (bbs[bi] == 2 && (txs[ti] != 256 || w.elem_bytes() != 4)) continue;
                        w.set_group_want(gi, txs[ti], stages[si], gau ? 0 : bbs[bi]);
                        st = w.rebuild(err);
                        if (st != SWIH_OK) {
                            st = bfail(st, err);
                            break;
                        }
                        if (!w.group_tiled(gi)) continue;
                        e = cudaStreamSynchronize(s);
                        if (e == cudaSuccess) st = upload_tables(b);
                        if (st != SWIH_OK) break;
                        if (e == cudaSuccess) e = w.enqueue_group(gi, s);  // warm-up
                        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = w.enqueue_group(gi, s);
                        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        if (e != cudaSuccess) {
                            st = bcuda("autotune launch", e);
                            break;
                        }
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (ms < best) {
                            best = ms;
                            bt = txs[ti];
                            bs = stages[si];
                            bbb = gau ? 0 : bbs[bi];
                        }
                    }
            if (st == SWIH_OK) w.set_group_want(gi, bt, bs, bbb);
        }
        if (st == SWIH_OK && w.rebuild(err) != SWIH_OK) st = bfail(SWIH_ERR_INVALID_ARG, err);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SWIH_OK) return st;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda("cudaStreamSynchronize", e);
    st = upload_tables(b);
    if (st == SWIH_OK) st = capture(b);
    return st;
}

swih_status swih_batch_sync_status(swih_batch_t b, void *stream)
{
    if (!b) return bfail(SWIH_ERR_INVALID_ARG, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return bcuda("cudaStreamSynchronize", e);
    uint32_t any = 0;
    for (auto &w : b->sets) {
        uint32_t word = 0;
        e = cudaMemcpy(&word, w->status_device(), sizeof word, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bcuda("cudaMemcpy(status)", e);
        if (word) cudaMemset(w->status_device(), 0, sizeof word);
        any |= word;
    }
    if (any & kStatusTimeout) return bfail(SWIH_ERR_TIMEOUT, "a bounded device wait gave up");
    return SWIH_OK;
}

swih_status swih_batch_destroy(swih_batch_t b)
{
    if (!b) return SWIH_OK;
    cudaError_t e = cudaSuccess;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_mem) e = cudaFree(b->d_mem);
    delete b;
    if (e != cudaSuccess) return bcuda("cudaFree", e);
    return SWIH_OK;
}

}  // extern "C"
