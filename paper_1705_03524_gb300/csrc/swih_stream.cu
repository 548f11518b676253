// Streamed frames (swih_stream_*): likelihood maps over a frame whose
// integral histograms do not fit in device memory, one band of rows at a time.
//
// With R = (tallest window - 1) / 2, band k owns the centre rows
// [R + k Hb, R + (k+1) Hb) (the first band from row 0, the last up to the
// frame's end, so that shorter windows keep every valid centre); its region
// is the frame rows [k Hb, (k+1) Hb + 2R), which holds every window around
// those centres. Each band is a work set over one region whose jobs write
// straight into the frame-sized maps at the rows the band owns. All bands use
// the same device memory in turn: on one stream, band k+1's table upload and
// launches follow band k's gathers, so nothing is overwritten early.
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "swih_host.h"

using namespace swih;

// a map piece computed into scratch and copied into the frame-sized map
struct MapCopy {
    float *dst;
    int64_t dpitch;  // bytes
    const float *src;
    int64_t spitch;  // bytes
    int64_t width;   // bytes
    int height;
};

struct swih_stream_s {
    swih_plan_desc desc;
    std::vector<swih_frame_job> jobs;
    const void *image = nullptr;
    int band_h = 0, n_bands = 0, R = 0;
    // column tiles (frames wider than one region): tile t owns the centre
    // columns [Rx + t Tw, Rx + (t+1) Tw) (the first from 0, the last to W)
    int Rx = 0, tile_w = 0, n_tiles = 1;
    std::vector<std::unique_ptr<WorkSet>> bands;  // (band, tile) pieces, band-major
    std::vector<std::vector<MapCopy>> copies;     // per piece: maps placed after its gathers
    std::vector<uint64_t> scratch_off;            // per job: its map piece in the scratch
    uint64_t scratch_bytes = 0;
    char *d_mem = nullptr;
    uint64_t bytes = 0;
    char *h_tables = nullptr;  // pinned copies of every band's tables
    std::vector<uint64_t> tab_off;
    cudaStream_t cap = nullptr;
    std::vector<float *> h_maps;           // per job: host copy of its map (NULL: none)
    cudaStream_t down = nullptr;           // the graph branch of the host copies
    cudaEvent_t band_done = nullptr, down_done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

swih_status tfail(swih_status st, const std::string &msg)
{
    thread_error() = msg;
    return st;
}

WorkSpec spec_of(const swih_plan_desc &d)
{
    WorkSpec sp;
    sp.pixel_type = d.pixel_type;
    sp.bitdepth = d.bitdepth;
    sp.bins = d.bins;
    sp.kernel_mask = d.kernel_mask;
    sp.gauss_degree = d.gauss_degree;
    sp.gauss_sigma_frac = d.gauss_sigma_frac;
    sp.precision = d.precision;
    sp.band_rows = d.band_rows;
    return sp;
}

constexpr int kMaxRegionW = 8192;  // the widest region one work set holds

// Lay out the piece (band k, column tile t) of a pass with band height Hb
// (host only). With one tile the jobs write straight into the frame maps;
// with several, each job writes its piece into the scratch (at scratch + the
// job's offset; scratch NULL: layout only) and `copies` receives the copies
// into the frame maps.
swih_status plan_band(const swih_stream_s &S, int Hb, int n_bands, int k, int t, WorkSet &ws, std::string &err,
                      const char *scratch = nullptr, std::vector<MapCopy> *copies = nullptr,
                      std::vector<uint64_t> *piece_floats = nullptr)
{
    const int H = S.desc.height, W = S.desc.width, R = S.R, Rx = S.Rx, Tw = S.tile_w, nt = S.n_tiles;
    const int y0 = k * Hb;
    const int y1 = k == n_bands - 1 ? H : std::min(H, (k + 1) * Hb + 2 * R);
    const int lo = k == 0 ? 0 : R + k * Hb;
    const int hi = k == n_bands - 1 ? H : R + (k + 1) * Hb;
    const int x0 = t * Tw;
    const int x1 = t == nt - 1 ? W : std::min(W, (t + 1) * Tw + 2 * Rx);
    const int lox = t == 0 ? 0 : Rx + t * Tw;
    const int hix = t == nt - 1 ? W : Rx + (t + 1) * Tw;
    const int pb = S.desc.pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    WorkRegion reg;
    reg.image = static_cast<const uint8_t *>(S.image) + (int64_t)y0 * S.desc.pitch_bytes + (int64_t)x0 * pb;
    reg.pitch = S.desc.pitch_bytes;
    reg.H = y1 - y0;
    reg.W = x1 - x0;
    std::vector<WorkJob> jobs;
    if (piece_floats) piece_floats->assign(S.jobs.size(), 0);
    for (size_t j = 0; j < S.jobs.size(); ++j) {
        const swih_frame_job &fj = S.jobs[j];
        const int rx = (fj.win_w - 1) / 2, ry = (fj.win_h - 1) / 2;
        const int c_lo = std::max(lo, ry), c_hi = std::min(hi, H - ry);
        const int cx_lo = std::max(lox, rx), cx_hi = std::min(hix, W - rx);
        if (c_hi <= c_lo || cx_hi <= cx_lo) continue;
        WorkJob jb;
        jb.region = 0;
        jb.kernel = fj.kernel;
        jb.w = fj.win_w;
        jb.h = fj.win_h;
        jb.cx0 = cx_lo - x0;
        jb.ncx = cx_hi - cx_lo;
        jb.cy0 = c_lo - y0;
        jb.ncy = c_hi - c_lo;
        jb.target = fj.d_target;
        const int64_t frame_nx = W - fj.win_w + 1;
        float *dst = fj.d_map + (int64_t)(c_lo - ry) * frame_nx + (cx_lo - rx);
        if (nt == 1) {
            jb.map = dst;
        } else {
            jb.map = scratch ? reinterpret_cast<float *>(const_cast<char *>(scratch) + S.scratch_off[j])
                             : reinterpret_cast<float *>(256);  // layout only
            if (copies)
                copies->push_back(MapCopy{dst, frame_nx * 4, jb.map, (int64_t)jb.ncx * 4, (int64_t)jb.ncx * 4,
                                          jb.ncy});
            if (piece_floats) (*piece_floats)[j] = (uint64_t)jb.ncx * jb.ncy;
        }
        jobs.push_back(jb);
    }
    return ws.plan(spec_of(S.desc), {reg}, jobs, err);
}

// Every piece for band height Hb; bytes = the largest piece's memory.
swih_status plan_bands(swih_stream_s &S, int Hb, std::vector<std::unique_ptr<WorkSet>> &out, uint64_t &bytes,
                       std::string &err)
{
    const int rows = S.desc.height - 2 * S.R;  // centre rows of the tallest window
    const int n = std::max(1, (rows + Hb - 1) / Hb);
    out.clear();
    bytes = 0;
    for (int k = 0; k < n; ++k)
        for (int t = 0; t < S.n_tiles; ++t) {
            std::unique_ptr<WorkSet> ws(new WorkSet());
            const swih_status st = plan_band(S, Hb, n, k, t, *ws, err);
            if (st != SWIH_OK) return st;
            bytes = std::max(bytes, ws->bytes());
            out.push_back(std::move(ws));
        }
    return SWIH_OK;
}

// the map pieces of piece k into the frame maps (several column tiles only)
cudaError_t enqueue_copies(const swih_stream_s &S, size_t k, cudaStream_t s)
{
    if (k >= S.copies.size()) return cudaSuccess;
    for (const MapCopy &c : S.copies[k]) {
        const cudaError_t e = cudaMemcpy2DAsync(c.dst, (size_t)c.dpitch, c.src, (size_t)c.spitch, (size_t)c.width,
                                                (size_t)c.height, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// band k's rows of every job's map into the job's host map (whole rows: one
// contiguous copy per job), on stream s
cudaError_t enqueue_downloads(const swih_stream_s &S, int k, cudaStream_t s)
{
    const int H = S.desc.height, W = S.desc.width, R = S.R, Hb = S.band_h, nb = S.n_bands;
    const int lo = k == 0 ? 0 : R + k * Hb;
    const int hi = k == nb - 1 ? H : R + (k + 1) * Hb;
    for (size_t j = 0; j < S.jobs.size(); ++j) {
        float *h = j < S.h_maps.size() ? S.h_maps[j] : nullptr;
        if (!h) continue;
        const swih_frame_job &fj = S.jobs[j];
        const int ry = (fj.win_h - 1) / 2;
        const int c_lo = std::max(lo, ry), c_hi = std::min(hi, H - ry);
        if (c_hi <= c_lo) continue;
        const int64_t nx = W - fj.win_w + 1;
        const int64_t off = (int64_t)(c_lo - ry) * nx;
        const cudaError_t e = cudaMemcpyAsync(h + off, fj.d_map + off, (size_t)(c_hi - c_lo) * nx * sizeof(float),
                                              cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

swih_status capture(swih_stream_s *S)
{
    cudaError_t e = cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaStreamBeginCapture", e);
    cudaError_t le = cudaSuccess;
    bool down = false;
    for (float *h : S->h_maps) down |= h != nullptr;
    for (size_t k = 0; k < S->bands.size() && le == cudaSuccess; ++k) {
        WorkSet &ws = *S->bands[k];
        le = cudaMemcpyAsync(ws.tables_device(), S->h_tables + S->tab_off[k], ws.tables_bytes(),
                             cudaMemcpyHostToDevice, S->cap);
        if (le == cudaSuccess) le = ws.enqueue(S->cap, false);
        if (le == cudaSuccess) le = enqueue_copies(*S, k, S->cap);
        if (down && le == cudaSuccess && (k + 1) % S->n_tiles == 0) {
            // the band is complete: its map rows go down beside the next band
            le = cudaEventRecord(S->band_done, S->cap);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(S->down, S->band_done, 0);
            if (le == cudaSuccess) le = enqueue_downloads(*S, (int)(k / S->n_tiles), S->down);
        }
    }
    if (down && le == cudaSuccess) {  // the pass ends with its last copy
        le = cudaEventRecord(S->down_done, S->down);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(S->cap, S->down_done, 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(S->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(nullptr, "streamed pass launch (capture)", le);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaStreamEndCapture", e);
    S->graph = g;
    e = cudaGraphInstantiate(&S->exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaGraphInstantiate", e);
    return SWIH_OK;
}

}  // namespace

extern "C" {

swih_status swih_stream_plan(const swih_plan_desc *desc, const swih_frame_job *jobs, int n_jobs, const void *d_image,
                             int32_t band_height, swih_stream_t *out)
{
    if (!out) return tfail(SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc || !jobs || n_jobs < 1 || !d_image)
        return tfail(SWIH_ERR_INVALID_ARG, "desc, jobs (n_jobs >= 1) and d_image are required");
    if (band_height < 0) return tfail(SWIH_ERR_INVALID_ARG, "band_height must be >= 0");
    if (band_height == 0 && desc->hbm_budget_bytes == 0)
        return tfail(SWIH_ERR_INVALID_ARG, "band_height 0 needs hbm_budget_bytes");
    if (desc->height < 3 || desc->width < 3) return tfail(SWIH_ERR_INVALID_ARG, "frame must be at least 3 x 3");
    std::unique_ptr<swih_stream_s> S(new swih_stream_s());
    S->desc = *desc;
    S->jobs.assign(jobs, jobs + n_jobs);
    S->image = d_image;
    int hmax = 3, wmax = 3;
    for (int j = 0; j < n_jobs; ++j) {
        const swih_frame_job &fj = jobs[j];
        if (!odd_window(fj.win_w) || !odd_window(fj.win_h) || fj.win_w > desc->width || fj.win_h > desc->height)
            return tfail(SWIH_ERR_INVALID_ARG, "job " + std::to_string(j) + ": window must be odd, >= 3, inside the frame");
        if (!fj.d_target || !fj.d_map) return tfail(SWIH_ERR_INVALID_ARG, "job " + std::to_string(j) + ": NULL target or map");
        hmax = std::max(hmax, fj.win_h);
        wmax = std::max(wmax, fj.win_w);
    }
    S->R = (hmax - 1) / 2;
    S->Rx = (wmax - 1) / 2;
    if (desc->width <= kMaxRegionW) {
        S->n_tiles = 1;
        S->tile_w = std::max(1, desc->width - 2 * S->Rx);
    } else {
        // column tiles of at most kMaxRegionW columns, halo 2 Rx
        S->tile_w = kMaxRegionW - 2 * S->Rx;
        if (S->tile_w < 256) return tfail(SWIH_ERR_UNSUPPORTED, "windows too wide for column tiles");
        S->n_tiles = (desc->width - 2 * S->Rx + S->tile_w - 1) / S->tile_w;
    }
    const int rows = desc->height - 2 * S->R;
    std::string err;
    uint64_t bytes = 0;
    int Hb = band_height > 0 ? std::min(band_height, std::max(1, rows)) : 0;
    if (Hb == 0) {
        // the largest band height whose band fits the budget (memory grows with it)
        int lo = 1, hi = std::max(1, rows), best = 0;
        while (lo <= hi) {
            const int mid = lo + (hi - lo) / 2;
            std::unique_ptr<WorkSet> ws(new WorkSet());
            const int n = std::max(1, (rows + mid - 1) / mid);
            swih_status st = plan_band(*S, mid, n, n > 1 ? 1 : 0, 0, *ws, err);
            if (st == SWIH_OK && n > 1) {  // the first band can be the tallest region too
                std::unique_ptr<WorkSet> w0(new WorkSet());
                st = plan_band(*S, mid, n, 0, 0, *w0, err);
                if (st == SWIH_OK && w0->bytes() > ws->bytes()) ws = std::move(w0);
            }
            if (st != SWIH_OK) return tfail(st, err);
            if (ws->bytes() <= desc->hbm_budget_bytes) {
                best = mid;
                lo = mid + 1;
            } else {
                hi = mid - 1;
            }
        }
        if (best == 0) return tfail(SWIH_ERR_BUDGET, "even one-row bands exceed hbm_budget_bytes");
        Hb = best;
    }
    for (;;) {
        const swih_status st = plan_bands(*S, Hb, S->bands, bytes, err);
        if (st != SWIH_OK) return tfail(st, err);
        if (!desc->hbm_budget_bytes || bytes <= desc->hbm_budget_bytes) break;
        if (Hb == 1) return tfail(SWIH_ERR_BUDGET, "even one-row bands exceed hbm_budget_bytes");
        Hb = std::max(1, Hb - std::max(1, Hb / 16));  // a last band taller than the probe: shrink
    }
    S->band_h = Hb;
    const int n_bands = (int)S->bands.size() / S->n_tiles;
    S->n_bands = n_bands;
    // column tiles: each job's largest piece in a scratch after the work memory
    S->scratch_off.assign(S->jobs.size(), 0);
    if (S->n_tiles > 1) {
        std::vector<uint64_t> most(S->jobs.size(), 0), piece;
        for (int k = 0; k < n_bands; ++k)
            for (int t = 0; t < S->n_tiles; ++t) {
                WorkSet probe;
                const swih_status st = plan_band(*S, Hb, n_bands, k, t, probe, err, nullptr, nullptr, &piece);
                if (st != SWIH_OK) return tfail(st, err);
                for (size_t j = 0; j < piece.size(); ++j) most[j] = std::max(most[j], piece[j]);
            }
        uint64_t off = (bytes + 255) / 256 * 256;
        for (size_t j = 0; j < most.size(); ++j) {
            S->scratch_off[j] = off;
            off += (most[j] * sizeof(float) + 255) / 256 * 256;
        }
        S->scratch_bytes = off - bytes;
        if (desc->hbm_budget_bytes && off > desc->hbm_budget_bytes)
            return tfail(SWIH_ERR_BUDGET, "the maps' tile pieces do not fit hbm_budget_bytes with this band height");
    }
    S->bytes = bytes + S->scratch_bytes;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&S->d_mem), S->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(nullptr, "cudaMalloc(stream workspace)", e);
    }
    if (S->n_tiles > 1) {
        // the pieces again, now writing their maps into the scratch, with the copies
        S->copies.assign(S->bands.size(), {});
        for (int k = 0; k < n_bands; ++k)
            for (int t = 0; t < S->n_tiles; ++t) {
                const size_t i = (size_t)k * S->n_tiles + t;
                S->bands[i].reset(new WorkSet());
                const swih_status st = plan_band(*S, Hb, n_bands, k, t, *S->bands[i], err, S->d_mem, &S->copies[i]);
                if (st != SWIH_OK) {
                    cudaFree(S->d_mem);
                    return tfail(st, err);
                }
            }
    }
    uint64_t tab_total = 0;
    for (auto &ws : S->bands) {
        const swih_status st = ws->bind(S->d_mem, err);
        if (st != SWIH_OK) {
            cudaFree(S->d_mem);
            return tfail(st, err);
        }
        S->tab_off.push_back(tab_total);
        tab_total += (ws->tables_bytes() + 255) / 256 * 256;
    }
    e = cudaMallocHost(reinterpret_cast<void **>(&S->h_tables), std::max<uint64_t>(tab_total, 256));
    if (e == cudaSuccess) e = cudaMemset(S->d_mem, 0, 256);  // status word
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->down, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->band_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->down_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        swih_stream_destroy(S.release());
        return cuda_fail(nullptr, "stream set-up", e);
    }
    for (size_t k = 0; k < S->bands.size(); ++k)
        std::memcpy(S->h_tables + S->tab_off[k], S->bands[k]->tables(), S->bands[k]->tables_bytes());
    *out = S.release();
    return SWIH_OK;
}

swih_status swih_stream_run(swih_stream_t S, void *stream)
{
    if (!S) return tfail(SWIH_ERR_INVALID_ARG, "stream plan is NULL");
    if (!S->exec) {
        const swih_status st = capture(S);
        if (st != SWIH_OK) return st;
    }
    const cudaError_t e = cudaGraphLaunch(S->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaGraphLaunch", e);
    return SWIH_OK;
}

swih_status swih_stream_set_host_maps(swih_stream_t S, float *const *h_maps)
{
    if (!S) return tfail(SWIH_ERR_INVALID_ARG, "stream plan is NULL");
    std::vector<float *> v(S->jobs.size(), nullptr);
    if (h_maps)
        for (size_t j = 0; j < v.size(); ++j) v[j] = h_maps[j];
    if (v == S->h_maps) return SWIH_OK;
    S->h_maps = v;
    // capture the pass again at the next run
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    S->exec = nullptr;
    S->graph = nullptr;
    return SWIH_OK;
}

swih_status swih_stream_run_timed(swih_stream_t S, void *stream, float *stage_ms)
{
    if (!S || !stage_ms) return tfail(SWIH_ERR_INVALID_ARG, "stream plan and stage_ms are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < 7; ++i) stage_ms[i] = 0.f;
    // per band: start, after the scan, after each job group
    std::vector<std::vector<cudaEvent_t>> ev(S->bands.size());
    auto destroy = [&]() {
        for (auto &v : ev)
            for (cudaEvent_t x : v) cudaEventDestroy(x);
    };
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < S->bands.size() && e == cudaSuccess; ++k) {
        const WorkSet &ws = *S->bands[k];
        ev[k].assign(2 + ws.n_groups(), nullptr);
        for (auto &x : ev[k])
            if (e == cudaSuccess) e = cudaEventCreate(&x);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k][0], s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.tables_device(), S->h_tables + S->tab_off[k], ws.tables_bytes(),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = ws.enqueue(s, false, ev[k].data() + 1);
        if (e == cudaSuccess) e = enqueue_copies(*S, k, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t k = 0; k < S->bands.size() && e == cudaSuccess; ++k) {
        const WorkSet &ws = *S->bands[k];
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[k][0], ev[k][1]);
        stage_ms[0] += ms;
        for (int g = 0; g < ws.n_groups() && e == cudaSuccess; ++g) {
            e = cudaEventElapsedTime(&ms, ev[k][1 + g], ev[k][2 + g]);
            stage_ms[1 + ws.group_kind(g)] += ms;  // GatherKind numbers the kernels as swih_kernel does
        }
    }
    destroy();
    if (e != cudaSuccess) return cuda_fail(nullptr, "timed streamed pass", e);
    return SWIH_OK;
}

swih_status swih_stream_load_bytes(swih_stream_t S, uint64_t *bytes, int reset)
{
    if (!S || !bytes) return tfail(SWIH_ERR_INVALID_ARG, "stream plan and bytes are required");
    unsigned long long c[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, S->d_mem + 8, sizeof c, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(S->d_mem + 8, 0, sizeof c);
    if (e != cudaSuccess) return cuda_fail(nullptr, "stream load counters", e);
    for (int i = 0; i < 5; ++i) bytes[i] = c[i];
    return SWIH_OK;
}

swih_status swih_stream_sync_status(swih_stream_t S, void *stream)
{
    if (!S) return tfail(SWIH_ERR_INVALID_ARG, "stream plan is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaStreamSynchronize", e);
    uint32_t word = 0;
    e = cudaMemcpy(&word, S->d_mem, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaMemcpy(status)", e);
    if (word) {
        cudaMemset(S->d_mem, 0, sizeof word);
        if (word & kStatusTimeout) return tfail(SWIH_ERR_TIMEOUT, "a bounded device wait gave up");
    }
    return SWIH_OK;
}

swih_status swih_stream_get_info(swih_stream_t S, int32_t *band_height, int32_t *n_bands, uint64_t *workspace_bytes)
{
    if (!S) return tfail(SWIH_ERR_INVALID_ARG, "stream plan is NULL");
    if (band_height) *band_height = S->band_h;
    if (n_bands) *n_bands = S->n_bands;
    if (workspace_bytes) *workspace_bytes = S->bytes;
    return SWIH_OK;
}

swih_status swih_stream_destroy(swih_stream_t S)
{
    if (!S) return SWIH_OK;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->cap) cudaStreamDestroy(S->cap);
    if (S->down) cudaStreamDestroy(S->down);
    if (S->band_done) cudaEventDestroy(S->band_done);
    if (S->down_done) cudaEventDestroy(S->down_done);
    cudaError_t e = cudaSuccess;
    if (S->d_mem) e = cudaFree(S->d_mem);
    if (S->h_tables) cudaFreeHost(S->h_tables);
    delete S;
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaFree", e);
    return SWIH_OK;
}

}  // extern "C"
