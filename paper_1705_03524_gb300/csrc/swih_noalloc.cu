// swih_build_ih_noalloc: the integral-histogram build for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: processes that hand all device
// memory to a fixed pool up front (embedded tracking pipelines), real-time loops
// that may not take the device-wide synchronisation a driver allocation can
// cause, or hosts whose allocator policy forbids driver allocations after
// start-up. They can
// own the input frame and the output integral histograms, but not a plan (which
// allocates its own workspace). For them this entry point runs the same
// quantisation and scan kernels with the scan's intermediate data -- the bin
// image, the look-back state vectors, tile flags, ticket and status word --
// placed in one file-scope device array of fixed size, kStaticScratchBytes.
//
// The array exists once per device that loads the library and stays allocated
// until the process exits. Host code must not use its name as a pointer: the
// device address is looked up once per device with cudaGetSymbolAddress, on the
// first call made with that device current, and cached.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "swih.h"
#include "swih_internal.h"

namespace swih {
swih_status plan_layout(const swih_plan_desc *d, PlanLayout *out);
void set_thread_error(const char *msg);
}  // namespace swih

using namespace swih;

namespace {

constexpr uint64_t kStaticScratchBytes = 8ull << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

swih_status fail_na(swih_status st, const char *msg)
{
    set_thread_error(msg);
    return st;
}

swih_status cuda_fail_na(const char *what, cudaError_t e)
{
    char m[256];
    std::snprintf(m, sizeof m, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    set_thread_error(m);
    return SWIH_ERR_CUDA;
}

// device address of the static scratch on the current device (set up once per device)
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

inline uint64_t align256(uint64_t v) { return (v + 255) / 256 * 256; }

struct ScratchMap {
    uint64_t bins = 0, agg = 0, incl = 0, flags = 0, status = 0, total = 0, flags_bytes = 0;
};

ScratchMap scratch_map(const swih_plan_desc &d, const PlanLayout &L)
{
    ScratchMap m;
    const uint64_t chains = (uint64_t)d.bins * L.n_q;
    const uint64_t state = chains * L.n_bands * L.ih_pitch * L.elem_bytes;
    uint64_t off = 0;
    m.bins = off;
    off = align256(off + (uint64_t)d.height * L.bins_pitch);
    m.agg = off;
    off = align256(off + state);
    m.incl = off;
    off = align256(off + state);
    m.flags = off;
    m.flags_bytes = (chains * L.n_bands + 1) * sizeof(int);
    off = align256(off + m.flags_bytes);
    m.status = off;
    off = align256(off + sizeof(uint32_t));
    m.total = off;
    return m;
}

}  // namespace

extern "C" swih_status swih_build_ih_noalloc(const swih_plan_desc *desc, const void *d_image,
                                             void *d_ih, uint64_t ih_bytes, uint32_t *d_status,
                                             swih_plan_info *layout, void *stream)
{
    if (!desc) return fail_na(SWIH_ERR_INVALID_ARG, "desc is NULL");
    if (desc->kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_EXPONENTIAL))
        return fail_na(SWIH_ERR_UNSUPPORTED, "the allocation-free build serves the integer integral histograms only "
                                             "(no exponential kernel)");
    swih_plan_desc d = *desc;
    PlanLayout L;
    swih_status st = plan_layout(&d, &L);
    if (st != SWIH_OK) return st;
    ScratchMap m = scratch_map(d, L);
    if (m.total > kStaticScratchBytes && desc->band_rows == 0) {
        // taller bands -> fewer look-back state vectors
        const uint64_t per_band = 2 * align256((uint64_t)d.bins * L.n_q * L.ih_pitch * L.elem_bytes);
        const uint64_t fixed = align256((uint64_t)d.height * L.bins_pitch) + 2 * 256 + 4096;
        const uint64_t room = kStaticScratchBytes > fixed ? kStaticScratchBytes - fixed : 0;
        uint64_t max_bands = per_band ? room / (per_band + 16 * (uint64_t)d.bins * L.n_q) : 0;
        if (max_bands >= 1) {
            d.band_rows = (int)((d.height + max_bands - 1) / max_bands);
            st = plan_layout(&d, &L);
            if (st != SWIH_OK) return st;
            m = scratch_map(d, L);
        }
    }
    if (m.total > kStaticScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "needs %llu bytes of scratch; the static scratch holds %llu bytes "
                      "(use a smaller image, fewer bins or terms, or a plan)",
                      (unsigned long long)m.total, (unsigned long long)kStaticScratchBytes);
        return fail_na(SWIH_ERR_UNSUPPORTED, msg);
    }
    const uint64_t ih_need =
        (uint64_t)L.n_terms * d.bins * (uint64_t)L.plane * (uint64_t)L.elem_bytes;
    if (layout) {
        std::memset(layout, 0, sizeof *layout);
        layout->height = d.height;
        layout->width = d.width;
        layout->bins = d.bins;
        layout->elem_bytes = L.elem_bytes;
        layout->n_terms = L.n_terms;
        for (int t = 0; t < L.n_terms; ++t) {
            layout->term_p[t] = L.term_p[t];
            layout->term_q[t] = L.term_q[t];
        }
        layout->d_ih = d_ih;
        layout->bins_pitch = L.bins_pitch;
        layout->ih_pitch = L.ih_pitch;
        layout->plane_elems = L.plane;
        layout->band_rows = L.band_rows;
        layout->n_bands = L.n_bands;
        layout->workspace_bytes = ih_need;  // bytes the caller's d_ih must hold
        layout->n_channels = 1;
    }
    // Every call, a size query included, looks up the static array's device
    // address on the current device, so a size query made before a stream
    // capture already counts as the device's first call.
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail_na("cudaGetSymbolAddress(static scratch)", e);
    char *sc = static_cast<char *>(base);
    if (layout) layout->d_bins = sc + m.bins;
    if (!d_ih) return SWIH_OK;  // size query: nothing is enqueued
    if (ih_bytes < ih_need) return fail_na(SWIH_ERR_INVALID_ARG, "ih_bytes is smaller than the layout needs");
    if (!d_image) return fail_na(SWIH_ERR_INVALID_ARG, "d_image is NULL");
    if (d.pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_image) & 1))
        return fail_na(SWIH_ERR_INVALID_ARG, "a U16 image must be 2-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_ih) % 16)
        return fail_na(SWIH_ERR_INVALID_ARG, "d_ih must be 16-byte aligned");

    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // tile flags and ticket must start at zero; so must the built-in status word
    e = cudaMemsetAsync(sc + m.flags, 0, m.flags_bytes, s);
    if (e == cudaSuccess && !d_status) e = cudaMemsetAsync(sc + m.status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail_na("cudaMemsetAsync(static scratch)", e);

    QuantParams qp;
    qp.image = static_cast<const uint8_t *>(d_image);
    qp.pitch = d.pitch_bytes;
    qp.H = d.height;
    qp.W = d.width;
    qp.B = d.bins;
    qp.bitdepth = d.bitdepth;
    qp.bins = reinterpret_cast<uint8_t *>(sc + m.bins);
    qp.bins_pitch = L.bins_pitch;
    qp.pixel_bytes = d.pixel_type == SWIH_PIXEL_U8 ? 1 : 2;
    qp.vec = (d.pitch_bytes % 16 == 0) && (reinterpret_cast<uintptr_t>(d_image) % 16 == 0);
    e = launch_quantize(qp, s);
    if (e != cudaSuccess) return cuda_fail_na("quantize launch", e);

    ScanParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.bins = qp.bins;
    sp.bins_pitch = L.bins_pitch;
    sp.ih = d_ih;
    sp.ih_pitch = L.ih_pitch;
    sp.plane = L.plane;
    sp.agg = sc + m.agg;
    sp.incl = sc + m.incl;
    sp.flags = reinterpret_cast<int *>(sc + m.flags);
    sp.ticket = sp.flags + (int64_t)d.bins * L.n_q * L.n_bands;
    sp.status = d_status ? d_status : reinterpret_cast<uint32_t *>(sc + m.status);
    sp.H = d.height;
    sp.W = d.width;
    sp.B = d.bins;
    sp.band_rows = L.band_rows;
    sp.n_bands = L.n_bands;
    sp.n_q = L.n_q;
    for (int i = 0; i < L.n_q; ++i) {
        sp.q_val[i] = L.q_val[i];
        sp.p_count[i] = L.p_count[i];
        for (int k = 0; k < L.p_count[i]; ++k) {
            sp.p_val[i][k] = L.p_val[i][k];
            sp.term[i][k] = L.term[i][k];
        }
    }
    sp.spin_limit = 1LL << 22;
    sp.stall_tile = -1;
    e = launch_ih_scan(sp, L.elem_bytes, L.scan_E, L.scan_threads, s);
    if (e != cudaSuccess) return cuda_fail_na("ih_scan launch", e);
    return SWIH_OK;
}
