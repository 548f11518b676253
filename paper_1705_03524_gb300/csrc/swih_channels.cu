// Feature channels: several single-valued feature images per pixel (the
// chromatic, shape and texture features whose likelihood maps the tracker of
// Sec. 4 matches one by one), each quantised into its own bins.
//
// The plan numbers every channel's bins globally (channel c owns
// [bin0_c, bin0_c + B_c)) and keeps one bin plane per channel. K1 runs once per
// channel and adds bin0_c to its bins; the scan's chain for bin b reads the
// plane of b's channel; the gather treats the n_channels per-channel targets
// as n_channels targets over all bins, each zero outside its channel, so one
// launch scores every window against every channel and writes one map per
// channel. Every pixel falls in one bin of each channel, so all channels share
// the kernel's window mass M as their normaliser.
#include <cstring>
#include <string>

#include "swih_host.h"

using namespace swih;

namespace {

struct ChannelBins {
    int lo[SWIH_MAX_CHANNELS + 1];  // channel c owns the bins [lo[c], lo[c + 1])
};

// table[c][b] = q[b] for the bins b of channel c, else 0
__global__ void channel_targets_kernel(const float *__restrict__ q, float *__restrict__ table, int B, int C,
                                       ChannelBins cb)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C * B; i += gridDim.x * blockDim.x) {
        const int c = i / B, b = i - c * B;
        table[i] = (b >= cb.lo[c] && b < cb.lo[c + 1]) ? q[b] : 0.f;
    }
}

}  // namespace

extern "C" {

swih_status swih_plan_channels(const swih_plan_desc *desc, int n_channels, const swih_channel_desc *channels,
                               swih_plan_t *out)
{
    if (!out) return fail(nullptr, SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc || !channels) return fail(nullptr, SWIH_ERR_INVALID_ARG, "desc and channels are required");
    if (n_channels < 1 || n_channels > SWIH_MAX_CHANNELS)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "n_channels must be in [1, SWIH_MAX_CHANNELS]");
    swih_plan_s *pl = new swih_plan_s();
    pl->n_ch = n_channels;
    int B = 0;
    for (int c = 0; c < n_channels; ++c) {
        const swih_channel_desc &ch = channels[c];
        const std::string tag = "channel " + std::to_string(c);
        const int pb = ch.pixel_type == SWIH_PIXEL_U8 ? 1 : 2;
        std::string why;
        if (ch.pixel_type != SWIH_PIXEL_U8 && ch.pixel_type != SWIH_PIXEL_U16)
            why = "pixel_type must be U8 or U16";
        else if (ch.bitdepth < 1 || ch.bitdepth > 8 * pb)
            why = "bitdepth out of range for the pixel type";
        else if (ch.pitch_bytes < (int64_t)desc->width * pb)
            why = "pitch_bytes smaller than a row";
        else if (pb == 2 && (ch.pitch_bytes & 1))
            why = "pitch_bytes of a U16 image must be even";
        else if (ch.bins < 1)
            why = "bins must be >= 1";
        if (!why.empty()) {
            delete pl;
            return fail(nullptr, SWIH_ERR_INVALID_ARG, tag + ": " + why);
        }
        pl->ch[c] = ch;
        pl->ch_bin0[c] = B;
        B += ch.bins;
    }
    pl->ch_bin0[n_channels] = B;
    if (B > 256) {
        delete pl;
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "the channels' bins add up to more than 256");
    }
    swih_plan_desc d = *desc;
    d.bins = B;
    d.pixel_type = channels[0].pixel_type;  // validated per channel above
    d.bitdepth = channels[0].bitdepth;
    d.pitch_bytes = channels[0].pitch_bytes;
    const swih_status st = build_layout(&d, pl);
    if (st != SWIH_OK) {
        delete pl;
        return st;
    }
    return allocate_plan(pl, out);
}

swih_status swih_build_ih_channels(swih_plan_t pl, const void *const *d_images, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (pl->n_ch == 0) return fail(pl, SWIH_ERR_INVALID_ARG, "not a feature-channel plan (use swih_build_ih)");
    if (!d_images) return fail(pl, SWIH_ERR_INVALID_ARG, "d_images is NULL");
    for (int c = 0; c < pl->n_ch; ++c) {
        if (!d_images[c]) return fail(pl, SWIH_ERR_INVALID_ARG, "an image pointer is NULL");
        if (pl->ch[c].pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_images[c]) & 1))
            return fail(pl, SWIH_ERR_INVALID_ARG, "a U16 image must be 2-byte aligned");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const swih_plan_desc &d = pl->desc;
    for (int c = 0; c < pl->n_ch; ++c) {
        const swih_channel_desc &ch = pl->ch[c];
        QuantParams qp;
        qp.image = static_cast<const uint8_t *>(d_images[c]);
        qp.pitch = ch.pitch_bytes;
        qp.H = d.height;
        qp.W = d.width;
        qp.B = ch.bins;
        qp.bitdepth = ch.bitdepth;
        qp.bins = reinterpret_cast<uint8_t *>(pl->d_mem) + (int64_t)c * d.height * pl->bins_pitch;
        qp.bins_pitch = pl->bins_pitch;
        qp.pixel_bytes = ch.pixel_type == SWIH_PIXEL_U8 ? 1 : 2;
        qp.vec = (ch.pitch_bytes % 16 == 0) && (reinterpret_cast<uintptr_t>(d_images[c]) % 16 == 0);
        qp.bin0 = pl->ch_bin0[c];
        const cudaError_t e = launch_quantize(qp, s);
        if (e != cudaSuccess) return cuda_fail(pl, "quantize launch", e);
    }
    return build_scans(pl, s);
}

swih_status swih_likelihood_channels(swih_plan_t pl, int kernel, int win_w, int win_h, const float *d_target,
                                     float *d_maps, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (pl->n_ch == 0) return fail(pl, SWIH_ERR_INVALID_ARG, "not a feature-channel plan (use swih_likelihood)");
    swih_status st = check_window(pl, kernel, win_w, win_h);
    if (st != SWIH_OK) return st;
    if (!d_target || !d_maps) return fail(pl, SWIH_ERR_INVALID_ARG, "d_target or d_maps is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int B = pl->desc.bins, C = pl->n_ch;
    float *table = reinterpret_cast<float *>(pl->d_mem + pl->off_chtgt);
    ChannelBins cb;
    for (int c = 0; c <= SWIH_MAX_CHANNELS; ++c) cb.lo[c] = c <= C ? pl->ch_bin0[c] : B;
    channel_targets_kernel<<<(C * B + 255) / 256, 256, 0, s>>>(d_target, table, B, C, cb);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(pl, "channel target table launch", e);
    if (kernel == SWIH_KERNEL_GAUSSIAN && gauss_is_wide(pl, win_w, win_h)) {
        GaussWideParams gw;
        st = make_gauss_wide(pl, win_w, win_h, gw);
        if (st != SWIH_OK) return st;
        gw.cx0 = (win_w - 1) / 2;
        gw.cy0 = (win_h - 1) / 2;
        gw.ncx = pl->desc.width - win_w + 1;
        gw.ncy = pl->desc.height - win_h + 1;
        gw.target = table;
        gw.target_stride = B;
        gw.n_targets = C;
        gw.map = d_maps;
        gw.map_stride = (int64_t)gw.ncx * gw.ncy;
        e = launch_gauss_wide(gw, pl->elem_bytes, s);
        if (e != cudaSuccess) return cuda_fail(pl, "Gaussian gather launch", e);
        return SWIH_OK;
    }
    GatherParams g;
    int kind = 0;
    st = make_gather(pl, kernel, win_w, win_h, g, kind);
    if (st != SWIH_OK) return st;
    g.cx0 = (win_w - 1) / 2;
    g.cy0 = (win_h - 1) / 2;
    g.ncx = pl->desc.width - win_w + 1;
    g.ncy = pl->desc.height - win_h + 1;
    g.target = table;
    g.target_stride = B;
    g.n_targets = C;
    g.map = d_maps;
    g.map_stride = (int64_t)g.ncx * g.ncy;
    e = run_gather(pl, g, kind, s);
    if (e != cudaSuccess) return cuda_fail(pl, "gather launch", e);
    return SWIH_OK;
}

}  // extern "C"
