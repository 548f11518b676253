/*
 * swih.h -- C ABI of the GB300 library for spatially weighted local
 * histograms in O(1) per window (SWIH, arXiv 1705.03524).
 *
 * The pipeline (Sec. 1 steps (1)-(5), Fig. 2):
 *   quantise pixels into B bins (the quantiser Q of Sec. 2.1)
 *   -> one weighted integral histogram per bin and weight term (Eq. 2)
 *   -> for every window centre, rectangle sums from the 3 x 3 lattice of
 *      window corners, translated to the centre and combined into the
 *      kernel-weighted histogram, normalised by the kernel's total weight
 *      (which is the same at every location, Sec. 2.1)
 *   -> Bhattacharyya coefficient against a target histogram (the sliding
 *      window matching of Sec. 2 / Fig. 3, which the paper leaves unnamed).
 *
 * Conventions shared by every call:
 *   - x is the column, y the row; images are row-major.
 *   - A window is win_w x win_h pixels, both odd and >= 3, with half sizes
 *     rx = (win_w-1)/2, ry = (win_h-1)/2. A centre (xc, yc) is valid when its
 *     whole window lies inside the image: rx <= xc < W-rx, ry <= yc < H-ry.
 *     The valid centres form a (H-win_h+1) x (W-win_w+1) map.
 *   - "d_" pointers are device pointers owned by the caller; the library
 *     never frees them. A plan owns its own workspace (bins, integral
 *     histograms, scan state) from swih_plan until swih_destroy.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Calls only enqueue work; they never synchronise the stream,
 *     except swih_plan / swih_destroy (allocation) and swih_sync_status.
 *   - Every call returns a swih_status. Argument errors are detected on the
 *     host before anything is enqueued. swih_last_error gives a message.
 *   - A plan is not thread-safe: one host thread at a time per plan. Work
 *     enqueued on different streams against the same plan must be ordered
 *     by the caller (build before gather).
 */
#ifndef SWIH_H
#define SWIH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum swih_status {
    SWIH_OK = 0,
    SWIH_ERR_INVALID_ARG = 1, /* a size, pointer, window or enum out of range */
    SWIH_ERR_UNSUPPORTED = 2, /* valid request outside what this build serves */
    SWIH_ERR_OOM = 3,         /* device allocation failed */
    SWIH_ERR_BUDGET = 4,      /* workspace larger than hbm_budget_bytes */
    SWIH_ERR_CUDA = 5,        /* a CUDA runtime call failed (message has the name) */
    SWIH_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (scan look-back) */
    SWIH_ERR_CANCELLED = 7    /* a server query cancelled before it was admitted */
} swih_status;

typedef enum swih_pixel_type { SWIH_PIXEL_U8 = 0, SWIH_PIXEL_U16 = 1 } swih_pixel_type;

/* Spatial kernels K(dx, dy), dx = x - xc, dy = y - yc (Fig. 1, Fig. 4):
 *   PLAIN      K = 1 (Porikli's local histogram)
 *   MANHATTAN  K = (rx-|dx|) + (ry-|dy|): Eq. 1's city-block distance taken
 *              from its corner value, zero at the window corners, largest at
 *              the centre; linear in each quadrant (Sec. 2.1, Fig. 4(b))
 *   EUCLIDEAN  K = (rx^2-dx^2) + (ry^2-dy^2): the same on the squared
 *              Euclidean distance (the paper gives no formula)
 *   GAUSSIAN   K = Px(dx^2/rx^2) * Py(dy^2/ry^2), P the least-squares
 *              polynomial of degree min(D, r) fitted to exp(-d^2/(2 s^2)) on
 *              d = -r..r, s = gauss_sigma_frac * window side (the paper names
 *              the Gaussian without a decomposition). Largest distance from
 *              the true Gaussian on windows of 15-401 px: about 0.03 at
 *              D = 2, 0.005 at D = 3, 5e-4 at D = 4. Degrees above 2, and
 *              windows in the 128-bit ring, take a gather with one thread
 *              per centre (slower than the tiled gather of D <= 2).
 *   WEDDING    the wedding-cake approximation of Sec. 2 (Fig. 4(a)) to the
 *              Manhattan kernel: n nested windows around the centre with
 *              half-sides floor((2 i r + n) / (2 n)), i = 1..n, per axis; the
 *              ring between nested windows i-1 and i weighs the mean of the
 *              Manhattan kernel over that ring's pixels. Computed from plain
 *              (unweighted) integral histograms only; n = wedding_rings.
 *              The paper names the scheme without ring sizes or weights.
 *   EXPONENTIAL K = exp(-lambda (|dx| + |dy|)), lambda = exp_lambda per pixel
 *              (the paper names an exponential kernel without a formula).
 *              The same lambda serves every window size. Built from four
 *              directional weighted integral histograms (weights exp(+-lambda
 *              x) exp(+-lambda y), one per quadrant, each summed from the side
 *              where its weight is smallest and divided by the weight at the
 *              point), kept in unsigned 64-bit fixed point (see
 *              swih_plan_info.exp_frac_bits). A bin's window count comes from
 *              the exact plain integral histogram, so bins absent from a
 *              window give exactly 0; the others carry a rounding error below
 *              2^-28 of the window's total weight.                          */
typedef enum swih_kernel {
    SWIH_KERNEL_PLAIN = 0,
    SWIH_KERNEL_MANHATTAN = 1,
    SWIH_KERNEL_EUCLIDEAN = 2,
    SWIH_KERNEL_GAUSSIAN = 3,
    SWIH_KERNEL_WEDDING = 4,
    SWIH_KERNEL_EXPONENTIAL = 5
} swih_kernel;

#define SWIH_KERNEL_BIT(k) (1u << (unsigned)(k))

/* Element type of the integral histograms. The weights x^p y^q are integers,
 * so every integral histogram is kept exactly in the ring of integers modulo
 * 2^32, 2^64 or 2^128 (wrap-around arithmetic). Rectangle sums, translation to
 * the centre and kernel combination are ring operations, so every window's
 * result is exact whenever its true value fits the ring.
 *   AUTO    RING32 when every requested kernel's total window weight at the
 *           largest window is below 2^32 and no Gaussian is requested;
 *           RING64 when that holds for 2^64 and the Gaussian's largest
 *           Bernstein moment w h rx^2D ry^2D is below 2^64; else RING128
 *   RING32  4-byte elements (rejected with UNSUPPORTED if not exact)
 *   RING64  8-byte elements (likewise)
 *   RING128 16-byte elements: plans of the Gaussian kernel alone, widths up
 *           to 4096 and w h rx^2D ry^2D below 2^128 (D = 2: any window of
 *           such an image; D = 3: windows up to about 900 px; D = 4: up to
 *           255 px)                                                          */
typedef enum swih_precision {
    SWIH_PREC_AUTO = 0,
    SWIH_PREC_RING32 = 1,
    SWIH_PREC_RING64 = 2,
    SWIH_PREC_RING128 = 3
} swih_precision;

typedef struct swih_plan_desc {
    int32_t height;            /* H >= 3 */
    int32_t width;             /* W, 3 <= W <= 8192 */
    int64_t pitch_bytes;       /* input row stride in bytes, >= W * pixel size */
    int32_t pixel_type;        /* swih_pixel_type */
    int32_t bitdepth;          /* significant bits: 1..8 (U8) or 1..16 (U16) */
    int32_t bins;              /* B, 1..256 */
    uint32_t kernel_mask;      /* OR of SWIH_KERNEL_BIT(k) the plan must serve */
    int32_t gauss_degree;      /* D of the Gaussian approximant, 1..4 (0: 2) */
    double gauss_sigma_frac;   /* Gaussian sigma / window side (0: 0.25) */
    int32_t max_win_w;         /* largest window the plan serves (odd, <= W) */
    int32_t max_win_h;         /* (odd, <= H) */
    int32_t precision;         /* swih_precision */
    int32_t band_rows;         /* rows per scan band (0: automatic) */
    uint64_t hbm_budget_bytes; /* reject plans whose workspace exceeds it (0: no limit) */
    int32_t wedding_rings;     /* nested windows of the WEDDING kernel, 1..16 (0: 4) */
    double exp_lambda;         /* decay per pixel of the EXPONENTIAL kernel, 2^-10..16 (0: 0.1) */
} swih_plan_desc;

typedef struct swih_plan_s *swih_plan_t;

/* Workspace a plan with this description would allocate (host only, no CUDA
 * call). Used for admission against a memory budget. */
swih_status swih_plan_workspace_bytes(const swih_plan_desc *desc, uint64_t *bytes);

/* Validate the description, choose the term set and ring, allocate the
 * workspace on the current device. *out receives the plan (NULL on error). */
swih_status swih_plan(const swih_plan_desc *desc, swih_plan_t *out);

/* Steps (1)-(2) of Sec. 1: quantise the image (pixel_type, pitch_bytes from the
 * plan) and build every weighted integral histogram the plan's kernels need:
 *   IH_pq(x, y, b) = sum_{i<=x, j<=y} [Q(f(i,j)) = b] * i^p * j^q   (Eq. 2)
 * d_image: device pointer to H rows of pitch_bytes; read-only.
 * Device-side waits are bounded; a wait that gives up is reported by the next
 * swih_sync_status as SWIH_ERR_TIMEOUT. */
swih_status swih_build_ih(swih_plan_t plan, const void *d_image, void *stream);

/* Steps (3)-(5) of Sec. 1 for a rectangle of centres: the normalised kernel-
 * weighted histogram H_c(b) = U_c(b) / M, U_c(b) the kernel-weighted count of
 * bin b in the window and M the kernel's total window weight.
 * Centres xc in [cx0, cx0+ncx), yc in [cy0, cy0+ncy), all valid.
 * d_hist: float32 [ncy][ncx][B], written. Requires a prior swih_build_ih. */
swih_status swih_local_hist(swih_plan_t plan, int kernel, int win_w, int win_h, int cx0,
                            int cy0, int ncx, int ncy, float *d_hist, void *stream);

/* Steps (3)-(5) of Sec. 1 plus the matching of Sec. 2 / Fig. 3 for every valid
 * centre: L(c) = sum_b sqrt(H_c(b) * q(b)) (Bhattacharyya coefficient).
 * d_target: float32 [B], q(b) >= 0, summing to 1 (not checked on the device).
 * d_map: float32 [H-win_h+1][W-win_w+1], written, row-major.
 * A launch that would leave the GPU partly idle in its last wave splits each
 * window's bins over several CTAs; their partial sums go to a scratch area
 * inside the plan and a second launch adds them in a fixed order (results
 * are deterministic). Calls on one plan therefore must not overlap on the
 * GPU: enqueue them on one stream, or order them with events. */
swih_status swih_likelihood(swih_plan_t plan, int kernel, int win_w, int win_h,
                            const float *d_target, float *d_map, void *stream);

/* Multi-scale search: swih_likelihood for n_windows windows of one kernel
 * (1..SWIH_MAX_SCALES), map i for window win_w[i] x win_h[i] against target
 * d_targets[i] (float32 [B]) into d_maps[i] (float32 [H-win_h[i]+1][W-win_w[i]+1]).
 * win_w, win_h, d_targets and d_maps are host arrays (of device pointers for
 * the last two). The windows of the tiled kernels run as one launch over a job
 * table in the plan (the launch's last wave is a small part of it). The plan
 * keeps the last 8 distinct tables in slots: a call whose table (kernel,
 * windows, targets and maps) equals a slot's enqueues no copy; otherwise the
 * least recently used slot is uploaded with cudaMemcpyAsync on the stream from
 * host memory. So a call can be captured into a CUDA graph once the same call
 * has run uncaptured, and the graph stays valid while the plan's later
 * multi-window calls use at most 7 other distinct tables. The wedding cake, the exponential
 * kernel and Gaussian windows of different fitted degrees run one launch per
 * window. Results equal those of n_windows calls of swih_likelihood up to
 * float rounding (a single-window call may split its bins over CTA groups and
 * add their partial sums in another order). Calls on one plan must not overlap
 * on the GPU (the job table is shared). */
#define SWIH_MAX_SCALES 8
swih_status swih_likelihood_scales(swih_plan_t plan, int kernel, int n_windows, const int *win_w,
                                   const int *win_h, const float *const *d_targets, float *const *d_maps,
                                   void *stream);

/* Wait for the stream, then report the first device-side error the plan
 * recorded since the last call (SWIH_ERR_TIMEOUT) and clear it. */
swih_status swih_sync_status(swih_plan_t plan, void *stream);

/* Free the plan's workspace (synchronises the device). NULL is a no-op. */
swih_status swih_destroy(swih_plan_t plan);

/* Message for the last error on this plan (plan = NULL: the last error of
 * swih_plan / swih_plan_workspace_bytes on this host thread). Never NULL. */
const char *swih_last_error(swih_plan_t plan);

/* Introspection, for tests and tools. All pointers stay owned by the plan. */
typedef struct swih_plan_info {
    int32_t height, width, bins;
    int32_t elem_bytes;      /* 4 (RING32) or 8 (RING64) */
    int32_t n_terms;         /* number of weight terms x^p y^q (up to 81) */
    int32_t term_p[96];      /* term t has weight x^term_p[t] * y^term_q[t] */
    int32_t term_q[96];
    const void *d_bins;      /* uint8 [H][bins_pitch] */
    int64_t bins_pitch;      /* bytes */
    const void *d_ih;        /* plane (t, b) starts at element (t*B + b) * plane_elems */
    int64_t ih_pitch;        /* elements per integral-histogram row */
    int64_t plane_elems;     /* elements per plane (H * ih_pitch) */
    int32_t band_rows;       /* rows per scan band */
    int32_t n_bands;
    uint64_t workspace_bytes;
    /* EXPONENTIAL kernel (NULL / 0 when the plan does not serve it): the four
     * directional integral histograms J_d, d = (x side) + 2 (y side), side 0 =
     * sums over x' <= x (y' <= y), side 1 = over x' >= x (y' >= y), of
     * [bin = b] exp(-lambda (|x - x'| + |y - y'|)); uint64 plane (d, b) starts
     * at element (d*B + b) * plane_elems, rows of ih_pitch elements; the value
     * is element / 2^exp_frac_bits (rounded down at each step of the scan). */
    const void *d_exp;
    int32_t exp_frac_bits;
    /* Rows a plan does not store (bands of at most 64 rows, the default 32,
     * and at most 32767 rows):
     * a row holding no pixel of bin b equals the row above it in every plane
     * of b, so the scan neither computes nor writes it. d_row_map (int32
     * [bins][height]) gives for row y of bin b the row whose stored values
     * hold it (-1: the row is all zero); row y of plane (t, b) is read at row
     * d_row_map[b * height + y]. NULL: every row is stored (band_rows > 64,
     * or more than 32767 rows). */
    const int32_t *d_row_map;
    /* Feature channels (swih_plan_channels; 1 for a plan over one image): the
     * bin plane of channel c is at d_bins + c * height * bins_pitch and holds
     * global bin numbers (channel c's bins follow those of channels 0..c-1). */
    int32_t n_channels;
} swih_plan_info;

swih_status swih_plan_get_info(swih_plan_t plan, swih_plan_info *info);

/* ---------------------------------------------------------------- feature channels
 * Several features per pixel, each with its own likelihood map (Sec. 4: the
 * tracker matches chromatic, shape and texture features, one likelihood map per
 * feature). A channel is one single-valued image of the plan's size with its
 * own pixel type, bit depth, row pitch and bin count B_c, quantised with the
 * equal-width Q of Sec. 2.1 into its own bins. The plan numbers the bins of
 * all channels globally: channel c owns bins [bin0_c, bin0_c + B_c) with bin0_c =
 * B_0 + ... + B_{c-1}, B = sum B_c <= 256. Every pixel falls in exactly one bin
 * of each channel, so every channel's kernel-weighted window histogram has the
 * same total weight M and normalises by it. One quantisation launch per
 * channel, one scan launch for the integral histograms of every bin of every
 * channel, and one gather launch for every channel's map.
 *
 * On a channel plan swih_local_hist returns the histograms over all B global
 * bins (each channel's part sums to 1), and swih_likelihood with a [B] target
 * returns the sum over channels of the per-channel coefficients (targets that
 * sum to 1 per channel). The exponential kernel is not served (UNSUPPORTED). */
#define SWIH_MAX_CHANNELS 8

typedef struct swih_channel_desc {
    int64_t pitch_bytes;       /* row stride in bytes, >= width * pixel size */
    int32_t pixel_type;        /* swih_pixel_type */
    int32_t bitdepth;          /* significant bits, as in swih_plan_desc */
    int32_t bins;              /* B_c >= 1 */
    int32_t reserved;          /* 0 */
} swih_channel_desc;

/* Plan over n_channels (1..SWIH_MAX_CHANNELS) feature channels. From *desc:
 * height, width, kernel_mask, Gaussian settings, windows, precision, band_rows,
 * hbm_budget_bytes, wedding_rings; its bins, pixel_type, bitdepth and
 * pitch_bytes are ignored (taken from the channels). */
swih_status swih_plan_channels(const swih_plan_desc *desc, int n_channels, const swih_channel_desc *channels,
                               swih_plan_t *out);

/* Steps (1)-(2) of Sec. 1 for every channel: d_images is a host array of
 * n_channels device pointers, image c laid out as channels[c] says. */
swih_status swih_build_ih_channels(swih_plan_t plan, const void *const *d_images, void *stream);

/* Steps (3)-(5) and the matching of Fig. 3 for every channel at once:
 * d_maps (float32 [n_channels][H-win_h+1][W-win_w+1], packed, channel-major)
 * receives each channel's map L_c(x) = sum over channel c's bins of
 * sqrt(H_x(b) q(b)). d_target: float32 [B], the channels' target histograms
 * side by side, each channel's part summing to 1 (not checked). The per-channel
 * targets are laid out in a table inside the plan on the stream, so calls on
 * one plan must not overlap on the GPU. */
swih_status swih_likelihood_channels(swih_plan_t plan, int kernel, int win_w, int win_h, const float *d_target,
                                     float *d_maps, void *stream);

/* Kernels this library has enqueued in this process so far, counted on the
 * host at each launch (a CUDA graph's kernels count once, when the graph is
 * captured; replays do not add to it). For reporting how many launches a
 * piece of work took. */
swih_status swih_launch_count(uint64_t *count);

/* Bytes of integral histogram the plan's tiled gathers have requested from
 * device memory since the last reset (each CTA adds the row segments it
 * copied: rows of windows that hold a bin, for bins present in its windows).
 * Synchronous; reset = 1 zeroes the count. For reporting how much data the
 * gathers actually move. */
swih_status swih_plan_load_bytes(swih_plan_t plan, uint64_t *bytes, int reset);

/* ---------------------------------------------------------------- batches
 * Many regions of interest (ROIs) of one frame, each with its own size,
 * kernel, windows (scales), bin count and target histogram, processed by a
 * fixed set of launches per bin count among the ROIs: one quantisation over
 * its ROIs, one integral-histogram scan over them, and one window-gather
 * launch per group of jobs that share a kernel and fitted degree (a job = one
 * ROI at one window). The sequence is captured
 * into a CUDA graph once and replayed by swih_batch_run. This is the paper's
 * search problem (Sec. 1, Sec. 4: likelihood maps for many candidate regions)
 * run for many targets at once; the paper itself processes one region at a
 * time. */
typedef struct swih_batch_desc {
    int32_t height;            /* frame rows */
    int32_t width;             /* frame columns */
    int64_t pitch_bytes;       /* frame row stride in bytes */
    int32_t pixel_type;        /* swih_pixel_type */
    int32_t bitdepth;
    int32_t bins;              /* B of every ROI that does not set its own */
    uint32_t kernel_mask;      /* kernels any ROI may use */
    int32_t gauss_degree;      /* as in swih_plan_desc */
    double gauss_sigma_frac;
    int32_t precision;         /* swih_precision (AUTO: the widest any ROI needs) */
    int32_t band_rows;         /* scan band height (0: automatic) */
    uint64_t hbm_budget_bytes; /* reject batches whose workspace exceeds it (0: no limit) */
} swih_batch_desc;

typedef struct swih_roi_desc {
    int32_t x0, y0;            /* top-left pixel of the ROI in the frame */
    int32_t width, height;     /* ROI size (width <= 8192) */
    int32_t kernel;            /* swih_kernel, must be in kernel_mask */
    int32_t n_windows;         /* 1..SWIH_MAX_SCALES */
    int32_t win_w[SWIH_MAX_SCALES], win_h[SWIH_MAX_SCALES];  /* odd, >= 3, <= ROI size */
    const float *d_target;     /* device float32 [bins], q(b) >= 0 summing to 1 */
    float *d_map[SWIH_MAX_SCALES]; /* device float32 [height-win_h+1][width-win_w+1] each */
    int32_t bins;              /* B of this ROI, 1..256 (0: the batch's bins); ROIs of each
                                  bin count form one work set (its own three launches) */
    int32_t reserved;          /* 0 */
} swih_roi_desc;

typedef struct swih_batch_s *swih_batch_t;

/* Workspace a batch would allocate (host only). */
swih_status swih_batch_workspace_bytes(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois,
                                       uint64_t *bytes);

/* Validate, lay out and allocate a batch over the frame d_frame (device,
 * height rows of pitch_bytes, owned by the caller, read at every run; the
 * caller may rewrite its contents between runs). Targets and maps are the
 * caller's and are bound to the batch. One integral-histogram term set and
 * one ring serve every ROI: those a plan for the largest ROI with the largest
 * window of any ROI would pick, so every ROI's results are exact in it.
 * Errors of the batch calls are reported by swih_last_error(NULL) on the
 * calling thread. SWIH_ERR_BUDGET when the workspace exceeds hbm_budget_bytes. */
swih_status swih_batch_plan(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois,
                            const void *d_frame, swih_batch_t *out);

/* Enqueue one pass over every ROI and window on the stream: a replay of the
 * batch's CUDA graph (captured at the first run, and again after
 * swih_batch_autotune). Maps are written; nothing is synchronised. */
swih_status swih_batch_run(swih_batch_t batch, void *stream);

/* Time candidate gather launch shapes (tile width, copy-ring depth, bins per
 * step) for each job group on this batch's own data, keep the fastest, and
 * capture the graph again. Synchronises the stream; results are unchanged. */
swih_status swih_batch_autotune(swih_batch_t batch, void *stream);

/* As swih_sync_status, for a batch. */
swih_status swih_batch_sync_status(swih_batch_t batch, void *stream);

/* Free the batch (synchronises the device). NULL is a no-op. */
swih_status swih_batch_destroy(swih_batch_t batch);

/* Launch shape of the tiled window gather for one kernel of this plan:
 * tile_cols = centre columns per CTA (128 or 256; 0 = automatic), stages =
 * depth of the shared-memory copy ring (2..8; 0 = automatic, the deepest that
 * keeps the register-limited number of CTAs resident), bins_per_step = bins
 * carried per pipeline step by the plain, Manhattan and Euclidean kernels
 * (2, 4 or 8; 2 only with 256 columns and 32-bit elements, else 4 is used;
 * 0 = automatic; the Gaussian always carries one). A shape whose row
 * segments do not fit falls back to the automatic choice, then to the direct
 * gather. Results do not depend on the shape; only speed does. */
swih_status swih_set_gather_config(swih_plan_t plan, int kernel, int tile_cols, int stages,
                                   int bins_per_step);

/* Integral-histogram build for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface for hosts whose memory
 * rules forbid cudaMalloc at call time -- pipelines that give all device
 * memory to a fixed pool at start-up, real-time loops that may not take the
 * device-wide synchronisation a driver allocation can cause, or allocators
 * that refuse driver allocations after start-up.
 * Such callers cannot create a plan (swih_plan allocates a workspace).
 *
 * Computes exactly what swih_build_ih computes for a plan made from *desc,
 * into caller-owned memory: d_ih receives every weighted integral histogram
 * in the same layout as a plan's (plane (t, b) at element (t*B + b) *
 * plane_elems, rows of ih_pitch elements of elem_bytes each). The bins, the
 * scan's look-back state, its tile flags and its status word live in one
 * static device array of 8 MiB (8388608 bytes) inside the library, which
 * every GPU that loads the library holds until the process exits. Inputs
 * whose scratch (bins + look-back state, reported nowhere else) exceeds it
 * are rejected with SWIH_ERR_UNSUPPORTED and a message giving the size, and so
 * is a desc naming the EXPONENTIAL kernel (its tables are not built here); when
 * desc->band_rows is 0 the band height is raised until the state fits.
 *
 * Arguments:
 *   desc      plan description (hbm_budget_bytes is ignored)
 *   d_image   device image as for swih_build_ih
 *   d_ih      device output, 16-byte aligned, ih_bytes long; NULL = size
 *             query: fill *layout and return without enqueueing device work
 *   ih_bytes  capacity of d_ih; must be >= layout->workspace_bytes
 *   d_status  optional device uint32 the scan ORs its error bits into
 *             (1 = a bounded look-back wait gave up); the caller clears it.
 *             NULL: a word inside the static array is used (cleared per call)
 *             and such an error is not reported.
 *   layout    optional host struct, filled with the layout: elem_bytes,
 *             terms, pitches, plane_elems, and in workspace_bytes the bytes
 *             d_ih must hold; d_bins points into the static array (valid until
 *             the next call) and d_ih echoes the argument.
 *   stream    as for swih_build_ih
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine. The first
 * call on each device, a size query included, looks up the static array's
 * device address (cudaGetSymbolAddress) with that device current and caches
 * it; make that first call before any stream capture begins. A call that
 * cannot look the address up (no usable device) returns SWIH_ERR_CUDA. Every call shares the one
 * array and leaves its contents behind; the tile flags are cleared at each
 * call. Calls whose work overlaps on the GPU (other streams, other host
 * threads) race on the array and must be serialised by the caller. */
swih_status swih_build_ih_noalloc(const swih_plan_desc *desc, const void *d_image, void *d_ih,
                                  uint64_t ih_bytes, uint32_t *d_status, swih_plan_info *layout,
                                  void *stream);

/* Fault injection for tests (host-set, no device fault): with
 * SWIH_INJECT_STALL_SCAN_TILE the next swih_build_ih runs its scan with the
 * first band of the first (bin, term) chain never publishing its column sums,
 * and with a short wait bound. The bands below it give up waiting after the
 * bound, mark themselves failed and return; the next swih_sync_status then
 * returns SWIH_ERR_TIMEOUT and the plan's integral histograms are invalid until
 * the next swih_build_ih. The injection applies to one build only.
 * SWIH_INJECT_DIRECT_GATHER routes the plan's gathers through the direct
 * kernel (one thread per centre, corner reads from global memory) instead of
 * the tiled one, until cleared; results are the same, only speed differs.
 * what = 0 clears both. */
#define SWIH_INJECT_STALL_SCAN_TILE 1
#define SWIH_INJECT_DIRECT_GATHER 2
swih_status swih_debug_inject(swih_plan_t plan, int what);

/* ---------------------------------------------------------------- streamed frames
 * Likelihood maps over a frame whose integral histograms do not fit in device
 * memory at once (the paper's wide-area imagery, Sec. 4). The frame is cut
 * into bands of band_height centre rows; a band's integral histograms cover
 * its rows plus a halo of (tallest window - 1) rows, are built, gathered for
 * every job's centres in the band and then overwritten by the next band's.
 * Results equal those of one plan over the whole frame (integer integral
 * histograms are exact at any origin). Frames wider than 8192 columns are
 * also cut into column tiles of at most 8192 columns (a halo of the widest
 * window - 1 columns); each piece's maps are computed into a scratch area of
 * the workspace and copied into the frame-sized maps. The pass over all
 * pieces is captured into a CUDA graph at the first run. */
typedef struct swih_frame_job {
    int32_t kernel;             /* swih_kernel, in the desc's kernel_mask */
    int32_t win_w, win_h;       /* odd, >= 3 */
    const float *d_target;      /* device [bins] */
    float *d_map;               /* device [(height - win_h + 1) x (width - win_w + 1)], the frame's valid map */
} swih_frame_job;

typedef struct swih_stream_s *swih_stream_t;

/* Plan a streamed pass over the frame d_image (device, desc->height rows of
 * desc->pitch_bytes, caller-owned, read at every run; the caller may rewrite
 * its contents between runs). desc->max_win_w/max_win_h are ignored (taken
 * from the jobs); desc->band_rows is the scan's band height as for plans.
 * band_height = centre rows per band; 0 picks the largest that keeps the
 * workspace within desc->hbm_budget_bytes (which must then be set).
 * SWIH_ERR_BUDGET when even 1-row bands do not fit. */
swih_status swih_stream_plan(const swih_plan_desc *desc, const swih_frame_job *jobs, int n_jobs,
                             const void *d_image, int32_t band_height, swih_stream_t *out);

/* Enqueue one pass (every band, every job) on the stream. */
swih_status swih_stream_run(swih_stream_t st, void *stream);

/* Host copies of the maps, made during the pass: h_maps[j] (host memory of
 * job j's whole valid map, (height - win_h + 1) x (width - win_w + 1) floats,
 * caller-owned and page-locked: the copies are part of the pass's graph)
 * receives each band's rows of job j's map as soon as the band's gathers (and
 * column-tile copies) are done, on a second branch of the pass's graph, while
 * the next band computes; the pass (swih_stream_run) completes when every
 * copy has. NULL
 * h_maps (or a NULL entry) turns the copies off (for that job). Takes effect
 * at the next swih_stream_run (the pass is captured again); the host buffers
 * must stay valid while passes that copy into them run. Not used by
 * swih_stream_run_timed. */
swih_status swih_stream_set_host_maps(swih_stream_t st, float *const *h_maps);

/* One pass as swih_stream_run, for measurement: the bands' launches are
 * enqueued one by one (not as the graph) with CUDA events between stages, the
 * stream is synchronised, and stage_ms (7 floats) receives milliseconds summed
 * over the bands: stage_ms[0] = table upload + quantise + scan + row map,
 * stage_ms[1 + k] = the window gathers of kernel k (swih_kernel, 0..5).
 * Results are those of swih_stream_run. */
swih_status swih_stream_run_timed(swih_stream_t st, void *stream, float *stage_ms);

/* Integral-histogram bytes the tiled gathers of this streamed pass requested
 * since the last reset (as swih_plan_load_bytes), per kernel: bytes[k] for
 * swih_kernel k = 0..4 (5 entries). Synchronises the device; reset = 1 zeroes
 * the counts. */
swih_status swih_stream_load_bytes(swih_stream_t st, uint64_t *bytes, int reset);

/* As swih_sync_status, for a streamed pass. */
swih_status swih_stream_sync_status(swih_stream_t st, void *stream);

/* Band height, band count and device workspace of a streamed pass. */
swih_status swih_stream_get_info(swih_stream_t st, int32_t *band_height, int32_t *n_bands,
                                 uint64_t *workspace_bytes);

/* Free it (synchronises the device). NULL is a no-op. */
swih_status swih_stream_destroy(swih_stream_t st);

/* ---------------------------------------------------------------- serving
 * A server answers tracking queries (a crop of a resident frame, B, a kernel,
 * 1..8 target histograms and 1..SWIH_MAX_SCALES windows) as they arrive. A
 * scheduler thread inside the library admits waiting queries in micro-batches
 * as stream slots and device memory free up (continuous batching): queries
 * that share a frame, B and kernel run as one work set whose overlapping
 * crops share integral histograms (merged only where that adds no pixels),
 * and each micro-batch runs on its own stream, so micro-batches overlap on
 * the device. All device memory the work needs comes from one arena of
 * hbm_budget_bytes allocated at creation; a query waits until its work fits
 * and is refused at submission if it can never fit. Results do not depend on
 * which other queries share a micro-batch (integer integral histograms are
 * exact wherever their origin lies). Errors of the server calls are reported
 * by swih_last_error(NULL) on the calling thread. */
typedef struct swih_server_s *swih_server_t;

typedef struct swih_server_desc {
    uint64_t hbm_budget_bytes;  /* device arena for work (bins, IHs, scan state, tables) */
    int32_t max_inflight;       /* micro-batches on the device at once, 1..32 (one stream each) */
    int32_t max_batch_queries;  /* queries admitted into one micro-batch, >= 1 */
    int32_t merge_regions;      /* 1: overlapping crops of one frame share integral histograms */
    int32_t gauss_degree;       /* as in swih_plan_desc */
    double gauss_sigma_frac;
    uint64_t staging_bytes;     /* pinned host staging for job tables (0: 64 MiB) */
    int32_t keep_ih;            /* 1: keep built integral histograms resident in the arena after
                                   their micro-batch; a later query whose crop lies inside a
                                   resident region of the same frame (same pixel type, bit
                                   depth, B and term set) skips quantisation and scan. Resident
                                   regions nobody reads are evicted, least recently used first,
                                   when the arena is needed. */
    int32_t reserved;           /* 0 */
} swih_server_desc;

typedef struct swih_frame_desc {
    const void *d_pixels;       /* device frame, owned by the caller, read by every query on it */
    int32_t height, width;
    int64_t pitch_bytes;
    int32_t pixel_type;         /* swih_pixel_type */
    int32_t bitdepth;
} swih_frame_desc;

#define SWIH_MAX_TARGETS 8

typedef struct swih_query {
    int32_t frame;              /* id returned by swih_server_add_frame */
    int32_t x0, y0, width, height;  /* crop, inside the frame, width <= 8192 */
    int32_t bins;               /* B, 1..256 */
    int32_t kernel;             /* swih_kernel */
    int32_t n_targets;          /* 1..SWIH_MAX_TARGETS */
    int32_t n_scales;           /* 1..SWIH_MAX_SCALES */
    int32_t win_w[SWIH_MAX_SCALES], win_h[SWIH_MAX_SCALES];  /* odd, >= 3, <= crop */
    const float *d_targets;     /* device [n_targets][bins] */
    float *d_out;               /* device: n_targets * n_scales maps, target-major, each
                                   (height - win_h + 1) x (width - win_w + 1), packed */
    uint64_t user_tag;          /* returned in the completion */
} swih_query;

typedef struct swih_completion {
    uint64_t id;                /* from swih_server_submit */
    uint64_t user_tag;
    int32_t status;             /* swih_status of the query's work */
    int32_t batch_queries;      /* queries in its micro-batch */
    uint64_t submit_ns, start_ns, done_ns;  /* steady-clock (CLOCK_MONOTONIC) times */
    int32_t ih_reused;          /* 1: the query's integral histograms were resident (no K1, K2) */
    int32_t reserved;
} swih_completion;

/* Counters of a server since its creation. */
typedef struct swih_server_stats {
    uint64_t queries;           /* queries completed by micro-batches */
    uint64_t ih_reused;         /* of them, served from resident integral histograms */
    uint64_t regions_built;     /* crop regions quantised and scanned */
    uint64_t evictions;         /* resident blocks evicted to make room */
    uint64_t resident_bytes;    /* arena bytes held by resident integral histograms now */
} swih_server_stats;

/* Create a server on the current device: allocates the arena and staging
 * and starts the scheduler thread. */
swih_status swih_server_create(const swih_server_desc *desc, swih_server_t *out);

/* Register a resident frame; *frame_id is its handle for queries. The caller
 * may rewrite the pixels between queries (not while queries on it run; with
 * keep_ih, call swih_server_frame_changed afterwards). */
swih_status swih_server_add_frame(swih_server_t server, const swih_frame_desc *frame, int32_t *frame_id);

/* Floats d_out must hold for a query (host only, no server needed). */
swih_status swih_query_out_elems(const swih_query *query, uint64_t *elems);

/* Arena bytes the query needs when it runs alone (host only). */
swih_status swih_server_query_bytes(swih_server_t server, const swih_query *query, uint64_t *bytes);

/* Validate and queue a query; returns at once. SWIH_ERR_BUDGET when the
 * query alone needs more than the arena. */
swih_status swih_server_submit(swih_server_t server, const swih_query *query, uint64_t *id);

/* Move up to max completions into out (*n of them), waiting up to wait_us
 * microseconds for the first when none is ready. */
swih_status swih_server_poll(swih_server_t server, swih_completion *out, int32_t max, int32_t *n,
                             int32_t wait_us);

/* Cancel a query that is still waiting for admission: it completes at once
 * with status SWIH_ERR_CANCELLED and nothing of it runs. A query already
 * admitted (or finished, or unknown) is left alone and SWIH_ERR_INVALID_ARG
 * is returned. */
swih_status swih_server_cancel(swih_server_t server, uint64_t id);

/* The pixels of a frame were rewritten: its resident integral histograms are
 * dropped before any query submitted after this call is admitted. Call it
 * after rewriting the pixels and before submitting queries on the new
 * contents, with no query on the frame still waiting or running (with
 * keep_ih = 0 it is not needed). */
swih_status swih_server_frame_changed(swih_server_t server, int32_t frame_id);

/* Counters of the server (queries served, resident reuse, evictions). */
swih_status swih_server_get_stats(swih_server_t server, swih_server_stats *stats);

/* Block until every submitted query has completed (completions stay queued
 * for swih_server_poll). */
swih_status swih_server_drain(swih_server_t server);

/* Drain, stop the scheduler and free the server. NULL is a no-op. */
swih_status swih_server_destroy(swih_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* SWIH_H */
