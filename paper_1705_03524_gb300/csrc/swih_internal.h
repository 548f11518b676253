// Internal declarations shared by the CUDA translation units of libswih.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace swih {

constexpr int kMaxQ = 9;          // distinct y-exponents q of a plan (Gaussian of degree D: 0..2D, D <= 4)
constexpr int kMaxP = 9;          // x-exponents p per q
constexpr int kMaxTerms = 25;     // terms a tiled or table gather reads (Gaussian D <= 2)
constexpr int kMaxPlanTerms = 81; // terms of a plan (Gaussian D = 4: x^p y^q, p, q <= 8)
constexpr int kMaxScanThreads = 512;

// decoupled look-back tile states
constexpr int kFlagEmpty = 0;
constexpr int kFlagAggregate = 1;
constexpr int kFlagInclusive = 2;
constexpr int kFlagError = 3;

// bits of the plan's device status word
constexpr uint32_t kStatusTimeout = 1u;

// ---------------------------------------------------------------- K1 quantise
struct QuantParams {
    const uint8_t *image;
    int64_t pitch;       // bytes
    int H, W;
    int B, bitdepth;
    uint8_t *bins;
    int64_t bins_pitch;  // bytes, multiple of 16
    int pixel_bytes;     // 1 or 2
    int vec;             // 1 when every 16-pixel chunk can use aligned vector loads
    int bin0 = 0;        // added to every bin: a feature channel's first bin (B + bin0 <= 256)
};
cudaError_t launch_quantize(const QuantParams &p, cudaStream_t s);

// One image region of a batched quantisation.
struct QuantRoi {
    const uint8_t *image;  // first pixel of the region
    int64_t pitch;         // bytes
    int H, W;
    uint8_t *bins;
    int64_t bins_pitch;
    long long chunk0;      // first 16-pixel chunk of the region; regions in chunk order
    int vec;               // aligned 16-byte loads allowed
};
cudaError_t launch_quantize_table(const QuantRoi *d_table, int n, long long n_chunks, int B, int bitdepth,
                                  int pixel_bytes, cudaStream_t s);

// ---------------------------------------------------------------- K2 scan
// One chain per (bin b, y-exponent q); a chain's bands are scanned top to
// bottom with decoupled look-back on per-column state vectors.
struct ScanParams {
    const uint8_t *bins;
    int64_t bins_pitch;  // bytes
    void *ih;            // planes [t][b][H][ih_pitch]
    int64_t ih_pitch;    // elements
    int64_t plane;       // elements per plane
    void *agg;           // [chain][band][ih_pitch] band aggregates
    void *incl;          // [chain][band][ih_pitch] inclusive column sums
    int *flags;          // [chain][band]
    int *ticket;         // tile counter (zeroed before each launch)
    uint32_t *status;
    int H, W, B;
    int band_rows, n_bands;
    int n_q;
    int q_val[kMaxQ];
    int p_count[kMaxQ];
    int p_val[kMaxQ][kMaxP];
    int term[kMaxQ][kMaxP];
    long long spin_limit;
    int sb_rows;            // band rows whose bins the tile keeps in shared memory (set by the launcher)
    int stall_tile;      // ticket of a tile that never publishes (fault injection), else -1
    // Sparse rows (single-plan scan, band_rows <= 64): a row without a pixel of
    // bin b equals the row above in every plane of b, so it is neither computed
    // nor stored; occ[b * n_bands + band] receives the band's mask of stored rows
    // (bit r: band row r holds bin b). NULL: every row is stored.
    unsigned long long *occ;
    // Feature channels (several bin planes per pixel): bin b's chain reads the
    // bin plane bins + ch_of_bin[b] * ch_stride, whose pixels carry the global
    // bin numbers of one channel. ch_stride = 0: one plane.
    int64_t ch_stride;
    uint8_t ch_of_bin[256];
};
// row_map[b * H + y] = the last stored row <= y of bin b's planes (-1: none, the
// row is all zero), from the occupancy words of a sparse-row scan
cudaError_t launch_row_map(const unsigned long long *occ, int *row_map, int B, int H, int band_rows, int n_bands,
                           cudaStream_t s);
// E = columns per thread, threads = ceil(W/E) rounded to a warp multiple;
// elem_bytes 4, 8 or 16 (the 128-bit ring: E <= 8)
cudaError_t launch_ih_scan(const ScanParams &p, int elem_bytes, int E, int threads,
                           cudaStream_t s);
// the same for chains of more than 5 x-exponents or 16-byte elements (one plan)
cudaError_t launch_ih_scan_wide(const ScanParams &p, int elem_bytes, int E, int threads, cudaStream_t s);

// The per-region fields of a scan (one entry per image region of a batch).
struct ScanRoi {
    const uint8_t *bins;
    int64_t bins_pitch;
    void *ih;
    int64_t ih_pitch, plane;
    void *agg, *incl;
    int *flags;
    int H, W, n_bands;
    int ticket0;  // first ticket of the region; regions are in ticket order
    // sparse rows (when the launch's p.occ is non-NULL): the region's
    // occupancy words [b][band] and row map [b][H]
    unsigned long long *occ;
    int *row_map;
};
// One launch over several regions sharing B, terms, ring and band height;
// p carries those plus ticket/status/spin_limit; tiles = total tiles. A
// non-NULL p.occ selects sparse rows (each region's own occ is used).
cudaError_t launch_ih_scan_table(const ScanParams &p, const ScanRoi *d_table, int n_roi, long long tiles,
                                 int elem_bytes, int E, int threads, cudaStream_t s);
// The row maps of every region of a sparse table scan (table[i].occ ->
// table[i].row_map), one launch.
cudaError_t launch_row_map_table(const ScanRoi *d_table, int n_roi, int B, int band_rows, cudaStream_t s);

// ---------------------------------------------------------------- K2e scan
// The exponential kernel's four directional integral histograms J_d (Sec. 2.1
// with the weights exp(+-lambda x) exp(+-lambda y), divided by the weight at
// the point), in unsigned 64-bit fixed point with `one` = 2^F. A chain is
// (bin b, y side s): its column-filtered values C(x, y) = [bin = b] one +
// q C(x, y -+ 1) are shared by both x sides, whose rows are prefix scans of C
// with the decay q = exp(-lambda). Three launches: band aggregates of C,
// carries into each band (a sequential pass over the bands per column), and
// the scan that writes J. q^n is kept as floor(q^n 2^64) and applied as the
// high half of a 64 x 64-bit product.
constexpr int kExpMaxE = 16;
struct ExpScanParams {
    const uint8_t *bins;
    int64_t bins_pitch;        // bytes
    unsigned long long *J;     // planes [d][b][H][pitch], d = x side + 2 y side
    int64_t pitch, plane;      // elements
    unsigned long long *carry; // [s][b][band][pitch]: band aggregates, then carries into bands
    unsigned long long *rows;  // [s][b][band]: bit r = the band's r-th row in scan order holds bin b
    unsigned long long qrow[65]; // floor(q^d 2^F) = one * q^d, d = 0..64 (band aggregates)
    int H, W, B;
    int band_rows, n_bands;
    int E, threads;            // columns per scan thread, threads per block
    unsigned long long one;    // 2^F
    unsigned long long q1;     // q
    unsigned long long qband;  // q^band_rows
    unsigned long long qe[33];  // q^(E d), d = 1..32
    unsigned long long qw[17];  // q^(32 E d), d = 1..16
};
cudaError_t launch_exp_scan(const ExpScanParams &p, cudaStream_t s);

// One exponential-kernel gather: a thread per centre; per bin, the exact
// window count from the plain integral histogram (ring element type T) gates
// the 16 corner reads of the four J_d.
struct ExpGatherParams {
    const void *count;           // plain IH plane of bin b at count + b * plane (ring elements)
    const int *row_map;          // [b][H] stored row holding row y of the count plane (-1: zero); NULL: identity
    const unsigned long long *J; // as ExpScanParams::J
    int64_t pitch, plane;        // elements (shared by both)
    int B, H, W, rx, ry;
    int cx0, cy0, ncx, ncy;
    const float *target;         // [B] or NULL
    float *map;                  // [ncy][ncx] or NULL
    float *hist;                 // [ncy][ncx][B] or NULL
    unsigned long long qx1, qx0, qy1, qy0, q1;  // q^(rx+1), q^rx, q^(ry+1), q^ry, q
    float scale;                 // 2^-F / M
};
cudaError_t launch_exp_gather(const ExpGatherParams &p, int elem_bytes, cudaStream_t s);

// ---------------------------------------------------------------- K3 gather
enum GatherKind { kGatherPlain = 0, kGatherManhattan = 1, kGatherEuclidean = 2, kGatherGaussian = 3, kGatherWedding = 4 };
constexpr int kMaxRings = 16;

struct GatherParams {
    const void *ih;
    const int *row_map;     // [b][H]: row whose stored values hold row y of bin b (-1: zero); NULL: identity
    int64_t plane, pitch;   // elements
    int B, H, W;
    int rx, ry;
    int cx0, cy0, ncx, ncy; // centre rectangle
    // term (plane-group) indices
    int t1, tx, ty, txx, tyy;
    int tg[5][5];           // Gaussian: term index of x^k y^l
    int gdx, gdy;           // Gaussian: fitted degree per axis (1 or 2)
    unsigned long long rx2, rx4, ry2, ry4;  // r^2, r^4 per axis (ring constants)
    float gamma[3][3];      // Gaussian: beta_x[i] beta_y[j] / (rx^2Dx ry^2Dy M)
    float inv_mass;         // 1 / M (plain, Manhattan, Euclidean, wedding cake)
    int n_rings;            // wedding cake: nested windows, half-sides and weights
    int ring_rx[kMaxRings], ring_ry[kMaxRings];
    float ring_c[kMaxRings];  // weight of ring i minus weight of ring i+1
    const float *target;    // [n_targets][target_stride] (first B of each row used) or null
    float *map;             // n_targets maps of [ncy][ncx], map_stride floats apart, or null
    int n_targets;          // 1..kMaxTargets: one histogram per window, scored against each
    int64_t target_stride, map_stride;
    float *hist;            // [ncy][ncx][B] or null
    // tiled gather only
    uint32_t *status;       // error bits (bounded waits)
    int load_even[kMaxTerms], n_load_even;  // planes copied per corner row
    int load_odd[kMaxTerms], n_load_odd;    // planes copied per centre row (Manhattan)
    int nl;                 // shared-memory slots per stage (max of the two)
    int seg, stage_off;     // set by the launcher
    int dtop_off;           // Gaussian carried differences (set by the launcher)
    int nstage;             // shared-memory stages in the copy ring (set by the launcher)
    int want_stages;        // requested ring depth (0: default)
    int want_tx;            // requested tile width, 128 or 256 (0: default)
    int want_bb;            // requested bins per pipeline step, 4 or 8 (0: default)
    int kchain, nblk;       // windows per chain, chains per phase (set by the launcher)
    int nbg;                // bin groups: CTAs that split a chain's bins (1: one CTA, writes the map)
    float *partial;         // nbg > 1: per-group likelihoods [nbg][n_targets][ncy][ncx], then summed
    int64_t partial_cap;    // floats available at partial (0: no splitting)
    unsigned long long *load_bytes;  // optional: integral-histogram bytes the tiled gather requested (added)
};
cudaError_t launch_gather(const GatherParams &p, int kind, int elem_bytes, cudaStream_t s);

// Gaussian approximant of any fitted degree (1..4 per axis) in the 64- or
// 128-bit ring: one thread per centre, corner reads from global memory (the
// term planes of degrees above 2 do not fit the tiled gather's shared memory).
// Per bin: the exact window count (x^0 y^0 plane) gates the bin; the window's
// raw moments sum x^a y^b are translated to the centre (a Taylor shift in x per
// y-power, binomial sums in y), combined into the Bernstein moments
// F_ij = sum A_i(dx) B_j(dy), A_i(d) = sum_k ax[i][k] d^2k, exact in the ring,
// and U = sum_ij gamma_ij F_ij in double from the non-negative F_ij.
constexpr int kWideMaxD = 4;
struct GaussWideParams {
    const void *ih;
    const int *row_map;          // [b][H] (-1: zero row), or NULL
    int64_t plane, pitch;        // elements
    int B, H, W, rx, ry;
    int cx0, cy0, ncx, ncy;
    int dx, dy;                  // fitted degree per axis
    int tg[2 * kWideMaxD + 1][2 * kWideMaxD + 1];  // term index of x^a y^b
    unsigned long long ax_lo[kWideMaxD + 1][kWideMaxD + 1], ax_hi[kWideMaxD + 1][kWideMaxD + 1];
    unsigned long long ay_lo[kWideMaxD + 1][kWideMaxD + 1], ay_hi[kWideMaxD + 1][kWideMaxD + 1];
    double gamma[kWideMaxD + 1][kWideMaxD + 1];  // beta_x[i] beta_y[j] / (rx^2dx ry^2dy M)
    const float *target;         // [n_targets][target_stride] or NULL
    float *map;                  // n_targets maps [ncy][ncx], map_stride apart, or NULL
    float *hist;                 // [ncy][ncx][B] or NULL
    int n_targets;
    int64_t target_stride, map_stride;
};
cudaError_t launch_gauss_wide(const GaussWideParams &p, int elem_bytes, cudaStream_t s);

// kernels this library has enqueued in the process (host count, for reporting)
void count_launches(unsigned n);

// Tiled gather; returns cudaErrorNotSupported when a window's row segments do
// not fit in shared memory (the caller then uses launch_gather).
constexpr int kTiledChainMax = 8;
constexpr int kTiledRowSlots = kTiledChainMax + 1;  // lattice rows of a chain (K + 1, or 2 K + 1 with K <= 4)
constexpr int kTiledMaxRows = 32767;  // the tiled gather keeps rows as int16; taller images use the direct one
constexpr int kMaxTargets = 8;
cudaError_t launch_gather_tiled(const GatherParams &p, int kind, int elem_bytes, cudaStream_t s);

// Shape shared by every job of one tiled-gather launch: shared-memory layout
// and copy ring (a job = one kernel, window and centre rectangle over one set
// of integral histograms).
struct GatherShape {
    int tx;          // centre columns per CTA (128 or 256)
    int bb;          // bins per pipeline step
    int seg, nl, nstage, stage_off, dtop_off;
    int kchain_max;  // windows per chain
    int n_targets;   // likelihood accumulators per window (largest n_targets of the jobs)
    int ctas_per_sm; // resident CTAs per SM this shape allows (registers, shared memory, threads)
    size_t smem;     // dynamic shared memory bytes
};
// Shape for jobs of one kind with the given fitted degrees, largest window
// width and bin count; cudaErrorNotSupported when nothing fits. row_map: the
// launch reads rows through a row map (single-plan launches), which takes a
// table of B x kTiledRowSlots int16 in shared memory.
cudaError_t tiled_shape(int kind, int elem_bytes, int gdx, int gdy, int max_w, int B, int nl_per_bin,
                        int n_targets, int want_tx, int want_stages, int want_bb, bool row_map, GatherShape *shape);
// Fill a job's shape fields and chain split; returns its number of work items
// (column tiles x chains).
int tiled_items(GatherParams *job, const GatherShape &shape);
// One launch over a device table of jobs (all with the shape's fields set and
// the same B): one CTA per work item; item_start[j] = first item of job j.
cudaError_t launch_gather_table(const GatherParams *d_jobs, const int *d_item_start, int n_jobs,
                                int n_items, const GatherParams &shape_job, int kind, int elem_bytes,
                                int gdx, int gdy, const GatherShape &shape, cudaStream_t s);

// ---------------------------------------------------------------- layout of a description
// What a plan built from a description would use, computed on the host without
// allocating anything.
struct PlanLayout {
    int elem_bytes, n_terms;
    int term_p[kMaxPlanTerms], term_q[kMaxPlanTerms];
    int n_q;
    int q_val[kMaxQ], p_count[kMaxQ], p_val[kMaxQ][kMaxP], term[kMaxQ][kMaxP];
    int64_t bins_pitch, ih_pitch, plane;
    int band_rows, n_bands, scan_E, scan_threads;
};

}  // namespace swih
