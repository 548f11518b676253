// Host side of the C ABI declared in include/swih.h: plan construction,
// argument validation, kernel parameters and launches. No compute happens
// here; every step of the pipeline runs in the CUDA kernels K1-K3.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "swih.h"
#include "swih_host.h"
#include "swih_internal.h"

using namespace swih;


namespace swih {

thread_local std::string g_err;

// bytes of one job-table slot of swih_likelihood_scales (256-byte multiple)
constexpr uint64_t kJobSlotBytes =
    (sizeof(GatherParams) * SWIH_MAX_SCALES + sizeof(int) * (SWIH_MAX_SCALES + 1) + 255) / 256 * 256;

std::string &thread_error() { return g_err; }

swih_status fail(swih_plan_s *plan, swih_status st, const std::string &msg)
{
    if (plan)
        plan->err = msg;
    else
        g_err = msg;
    return st;
}

swih_status cuda_fail(swih_plan_s *plan, const char *what, cudaError_t e)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(plan, e == cudaErrorMemoryAllocation ? SWIH_ERR_OOM : SWIH_ERR_CUDA, m);
}

// total kernel weight over a w x h window, for the integer-valued kernels
long double int_kernel_mass(int kernel, int w, int h)
{
    const long double rx = (w - 1) / 2, ry = (h - 1) / 2;
    switch (kernel) {
    case SWIH_KERNEL_PLAIN: return (long double)w * h;
    case SWIH_KERNEL_MANHATTAN: return h * rx * rx + w * ry * ry;
    case SWIH_KERNEL_EUCLIDEAN:
        return h * rx * (2 * rx + 1) * (2 * rx - 1) / 3 + w * ry * (2 * ry + 1) * (2 * ry - 1) / 3;
    default: return 0;
    }
}

int gauss_axis_degree(int r, int D) { return std::max(0, std::min(D, r)); }

// Least-squares fit of P(t) = sum_i c_i t^i (i <= D) to exp(-d^2 / (2 s^2)) on the
// integer samples d = -r..r with t = d^2 / r^2: normal equations solved by
// Gaussian elimination with partial pivoting, in double.
bool gauss_fit(int r, double sigma, int D, double *c)
{
    const int n = D + 1;
    double A[kWideMaxD + 1][kWideMaxD + 2] = {};
    for (int d = -r; d <= r; ++d) {
        const double t = (double)d * d / ((double)r * r);
        const double y = std::exp(-(double)d * d / (2.0 * sigma * sigma));
        double pw[kWideMaxD + 1];
        pw[0] = 1.0;
        for (int i = 1; i < n; ++i) pw[i] = pw[i - 1] * t;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) A[i][j] += pw[i] * pw[j];
            A[i][n] += pw[i] * y;
        }
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r2 = col + 1; r2 < n; ++r2)
            if (std::fabs(A[r2][col]) > std::fabs(A[piv][col])) piv = r2;
        if (A[piv][col] == 0.0) return false;
        if (piv != col)
            for (int k = 0; k <= n; ++k) std::swap(A[piv][k], A[col][k]);
        for (int r2 = col + 1; r2 < n; ++r2) {
            const double f = A[r2][col] / A[col][col];
            for (int k = col; k <= n; ++k) A[r2][k] -= f * A[col][k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = A[i][n];
        for (int k = i + 1; k < n; ++k) s -= A[i][k] * c[k];
        c[i] = s / A[i][i];
    }
    return true;
}

double binom(int n, int k)
{
    double v = 1.0;
    for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
    return v;
}

struct GaussAxis {
    int D = 0;
    double beta[kWideMaxD + 1] = {};  // Bernstein coefficients of the fitted polynomial
    double mass = 0;                  // sum over d = -r..r of P(d^2 / r^2)
};

bool gauss_axis(int r, double sigma, int D_req, GaussAxis &g, std::string &why)
{
    g.D = gauss_axis_degree(r, D_req);
    double c[kWideMaxD + 1] = {};
    if (g.D < 1) {
        why = "Gaussian window half-size must be >= 1";
        return false;
    }
    if (!gauss_fit(r, sigma, g.D, c)) {
        why = "Gaussian least-squares system is singular";
        return false;
    }
    // power basis -> Bernstein basis: beta_i = sum_{k<=i} C(i,k)/C(D,k) c_k
    for (int i = 0; i <= g.D; ++i) {
        g.beta[i] = 0.0;
        for (int k = 0; k <= i; ++k) g.beta[i] += binom(i, k) / binom(g.D, k) * c[k];
    }
    for (int i = 0; i <= g.D; ++i)
        if (!(g.beta[i] >= 0.0)) {
            why = "Gaussian approximant has a negative Bernstein coefficient for this window";
            return false;
        }
    g.mass = 0.0;
    for (int d = -r; d <= r; ++d) {
        const double t = (double)d * d / ((double)r * r);
        double v = 0.0;
        for (int i = g.D; i >= 0; --i) v = v * t + c[i];
        g.mass += v;
    }
    return true;
}

// Largest Bernstein moment of the Gaussian path, w h rx^2Dx ry^2Dy: it must fit
// the 64-bit ring for the per-window integers to be exact.
long double gauss_bound(int w, int h, int D)
{
    const int rx = (w - 1) / 2, ry = (h - 1) / 2;
    const int dx = gauss_axis_degree(rx, D), dy = gauss_axis_degree(ry, D);
    return (long double)w * h * std::pow((long double)rx, 2 * dx) * std::pow((long double)ry, 2 * dy);
}

swih_status build_layout(const swih_plan_desc *d, swih_plan_s *pl)
{
    if (!d) return fail(nullptr, SWIH_ERR_INVALID_ARG, "desc is NULL");
    if (d->height < 3 || d->width < 3)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "image must be at least 3 x 3");
    if (d->width > 8192)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED, "image width above 8192 is not supported");
    if (d->height > (1 << 24))
        return fail(nullptr, SWIH_ERR_UNSUPPORTED, "image height above 2^24 is not supported");
    if (d->pixel_type != SWIH_PIXEL_U8 && d->pixel_type != SWIH_PIXEL_U16)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "pixel_type must be U8 or U16");
    const int pb = d->pixel_type == SWIH_PIXEL_U8 ? 1 : 2;
    if (d->bitdepth < 1 || d->bitdepth > 8 * pb)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "bitdepth out of range for the pixel type");
    if (d->pitch_bytes < (int64_t)d->width * pb)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "pitch_bytes smaller than a row");
    if (d->pixel_type == SWIH_PIXEL_U16 && (d->pitch_bytes & 1))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "pitch_bytes of a U16 image must be even");
    if (d->bins < 1 || d->bins > 256)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "bins must be in [1, 256]");
    if (d->kernel_mask == 0 || (d->kernel_mask & ~0x3Fu))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "kernel_mask must name kernels 0..5");
    if (d->wedding_rings < 0 || d->wedding_rings > kMaxRings)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "wedding_rings must be in [0, 16]");
    if (!odd_window(d->max_win_w) || !odd_window(d->max_win_h))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "max window sides must be odd and >= 3");
    if (d->max_win_w > d->width || d->max_win_h > d->height)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "max window larger than the image");
    if (d->precision < SWIH_PREC_AUTO || d->precision > SWIH_PREC_RING128)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "precision out of range");
    if (d->band_rows < 0) return fail(nullptr, SWIH_ERR_INVALID_ARG, "band_rows must be >= 0");
    const int D = d->gauss_degree == 0 ? 2 : d->gauss_degree;
    if (D < 1 || D > kWideMaxD) return fail(nullptr, SWIH_ERR_UNSUPPORTED, "gauss_degree must be in [1, 4]");
    const double sf = d->gauss_sigma_frac == 0.0 ? 0.25 : d->gauss_sigma_frac;
    if (!(sf > 0.0) || !std::isfinite(sf))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "gauss_sigma_frac must be positive");
    const bool want_exp = d->kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_EXPONENTIAL);
    if (want_exp && pl->n_ch > 0)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED, "feature channels serve the integer kernels only (no exponential)");
    const double lam = d->exp_lambda == 0.0 ? 0.1 : d->exp_lambda;
    if (want_exp && !(lam >= 1.0 / 1024.0 && lam <= 16.0))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "exp_lambda must be in [2^-10, 16]");

    pl->desc = *d;
    pl->gauss_degree = D;
    pl->sigma_frac = sf;
    pl->has_exp = want_exp;
    pl->exp_lambda = lam;
    if (want_exp) {
        // J_d < 1 / (1 - q)^2 and every window sum < 4 / (1 - q)^2: with
        // F = 60 - ceil(log2(1 / (1 - q)^2)) fraction bits all stay below 2^62
        const long double q = expl(-(long double)lam);
        const long double jmax = 1.0L / ((1.0L - q) * (1.0L - q));
        pl->exp_F = 60 - (int)ceill(log2l(jmax));
        // columns per scan thread: 4 up to 2048 columns (more warps per CTA hide
        // the latency of the rows that are scanned), 8 up to 4096, 16 above
        pl->exp_E = d->width > 4096 ? 16 : (d->width > 2048 ? 8 : 4);
        pl->exp_threads = (int)round_up((d->width + pl->exp_E - 1) / pl->exp_E, 32);
    }
    bool mark[kMaxP][kMaxQ] = {};
    const bool want_man = d->kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_MANHATTAN);
    const bool want_euc = d->kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_EUCLIDEAN);
    const bool want_gau = d->kernel_mask & SWIH_KERNEL_BIT(SWIH_KERNEL_GAUSSIAN);
    mark[0][0] = true;
    if (want_man || want_euc) mark[1][0] = mark[0][1] = true;
    if (want_euc) mark[2][0] = mark[0][2] = true;
    if (want_gau) {
        const int kx = 2 * gauss_axis_degree((d->max_win_w - 1) / 2, D);
        const int ky = 2 * gauss_axis_degree((d->max_win_h - 1) / 2, D);
        for (int p = 0; p <= kx; ++p)
            for (int q = 0; q <= ky; ++q) mark[p][q] = true;
    }
    // canonical order: grouped by q (one scan chain per q), p ascending
    for (auto &row : pl->term_index)
        for (int &v : row) v = -1;
    pl->n_terms = 0;
    pl->n_q = 0;
    for (int q = 0; q < kMaxQ; ++q) {
        int cnt = 0;
        for (int p = 0; p < kMaxP; ++p) {
            if (!mark[p][q]) continue;
            pl->term_p[pl->n_terms] = p;
            pl->term_q[pl->n_terms] = q;
            pl->p_val[pl->n_q][cnt++] = p;
            pl->term_index[p][q] = pl->n_terms++;
        }
        // the scan kernel relies on each chain's x-exponents being 0..cnt-1
        for (int k = 0; k < cnt; ++k)
            if (pl->p_val[pl->n_q][k] != k)
                return fail(nullptr, SWIH_ERR_UNSUPPORTED, "internal: non-contiguous term set");
        if (cnt) {
            pl->q_val[pl->n_q] = q;
            pl->p_count[pl->n_q] = cnt;
            ++pl->n_q;
        }
    }

    // ring: every window result must be exact in it
    long double need = 0;
    for (int k = SWIH_KERNEL_PLAIN; k <= SWIH_KERNEL_EUCLIDEAN; ++k)
        if (d->kernel_mask & SWIH_KERNEL_BIT(k))
            need = std::max(need, int_kernel_mass(k, d->max_win_w, d->max_win_h));
    if (d->kernel_mask & (SWIH_KERNEL_BIT(SWIH_KERNEL_WEDDING) | SWIH_KERNEL_BIT(SWIH_KERNEL_EXPONENTIAL)))
        need = std::max(need, int_kernel_mass(SWIH_KERNEL_PLAIN, d->max_win_w, d->max_win_h));  // window counts
    const bool fits32 = !want_gau && need < 4294967296.0L;
    // Gaussian: the per-window Bernstein moments are below w h rx^2D ry^2D;
    // past 2^64 they are kept in the ring mod 2^128 (Gaussian-only plans)
    const long double gb = want_gau ? gauss_bound(d->max_win_w, d->max_win_h, D) : 0.0L;
    const bool fits64 = gb < 18446744073709551616.0L;
    const bool fits128 = gb < 340282366920938463463374607431768211456.0L;
    const bool gau_only = d->kernel_mask == SWIH_KERNEL_BIT(SWIH_KERNEL_GAUSSIAN);
    if (d->precision == SWIH_PREC_RING32 && !fits32)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED,
                    "RING32 is not exact for these kernels and windows; use AUTO or RING64");
    if (d->precision == SWIH_PREC_RING64 && !fits64)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED,
                    "RING64 is not exact for this Gaussian window (w*h*rx^2D*ry^2D >= 2^64); use AUTO or RING128");
    const bool want128 = d->precision == SWIH_PREC_RING128 || (want_gau && !fits64);
    if (want128) {
        if (!want_gau || !gau_only)
            return fail(nullptr, SWIH_ERR_UNSUPPORTED, "the 128-bit ring serves plans of the Gaussian kernel alone");
        if (!fits128)
            return fail(nullptr, SWIH_ERR_UNSUPPORTED,
                        "Gaussian window too large for exact 128-bit moments (w*h*rx^2D*ry^2D >= 2^128)");
        if (d->width > 4096)
            return fail(nullptr, SWIH_ERR_UNSUPPORTED, "the 128-bit ring serves images up to 4096 columns");
    }
    pl->elem_bytes = want128 ? 16 : (d->precision == SWIH_PREC_RING64 || !fits32) ? 8 : 4;

    // layout
    const int W = d->width, H = d->height;
    pl->bins_pitch = round_up(W, 128);
    pl->ih_pitch = round_up(W, 32);
    pl->plane = (int64_t)H * pl->ih_pitch;
    pl->band_rows = d->band_rows > 0 ? std::min(d->band_rows, H) : std::min(32, H);
    pl->n_bands = (H + pl->band_rows - 1) / pl->band_rows;
    // columns per scan thread: the fewest that keep the block at <= 512 threads
    int E = 4;
    while ((W + E - 1) / E > 512) E *= 2;
    pl->scan_E = E;
    pl->scan_threads = (int)round_up((W + E - 1) / E, 32);
    const uint64_t n_chains = (uint64_t)d->bins * pl->n_q;
    const uint64_t es = (uint64_t)pl->elem_bytes;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    take((uint64_t)std::max(1, pl->n_ch) * H * pl->bins_pitch);  // bins at offset 0 (one plane per channel)
    if (pl->n_ch > 0) pl->off_chtgt = take((uint64_t)pl->n_ch * d->bins * sizeof(float));
    pl->off_ih = take((uint64_t)pl->n_terms * d->bins * pl->plane * es);
    pl->off_agg = take(n_chains * pl->n_bands * pl->ih_pitch * es);
    pl->off_incl = take(n_chains * pl->n_bands * pl->ih_pitch * es);
    pl->flags_bytes = (n_chains * pl->n_bands + 1) * sizeof(int);  // flags + ticket
    pl->off_flags = take(pl->flags_bytes);
    // per-bin-group likelihoods of a split gather: up to 8 groups of the
    // largest map, at most 64 MB
    pl->partial_floats = std::min<uint64_t>((uint64_t)8 * H * W, (64ull << 20) / sizeof(float));
    pl->off_partial = take(pl->partial_floats * sizeof(float));
    pl->sparse_rows = pl->band_rows <= 64 && H <= 32767;  // the gather keeps stored rows as int16
    if (pl->sparse_rows) {
        pl->off_occ = take((uint64_t)d->bins * pl->n_bands * sizeof(unsigned long long));
        pl->off_row_map = take((uint64_t)d->bins * H * sizeof(int));
    }
    if (want_exp) {
        pl->off_exp = take((uint64_t)4 * d->bins * pl->plane * sizeof(unsigned long long));
        pl->off_exp_carry = take((uint64_t)2 * d->bins * pl->n_bands * pl->ih_pitch * sizeof(unsigned long long));
        pl->off_exp_rows = take((uint64_t)2 * d->bins * pl->n_bands * sizeof(unsigned long long));
    }
    pl->off_jobs = take((uint64_t)swih_plan_s::kJobSlots * kJobSlotBytes);
    take(sizeof(uint32_t) * 64);  // status word
    pl->total = off;
    if (d->hbm_budget_bytes && pl->total > d->hbm_budget_bytes) {
        char m[160];
        std::snprintf(m, sizeof m, "workspace %llu bytes exceeds the budget of %llu bytes",
                      (unsigned long long)pl->total, (unsigned long long)d->hbm_budget_bytes);
        return fail(nullptr, SWIH_ERR_BUDGET, m);
    }
    return SWIH_OK;
}

swih_status check_window(swih_plan_s *pl, int kernel, int w, int h)
{
    if (kernel < SWIH_KERNEL_PLAIN || kernel > SWIH_KERNEL_EXPONENTIAL)
        return fail(pl, SWIH_ERR_INVALID_ARG, "unknown kernel");
    if (!(pl->desc.kernel_mask & SWIH_KERNEL_BIT(kernel)))
        return fail(pl, SWIH_ERR_INVALID_ARG, "kernel not in the plan's kernel_mask");
    if (!odd_window(w) || !odd_window(h))
        return fail(pl, SWIH_ERR_INVALID_ARG, "window sides must be odd and >= 3");
    if (w > pl->desc.max_win_w || h > pl->desc.max_win_h)
        return fail(pl, SWIH_ERR_INVALID_ARG, "window larger than the plan's max window");
    if (!pl->built) return fail(pl, SWIH_ERR_INVALID_ARG, "swih_build_ih has not been called");
    return SWIH_OK;
}

// Wedding-cake rings of a w x h window: nested half-sides floor((2 i r + n) /
// (2 n)), i = 1..n, per axis (repeats dropped), each ring weighted by the
// mean Manhattan weight over its pixels. Sums are exact integers:
// sum over |dx| <= a, |dy| <= b of (rx - |dx|) + (ry - |dy|)
//   = (2b+1) ((2a+1) rx - a (a+1)) + (2a+1) ((2b+1) ry - b (b+1)).
int wedding_rings(int w, int h, int n, int *rx_i, int *ry_i, double *weight)
{
    const long long rx = (w - 1) / 2, ry = (h - 1) / 2;
    auto rect_sum = [&](long long a, long long b) -> long long {
        return (2 * b + 1) * ((2 * a + 1) * rx - a * (a + 1)) + (2 * a + 1) * ((2 * b + 1) * ry - b * (b + 1));
    };
    int m = 0;
    long long prev_sum = 0, prev_cnt = 0;
    for (int i = 1; i <= n; ++i) {
        const int a = (int)((2LL * i * rx + n) / (2LL * n)), b = (int)((2LL * i * ry + n) / (2LL * n));
        if (m > 0 && a == rx_i[m - 1] && b == ry_i[m - 1]) continue;
        const long long cnt = (2LL * a + 1) * (2LL * b + 1), sum = rect_sum(a, b);
        rx_i[m] = a;
        ry_i[m] = b;
        weight[m] = (double)(sum - prev_sum) / (double)(cnt - prev_cnt);
        prev_sum = sum;
        prev_cnt = cnt;
        ++m;
    }
    return m;
}

swih_status make_gather(swih_plan_s *pl, int kernel, int w, int h, GatherParams &g, int &kind)
{
    std::memset(&g, 0, sizeof g);
    g.ih = pl->d_mem + pl->off_ih;
    g.row_map = (pl->sparse_rows && pl->d_mem) ? reinterpret_cast<const int *>(pl->d_mem + pl->off_row_map) : nullptr;
    g.plane = pl->plane;
    g.pitch = pl->ih_pitch;
    g.B = pl->desc.bins;
    g.H = pl->desc.height;
    g.W = pl->desc.width;
    g.rx = (w - 1) / 2;
    g.ry = (h - 1) / 2;
    g.t1 = pl->term_index[0][0];
    g.tx = pl->term_index[1][0];
    g.ty = pl->term_index[0][1];
    g.txx = pl->term_index[2][0];
    g.tyy = pl->term_index[0][2];
    for (int k = 0; k < 5; ++k)
        for (int l = 0; l < 5; ++l) g.tg[k][l] = pl->term_index[k][l];
    g.status = pl->d_status;
    g.n_targets = 1;
    g.target_stride = pl->desc.bins;
    g.map_stride = 0;
    g.nbg = 1;
    g.load_bytes = reinterpret_cast<unsigned long long *>(pl->d_status + 2);  // 8-byte aligned word of the status block
    g.partial = pl->partial_floats ? reinterpret_cast<float *>(pl->d_mem + pl->off_partial) : nullptr;
    g.partial_cap = (int64_t)pl->partial_floats;
    g.want_tx = pl->cfg_tx[kernel];
    g.want_stages = pl->cfg_stages[kernel];
    g.want_bb = pl->cfg_bb[kernel];
    if (kernel == SWIH_KERNEL_GAUSSIAN) {
        if (gauss_is_wide(pl, w, h))
            return fail(pl, SWIH_ERR_UNSUPPORTED,
                        "a Gaussian of degree above 2 or in the 128-bit ring takes the any-degree gather");
        GaussAxis ax, ay;
        std::string why;
        if (!gauss_axis(g.rx, pl->sigma_frac * w, pl->gauss_degree, ax, why) ||
            !gauss_axis(g.ry, pl->sigma_frac * h, pl->gauss_degree, ay, why))
            return fail(pl, SWIH_ERR_UNSUPPORTED, why);
        g.gdx = ax.D;
        g.gdy = ay.D;
        const unsigned long long rx2 = (unsigned long long)g.rx * g.rx, ry2 = (unsigned long long)g.ry * g.ry;
        g.rx2 = rx2;
        g.rx4 = rx2 * rx2;
        g.ry2 = ry2;
        g.ry4 = ry2 * ry2;
        const double mass = ax.mass * ay.mass;
        const double sx = std::pow((double)g.rx, 2 * ax.D), sy = std::pow((double)g.ry, 2 * ay.D);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                g.gamma[i][j] = (float)(ax.beta[i] * ay.beta[j] / (sx * sy * mass));
        kind = kGatherGaussian;
        const int kx = 2 * ax.D, ky = 2 * ay.D;
        g.n_load_even = 0;
        for (int l = 0; l <= ky; ++l)
            for (int k = 0; k <= kx; ++k) g.load_even[g.n_load_even++] = g.tg[k][l];
        g.n_load_odd = 0;
        g.nl = g.n_load_even;
    } else if (kernel == SWIH_KERNEL_WEDDING) {
        kind = kGatherWedding;
        double wt[kMaxRings];
        const int n = pl->desc.wedding_rings ? pl->desc.wedding_rings : 4;
        g.n_rings = wedding_rings(w, h, n, g.ring_rx, g.ring_ry, wt);
        for (int i = 0; i < g.n_rings; ++i) g.ring_c[i] = (float)(wt[i] - (i + 1 < g.n_rings ? wt[i + 1] : 0.0));
        // the rings partition the window and carry the Manhattan kernel's mass
        g.inv_mass = (float)(1.0L / int_kernel_mass(SWIH_KERNEL_MANHATTAN, w, h));
        g.load_even[0] = g.t1;
        g.n_load_even = 1;
        g.n_load_odd = 0;
        g.nl = 1;
    } else {
        g.inv_mass = (float)(1.0L / int_kernel_mass(kernel, w, h));
        kind = kernel == SWIH_KERNEL_PLAIN ? kGatherPlain
               : kernel == SWIH_KERNEL_MANHATTAN ? kGatherManhattan
                                                 : kGatherEuclidean;
        if (kind == kGatherPlain) {
            g.load_even[0] = g.t1;
            g.n_load_even = 1;
            g.n_load_odd = 0;
        } else if (kind == kGatherManhattan) {
            g.load_even[0] = g.t1;
            g.load_even[1] = g.tx;
            g.load_even[2] = g.ty;
            g.n_load_even = 3;
            g.load_odd[0] = g.t1;
            g.load_odd[1] = g.ty;
            g.n_load_odd = 2;
        } else {
            g.load_even[0] = g.t1;
            g.load_even[1] = g.tx;
            g.load_even[2] = g.ty;
            g.load_even[3] = g.txx;
            g.load_even[4] = g.tyy;
            g.n_load_even = 5;
            g.n_load_odd = 0;
        }
        g.nl = std::max(g.n_load_even, g.n_load_odd);
    }
    return SWIH_OK;
}

// the Gaussian at this window needs the any-degree gather: a fitted degree
// above 2 on either axis, or 16-byte ring elements
bool gauss_is_wide(const swih_plan_s *pl, int w, int h)
{
    return pl->elem_bytes == 16 || gauss_axis_degree((w - 1) / 2, pl->gauss_degree) > 2 ||
           gauss_axis_degree((h - 1) / 2, pl->gauss_degree) > 2;
}

// Integer coefficients of the Bernstein moments on one axis, as ring elements:
// A_i(d) = C(D, i) d^2i (r^2 - d^2)^(D - i) = sum_k a[i][k] d^2k with
// a[i][k] = C(D, i) C(D - i, k - i) (-1)^(k - i) r^(2 (D - k)) for i <= k <= D
// (zero elsewhere), reduced mod 2^128 (the low word serves the 64-bit ring).
static void bernstein_axis(int D, int r, unsigned long long (*lo)[kWideMaxD + 1],
                           unsigned long long (*hi)[kWideMaxD + 1])
{
    for (int i = 0; i <= kWideMaxD; ++i)
        for (int k = 0; k <= kWideMaxD; ++k) lo[i][k] = hi[i][k] = 0ull;
    for (int i = 0; i <= D; ++i)
        for (int k = i; k <= D; ++k) {
            unsigned __int128 v = (unsigned __int128)(unsigned long long)(binom(D, i) * binom(D - i, k - i) + 0.5);
            for (int e = 0; e < 2 * (D - k); ++e) v *= (unsigned __int128)(unsigned)r;
            if ((k - i) & 1) v = (unsigned __int128)0 - v;
            lo[i][k] = (unsigned long long)v;
            hi[i][k] = (unsigned long long)(v >> 64);
        }
}

swih_status make_gauss_wide(swih_plan_s *pl, int w, int h, GaussWideParams &g)
{
    std::memset(&g, 0, sizeof g);
    g.ih = pl->d_mem + pl->off_ih;
    g.row_map = (pl->sparse_rows && pl->d_mem) ? reinterpret_cast<const int *>(pl->d_mem + pl->off_row_map) : nullptr;
    g.plane = pl->plane;
    g.pitch = pl->ih_pitch;
    g.B = pl->desc.bins;
    g.H = pl->desc.height;
    g.W = pl->desc.width;
    g.rx = (w - 1) / 2;
    g.ry = (h - 1) / 2;
    GaussAxis ax, ay;
    std::string why;
    if (!gauss_axis(g.rx, pl->sigma_frac * w, pl->gauss_degree, ax, why) ||
        !gauss_axis(g.ry, pl->sigma_frac * h, pl->gauss_degree, ay, why))
        return fail(pl, SWIH_ERR_UNSUPPORTED, why);
    g.dx = ax.D;
    g.dy = ay.D;
    for (int a = 0; a <= 2 * g.dx; ++a)
        for (int b = 0; b <= 2 * g.dy; ++b) {
            g.tg[a][b] = pl->term_index[a][b];
            if (g.tg[a][b] < 0) return fail(pl, SWIH_ERR_UNSUPPORTED, "internal: a Gaussian term is missing");
        }
    bernstein_axis(g.dx, g.rx, g.ax_lo, g.ax_hi);
    bernstein_axis(g.dy, g.ry, g.ay_lo, g.ay_hi);
    const long double sx = powl((long double)g.rx, 2 * g.dx), sy = powl((long double)g.ry, 2 * g.dy);
    const long double mass = (long double)ax.mass * ay.mass;
    for (int i = 0; i <= g.dx; ++i)
        for (int j = 0; j <= g.dy; ++j) g.gamma[i][j] = (double)(ax.beta[i] * (long double)ay.beta[j] / (sx * sy * mass));
    g.n_targets = 1;
    g.target_stride = g.B;
    return SWIH_OK;
}

unsigned long long exp_pow_fixed(long double lambda, long double n)
{
    const long double v = ldexpl(expl(-lambda * n), 64);
    if (v >= 18446744073709551615.0L) return ~0ull;
    if (!(v >= 1.0L)) return 0ull;
    return (unsigned long long)v;  // truncation: floor of a positive value
}

// Exponential-kernel gather over a rectangle of centres (likelihood map and/or
// histograms). The window's total weight is M = Sx Sy with
// S = sum_{d=-r..r} q^|d| = 1 + 2 q (1 - q^r) / (1 - q).
cudaError_t run_exp_gather(swih_plan_s *pl, int w, int h, int cx0, int cy0, int ncx, int ncy,
                           const float *target, float *map, float *hist, cudaStream_t s)
{
    ExpGatherParams g;
    std::memset(&g, 0, sizeof g);
    const int B = pl->desc.bins;
    g.count = pl->d_mem + pl->off_ih + (uint64_t)pl->term_index[0][0] * B * pl->plane * pl->elem_bytes;
    g.row_map = pl->sparse_rows ? reinterpret_cast<const int *>(pl->d_mem + pl->off_row_map) : nullptr;
    g.J = reinterpret_cast<const unsigned long long *>(pl->d_mem + pl->off_exp);
    g.pitch = pl->ih_pitch;
    g.plane = pl->plane;
    g.B = B;
    g.H = pl->desc.height;
    g.W = pl->desc.width;
    g.rx = (w - 1) / 2;
    g.ry = (h - 1) / 2;
    g.cx0 = cx0;
    g.cy0 = cy0;
    g.ncx = ncx;
    g.ncy = ncy;
    g.target = target;
    g.map = map;
    g.hist = hist;
    const long double lam = pl->exp_lambda;
    g.qx1 = exp_pow_fixed(lam, g.rx + 1);
    g.qx0 = exp_pow_fixed(lam, g.rx);
    g.qy1 = exp_pow_fixed(lam, g.ry + 1);
    g.qy0 = exp_pow_fixed(lam, g.ry);
    g.q1 = exp_pow_fixed(lam, 1);
    const long double q = expl(-lam);
    auto axis = [&](int r) { return 1.0L + 2.0L * q * (1.0L - powl(q, r)) / (1.0L - q); };
    g.scale = (float)(ldexpl(1.0L, -pl->exp_F) / (axis(g.rx) * axis(g.ry)));
    return launch_exp_gather(g, pl->elem_bytes, s);
}

// tiled gather when its row segments fit in shared memory, else the direct one
cudaError_t run_gather(swih_plan_s *pl, const GatherParams &g, int kind, cudaStream_t s)
{
    if (pl->gather_path != 1) {
        const cudaError_t e = launch_gather_tiled(g, kind, pl->elem_bytes, s);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    return launch_gather(g, kind, pl->elem_bytes, s);
}

}  // namespace swih

namespace swih {

swih_status plan_layout(const swih_plan_desc *d, PlanLayout *out)
{
    swih_plan_s tmp;
    swih_plan_desc d2 = *d;
    d2.hbm_budget_bytes = 0;
    const swih_status st = build_layout(&d2, &tmp);
    if (st != SWIH_OK) return st;
    out->elem_bytes = tmp.elem_bytes;
    out->n_terms = tmp.n_terms;
    for (int t = 0; t < tmp.n_terms; ++t) {
        out->term_p[t] = tmp.term_p[t];
        out->term_q[t] = tmp.term_q[t];
    }
    out->n_q = tmp.n_q;
    for (int i = 0; i < tmp.n_q; ++i) {
        out->q_val[i] = tmp.q_val[i];
        out->p_count[i] = tmp.p_count[i];
        for (int k = 0; k < tmp.p_count[i]; ++k) {
            out->p_val[i][k] = tmp.p_val[i][k];
            out->term[i][k] = tmp.term_index[tmp.p_val[i][k]][tmp.q_val[i]];
        }
    }
    out->bins_pitch = tmp.bins_pitch;
    out->ih_pitch = tmp.ih_pitch;
    out->plane = tmp.plane;
    out->band_rows = tmp.band_rows;
    out->n_bands = tmp.n_bands;
    out->scan_E = tmp.scan_E;
    out->scan_threads = tmp.scan_threads;
    return SWIH_OK;
}

void set_thread_error(const char *msg) { g_err = msg; }

std::atomic<unsigned long long> g_launches{0};

void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace swih

extern "C" {

swih_status swih_plan_workspace_bytes(const swih_plan_desc *desc, uint64_t *bytes)
{
    if (!bytes) return fail(nullptr, SWIH_ERR_INVALID_ARG, "bytes is NULL");
    swih_plan_s tmp;
    swih_plan_desc d2;
    if (desc) {
        d2 = *desc;
        d2.hbm_budget_bytes = 0;  // report the size even when over budget
    }
    const swih_status st = build_layout(desc ? &d2 : nullptr, &tmp);
    if (st != SWIH_OK) return st;
    *bytes = tmp.total;
    return SWIH_OK;
}

swih_status swih_plan(const swih_plan_desc *desc, swih_plan_t *out)
{
    if (!out) return fail(nullptr, SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    swih_plan_s *pl = new swih_plan_s();
    swih_status st = build_layout(desc, pl);
    if (st != SWIH_OK) {
        delete pl;
        return st;
    }
    return swih::allocate_plan(pl, out);
}

}  // extern "C"

namespace swih {

swih_status allocate_plan(swih_plan_s *pl, swih_plan_t *out)
{
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(nullptr, "cudaGetDevice", e);
    }
    e = cudaMalloc(reinterpret_cast<void **>(&pl->d_mem), pl->total);
    if (e != cudaSuccess) {
        delete pl;
        cudaGetLastError();
        return cuda_fail(nullptr, "cudaMalloc(workspace)", e);
    }
    pl->d_status = reinterpret_cast<uint32_t *>(pl->d_mem + pl->total - sizeof(uint32_t) * 64);
    e = cudaMemset(pl->d_status, 0, sizeof(uint32_t) * 64);
    if (e == cudaSuccess) e = cudaMemset(pl->d_mem + pl->off_flags, 0, pl->flags_bytes);
    if (e != cudaSuccess) {
        cudaFree(pl->d_mem);
        delete pl;
        return cuda_fail(nullptr, "cudaMemset(status)", e);
    }
    *out = pl;
    return SWIH_OK;
}

// Steps after quantisation: the weighted integral histograms (K2), the row map
// and the exponential kernel's tables (K2e), from the plan's bin planes.
swih_status build_scans(swih_plan_s *pl, cudaStream_t s)
{
    const swih_plan_desc &d = pl->desc;
    cudaError_t e;
    e = cudaMemsetAsync(pl->d_mem + pl->off_flags, 0, pl->flags_bytes, s);
    if (e != cudaSuccess) return cuda_fail(pl, "cudaMemsetAsync(scan flags)", e);

    ScanParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.bins = reinterpret_cast<const uint8_t *>(pl->d_mem);
    sp.bins_pitch = pl->bins_pitch;
    sp.ih = pl->d_mem + pl->off_ih;
    sp.ih_pitch = pl->ih_pitch;
    sp.plane = pl->plane;
    sp.agg = pl->d_mem + pl->off_agg;
    sp.incl = pl->d_mem + pl->off_incl;
    sp.flags = reinterpret_cast<int *>(pl->d_mem + pl->off_flags);
    sp.ticket = sp.flags + (int64_t)d.bins * pl->n_q * pl->n_bands;
    sp.status = pl->d_status;
    sp.H = d.height;
    sp.W = d.width;
    sp.B = d.bins;
    sp.band_rows = pl->band_rows;
    sp.n_bands = pl->n_bands;
    sp.n_q = pl->n_q;
    for (int i = 0; i < pl->n_q; ++i) {
        sp.q_val[i] = pl->q_val[i];
        sp.p_count[i] = pl->p_count[i];
        for (int k = 0; k < pl->p_count[i]; ++k) {
            sp.p_val[i][k] = pl->p_val[i][k];
            sp.term[i][k] = pl->term_index[pl->p_val[i][k]][pl->q_val[i]];
        }
    }
    sp.spin_limit = 1LL << 22;  // with 64 ns sleeps: well under a few seconds
    sp.stall_tile = -1;
    sp.occ = pl->sparse_rows ? reinterpret_cast<unsigned long long *>(pl->d_mem + pl->off_occ) : nullptr;
    if (pl->n_ch > 0) {  // bin b's chain reads its channel's bin plane
        sp.ch_stride = (int64_t)d.height * pl->bins_pitch;
        for (int c = 0; c < pl->n_ch; ++c)
            for (int b = pl->ch_bin0[c]; b < pl->ch_bin0[c + 1]; ++b) sp.ch_of_bin[b] = (uint8_t)c;
    }
    if (pl->inject == SWIH_INJECT_STALL_SCAN_TILE) {
        sp.stall_tile = 0;        // chain 0, band 0 never publishes
        sp.spin_limit = 1LL << 12;
        pl->inject = 0;
    }
    e = launch_ih_scan(sp, pl->elem_bytes, pl->scan_E, pl->scan_threads, s);
    if (e != cudaSuccess) return cuda_fail(pl, "ih_scan launch", e);
    if (pl->sparse_rows) {
        e = launch_row_map(sp.occ, reinterpret_cast<int *>(pl->d_mem + pl->off_row_map), d.bins, d.height,
                           pl->band_rows, pl->n_bands, s);
        if (e != cudaSuccess) return cuda_fail(pl, "row map launch", e);
    }
    if (pl->has_exp) {
        ExpScanParams xp;
        std::memset(&xp, 0, sizeof xp);
        xp.bins = reinterpret_cast<const uint8_t *>(pl->d_mem);
        xp.bins_pitch = pl->bins_pitch;
        xp.J = reinterpret_cast<unsigned long long *>(pl->d_mem + pl->off_exp);
        xp.pitch = pl->ih_pitch;
        xp.plane = pl->plane;
        xp.carry = reinterpret_cast<unsigned long long *>(pl->d_mem + pl->off_exp_carry);
        xp.H = d.height;
        xp.W = d.width;
        xp.B = d.bins;
        xp.band_rows = pl->band_rows;
        xp.n_bands = pl->n_bands;
        xp.E = pl->exp_E;
        xp.threads = pl->exp_threads;
        xp.one = 1ull << pl->exp_F;
        const long double lam = pl->exp_lambda;
        xp.q1 = exp_pow_fixed(lam, 1);
        xp.qband = exp_pow_fixed(lam, pl->band_rows);
        xp.rows = reinterpret_cast<unsigned long long *>(pl->d_mem + pl->off_exp_rows);
        xp.qrow[0] = xp.one;
        for (int k = 1; k <= 64; ++k) xp.qrow[k] = exp_pow_fixed(lam, k) >> (64 - pl->exp_F);
        for (int k = 1; k <= 32; ++k) xp.qe[k] = exp_pow_fixed(lam, (long double)xp.E * k);
        for (int k = 1; k <= 16; ++k) xp.qw[k] = exp_pow_fixed(lam, 32.0L * xp.E * k);
        e = launch_exp_scan(xp, s);
        if (e != cudaSuccess) return cuda_fail(pl, "exponential scan launch", e);
    }
    pl->built = true;
    return SWIH_OK;
}

}  // namespace swih

extern "C" {

swih_status swih_build_ih(swih_plan_t pl, const void *d_image, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (!d_image) return fail(pl, SWIH_ERR_INVALID_ARG, "d_image is NULL");
    const swih_plan_desc &d = pl->desc;
    if (d.pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_image) & 1))
        return fail(pl, SWIH_ERR_INVALID_ARG, "a U16 image must be 2-byte aligned");
    if (pl->n_ch > 0) return fail(pl, SWIH_ERR_INVALID_ARG, "a feature-channel plan is built by swih_build_ih_channels");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    QuantParams qp;
    qp.image = static_cast<const uint8_t *>(d_image);
    qp.pitch = d.pitch_bytes;
    qp.H = d.height;
    qp.W = d.width;
    qp.B = d.bins;
    qp.bitdepth = d.bitdepth;
    qp.bins = reinterpret_cast<uint8_t *>(pl->d_mem);
    qp.bins_pitch = pl->bins_pitch;
    qp.pixel_bytes = d.pixel_type == SWIH_PIXEL_U8 ? 1 : 2;
    qp.vec = (d.pitch_bytes % 16 == 0) && (reinterpret_cast<uintptr_t>(d_image) % 16 == 0);
    cudaError_t e = launch_quantize(qp, s);
    if (e != cudaSuccess) return cuda_fail(pl, "quantize launch", e);

    return build_scans(pl, s);
}

swih_status swih_local_hist(swih_plan_t pl, int kernel, int win_w, int win_h, int cx0, int cy0,
                            int ncx, int ncy, float *d_hist, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    swih_status st = check_window(pl, kernel, win_w, win_h);
    if (st != SWIH_OK) return st;
    if (!d_hist) return fail(pl, SWIH_ERR_INVALID_ARG, "d_hist is NULL");
    const int rx = (win_w - 1) / 2, ry = (win_h - 1) / 2;
    const int W = pl->desc.width, H = pl->desc.height;
    if (ncx < 0 || ncy < 0) return fail(pl, SWIH_ERR_INVALID_ARG, "negative centre count");
    if (ncx == 0 || ncy == 0) return SWIH_OK;
    if (cx0 < rx || cy0 < ry || (int64_t)cx0 + ncx > W - rx || (int64_t)cy0 + ncy > H - ry)
        return fail(pl, SWIH_ERR_INVALID_ARG, "centre rectangle has windows outside the image");
    if (kernel == SWIH_KERNEL_EXPONENTIAL) {
        const cudaError_t e = run_exp_gather(pl, win_w, win_h, cx0, cy0, ncx, ncy, nullptr, nullptr, d_hist,
                                             static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(pl, "exponential gather launch", e);
        return SWIH_OK;
    }
    if (kernel == SWIH_KERNEL_GAUSSIAN && gauss_is_wide(pl, win_w, win_h)) {
        GaussWideParams gw;
        st = make_gauss_wide(pl, win_w, win_h, gw);
        if (st != SWIH_OK) return st;
        gw.cx0 = cx0;
        gw.cy0 = cy0;
        gw.ncx = ncx;
        gw.ncy = ncy;
        gw.hist = d_hist;
        const cudaError_t e = launch_gauss_wide(gw, pl->elem_bytes, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(pl, "Gaussian gather launch", e);
        return SWIH_OK;
    }
    GatherParams g;
    int kind = 0;
    st = make_gather(pl, kernel, win_w, win_h, g, kind);
    if (st != SWIH_OK) return st;
    g.cx0 = cx0;
    g.cy0 = cy0;
    g.ncx = ncx;
    g.ncy = ncy;
    g.hist = d_hist;
    const cudaError_t e = run_gather(pl, g, kind, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(pl, "gather launch", e);
    return SWIH_OK;
}

swih_status swih_likelihood(swih_plan_t pl, int kernel, int win_w, int win_h, const float *d_target,
                            float *d_map, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    swih_status st = check_window(pl, kernel, win_w, win_h);
    if (st != SWIH_OK) return st;
    if (!d_target || !d_map) return fail(pl, SWIH_ERR_INVALID_ARG, "d_target or d_map is NULL");
    if (kernel == SWIH_KERNEL_EXPONENTIAL) {
        const cudaError_t e = run_exp_gather(pl, win_w, win_h, (win_w - 1) / 2, (win_h - 1) / 2,
                                             pl->desc.width - win_w + 1, pl->desc.height - win_h + 1, d_target,
                                             d_map, nullptr, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(pl, "exponential gather launch", e);
        return SWIH_OK;
    }
    if (kernel == SWIH_KERNEL_GAUSSIAN && gauss_is_wide(pl, win_w, win_h)) {
        GaussWideParams gw;
        st = make_gauss_wide(pl, win_w, win_h, gw);
        if (st != SWIH_OK) return st;
        gw.cx0 = (win_w - 1) / 2;
        gw.cy0 = (win_h - 1) / 2;
        gw.ncx = pl->desc.width - win_w + 1;
        gw.ncy = pl->desc.height - win_h + 1;
        gw.target = d_target;
        gw.map = d_map;
        const cudaError_t e = launch_gauss_wide(gw, pl->elem_bytes, static_cast<cudaStream_t>(stream));
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
    g.target = d_target;
    g.map = d_map;
    const cudaError_t e = run_gather(pl, g, kind, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(pl, "gather launch", e);
    return SWIH_OK;
}

swih_status swih_likelihood_scales(swih_plan_t pl, int kernel, int n_windows, const int *win_w, const int *win_h,
                                   const float *const *d_targets, float *const *d_maps, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (n_windows < 1 || n_windows > SWIH_MAX_SCALES)
        return fail(pl, SWIH_ERR_INVALID_ARG, "n_windows must be in [1, SWIH_MAX_SCALES]");
    if (!win_w || !win_h || !d_targets || !d_maps)
        return fail(pl, SWIH_ERR_INVALID_ARG, "win_w, win_h, d_targets and d_maps are required");
    for (int i = 0; i < n_windows; ++i) {
        const swih_status st = check_window(pl, kernel, win_w[i], win_h[i]);
        if (st != SWIH_OK) return st;
        if (!d_targets[i] || !d_maps[i]) return fail(pl, SWIH_ERR_INVALID_ARG, "a target or map is NULL");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto one_by_one = [&]() -> swih_status {
        for (int i = 0; i < n_windows; ++i) {
            const swih_status st = swih_likelihood(pl, kernel, win_w[i], win_h[i], d_targets[i], d_maps[i], stream);
            if (st != SWIH_OK) return st;
        }
        return SWIH_OK;
    };
    const bool tiled_kind = kernel == SWIH_KERNEL_PLAIN || kernel == SWIH_KERNEL_MANHATTAN ||
                            kernel == SWIH_KERNEL_EUCLIDEAN || kernel == SWIH_KERNEL_GAUSSIAN;
    if (n_windows == 1 || !tiled_kind || pl->gather_path == 1 || pl->desc.height > kTiledMaxRows)
        return one_by_one();
    if (kernel == SWIH_KERNEL_GAUSSIAN)
        for (int i = 0; i < n_windows; ++i)
            if (gauss_is_wide(pl, win_w[i], win_h[i])) return one_by_one();
    GatherParams jobs[SWIH_MAX_SCALES];
    int kind = 0, max_w = 3;
    for (int i = 0; i < n_windows; ++i) {
        int k = 0;
        const swih_status st = make_gather(pl, kernel, win_w[i], win_h[i], jobs[i], k);
        if (st != SWIH_OK) return st;
        if (i > 0 && (jobs[i].gdx != jobs[0].gdx || jobs[i].gdy != jobs[0].gdy)) return one_by_one();
        kind = k;
        jobs[i].cx0 = (win_w[i] - 1) / 2;
        jobs[i].cy0 = (win_h[i] - 1) / 2;
        jobs[i].ncx = pl->desc.width - win_w[i] + 1;
        jobs[i].ncy = pl->desc.height - win_h[i] + 1;
        jobs[i].target = d_targets[i];
        jobs[i].map = d_maps[i];
        jobs[i].nbg = 1;
        max_w = std::max(max_w, win_w[i]);
    }
    GatherShape sh;
    if (tiled_shape(kind, pl->elem_bytes, jobs[0].gdx, jobs[0].gdy, max_w, pl->desc.bins, jobs[0].nl, 1,
                    jobs[0].want_tx, jobs[0].want_stages, jobs[0].want_bb, true, &sh) != cudaSuccess) {
        cudaGetLastError();
        return one_by_one();
    }
    int start[SWIH_MAX_SCALES + 1];
    long long total = 0;
    for (int i = 0; i < n_windows; ++i) {
        start[i] = (int)total;
        total += tiled_items(&jobs[i], sh);
        if (total > 0x7fffffffLL) return one_by_one();
    }
    start[n_windows] = (int)total;
    // job table, then the item starts: a slot already holding this table is
    // reused as it is; otherwise the least recently used slot is uploaded on
    // the stream (stream-ordered)
    std::vector<unsigned char> host(kJobSlotBytes, 0);
    std::memcpy(host.data(), jobs, sizeof(GatherParams) * n_windows);
    std::memcpy(host.data() + sizeof(GatherParams) * SWIH_MAX_SCALES, start, sizeof(int) * (n_windows + 1));
    int slot = -1, lru = 0;
    for (int k = 0; k < swih_plan_s::kJobSlots; ++k) {
        if (pl->job_slot[k] == host) slot = k;
        if (pl->job_slot_use[k] < pl->job_slot_use[lru]) lru = k;
    }
    const bool upload = slot < 0;
    if (upload) slot = lru;
    pl->job_slot_use[slot] = ++pl->job_clock;
    char *d_tab = pl->d_mem + pl->off_jobs + (uint64_t)slot * kJobSlotBytes;
    cudaError_t e = cudaSuccess;
    if (upload) {
        pl->job_slot[slot] = host;
        e = cudaMemcpyAsync(d_tab, pl->job_slot[slot].data(), kJobSlotBytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            pl->job_slot[slot].clear();
            return cuda_fail(pl, "cudaMemcpyAsync(job table)", e);
        }
    }
    e = launch_gather_table(reinterpret_cast<const GatherParams *>(d_tab),
                            reinterpret_cast<const int *>(d_tab + sizeof(GatherParams) * SWIH_MAX_SCALES), n_windows,
                            (int)total, jobs[0], kind, pl->elem_bytes, jobs[0].gdx, jobs[0].gdy, sh, s);
    if (e != cudaSuccess) return cuda_fail(pl, "gather launch", e);
    return SWIH_OK;
}

swih_status swih_sync_status(swih_plan_t pl, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(pl, "cudaStreamSynchronize", e);
    uint32_t word = 0;
    e = cudaMemcpy(&word, pl->d_status, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(pl, "cudaMemcpy(status)", e);
    if (word) {
        e = cudaMemset(pl->d_status, 0, sizeof word);
        if (e != cudaSuccess) return cuda_fail(pl, "cudaMemset(status)", e);
        if (word & kStatusTimeout)
            return fail(pl, SWIH_ERR_TIMEOUT, "integral-histogram scan: a look-back wait gave up");
    }
    return SWIH_OK;
}

swih_status swih_destroy(swih_plan_t pl)
{
    if (!pl) return SWIH_OK;
    cudaError_t e = cudaSuccess;
    if (pl->d_mem) e = cudaFree(pl->d_mem);
    delete pl;
    if (e != cudaSuccess) return cuda_fail(nullptr, "cudaFree", e);
    return SWIH_OK;
}

swih_status swih_plan_load_bytes(swih_plan_t pl, uint64_t *bytes, int reset)
{
    if (!pl || !bytes) return fail(pl, SWIH_ERR_INVALID_ARG, "plan and bytes are required");
    unsigned long long *d = reinterpret_cast<unsigned long long *>(pl->d_status + 2);
    cudaError_t e = cudaMemcpy(bytes, d, sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(d, 0, sizeof(uint64_t));
    if (e != cudaSuccess) return cuda_fail(pl, "cudaMemcpy(load bytes)", e);
    return SWIH_OK;
}

swih_status swih_launch_count(uint64_t *count)
{
    if (!count) return fail(nullptr, SWIH_ERR_INVALID_ARG, "count is NULL");
    *count = g_launches.load(std::memory_order_relaxed);
    return SWIH_OK;
}

const char *swih_last_error(swih_plan_t pl)
{
    if (pl) return pl->err.c_str();
    return g_err.c_str();
}

swih_status swih_debug_inject(swih_plan_t pl, int what)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (what != 0 && what != SWIH_INJECT_STALL_SCAN_TILE && what != SWIH_INJECT_DIRECT_GATHER)
        return fail(pl, SWIH_ERR_INVALID_ARG, "unknown injection");
    if (what == SWIH_INJECT_DIRECT_GATHER) {
        pl->gather_path = 1;
        return SWIH_OK;
    }
    if (what == 0) pl->gather_path = 0;
    pl->inject = what;
    return SWIH_OK;
}

swih_status swih_set_gather_config(swih_plan_t pl, int kernel, int tile_cols, int stages,
                                   int bins_per_step)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (kernel == SWIH_KERNEL_EXPONENTIAL)
        return fail(pl, SWIH_ERR_UNSUPPORTED, "the exponential kernel has no tiled gather to configure");
    if (kernel < SWIH_KERNEL_PLAIN || kernel > SWIH_KERNEL_WEDDING)
        return fail(pl, SWIH_ERR_INVALID_ARG, "unknown kernel");
    if (tile_cols != 0 && tile_cols != 128 && tile_cols != 256)
        return fail(pl, SWIH_ERR_INVALID_ARG, "tile_cols must be 0, 128 or 256");
    if (stages != 0 && (stages < 2 || stages > 8))
        return fail(pl, SWIH_ERR_INVALID_ARG, "stages must be 0 or 2..8");
    if (bins_per_step != 0 && bins_per_step != 2 && bins_per_step != 4 && bins_per_step != 8)
        return fail(pl, SWIH_ERR_INVALID_ARG, "bins_per_step must be 0, 2, 4 or 8");
    pl->cfg_tx[kernel] = tile_cols;
    pl->cfg_stages[kernel] = stages;
    pl->cfg_bb[kernel] = bins_per_step;
    return SWIH_OK;
}

swih_status swih_plan_get_info(swih_plan_t pl, swih_plan_info *info)
{
    if (!pl || !info) return fail(pl, SWIH_ERR_INVALID_ARG, "plan or info is NULL");
    std::memset(info, 0, sizeof *info);
    info->height = pl->desc.height;
    info->width = pl->desc.width;
    info->bins = pl->desc.bins;
    info->elem_bytes = pl->elem_bytes;
    info->n_terms = pl->n_terms;
    for (int t = 0; t < pl->n_terms; ++t) {
        info->term_p[t] = pl->term_p[t];
        info->term_q[t] = pl->term_q[t];
    }
    info->d_bins = pl->d_mem;
    info->bins_pitch = pl->bins_pitch;
    info->d_ih = pl->d_mem ? pl->d_mem + pl->off_ih : nullptr;
    info->ih_pitch = pl->ih_pitch;
    info->plane_elems = pl->plane;
    info->band_rows = pl->band_rows;
    info->n_bands = pl->n_bands;
    info->workspace_bytes = pl->total;
    if (pl->has_exp) {
        info->d_exp = pl->d_mem + pl->off_exp;
        info->exp_frac_bits = pl->exp_F;
    }
    if (pl->sparse_rows && pl->d_mem) info->d_row_map = reinterpret_cast<const int32_t *>(pl->d_mem + pl->off_row_map);
    info->n_channels = pl->n_ch > 0 ? pl->n_ch : 1;
    return SWIH_OK;
}

}  // extern "C"
