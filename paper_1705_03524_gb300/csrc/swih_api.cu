// Host side of the C ABI declared in include/swih.h: plan construction,
// argument validation, kernel parameters and launches. No compute happens
// here; every step of the pipeline runs in the CUDA kernels K1-K3.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "swih.h"
#include "swih_internal.h"

using namespace swih;

struct swih_plan_s {
    swih_plan_desc desc;
    int elem_bytes = 4;
    int n_terms = 0;
    int term_p[kMaxTerms];
    int term_q[kMaxTerms];
    int term_index[5][5];  // [p][q] -> term or -1
    // scan chains: distinct q values and their p lists
    int n_q = 0;
    int q_val[kMaxQ];
    int p_count[kMaxQ];
    int p_val[kMaxQ][kMaxP];
    int gauss_degree = 2;
    double sigma_frac = 0.25;
    int64_t bins_pitch = 0, ih_pitch = 0, plane = 0;
    int band_rows = 0, n_bands = 0;
    int scan_E = 4, scan_threads = 32;
    uint64_t off_ih = 0, off_agg = 0, off_incl = 0, off_flags = 0, total = 0;
    uint64_t flags_bytes = 0;
    char *d_mem = nullptr;
    uint32_t *d_status = nullptr;
    int device = 0;
    bool built = false;
    int inject = 0;  // SWIH_INJECT_* for the next swih_build_ih
    int gather_path = 0;  // 0: tiled when it fits, 1: direct gather only
    int cfg_tx[4] = {0, 0, 0, 0};      // tiled gather tile width per kernel (0: automatic)
    int cfg_stages[4] = {0, 0, 0, 0};  // tiled gather ring depth per kernel (0: automatic)
    int cfg_bb[4] = {0, 0, 0, 0};      // tiled gather bins per step per kernel (0: automatic)
    std::string err;
};

namespace {

thread_local std::string g_err;

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

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

inline bool odd_window(int w) { return w >= 3 && (w & 1); }

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
    double A[3][4] = {};
    for (int d = -r; d <= r; ++d) {
        const double t = (double)d * d / ((double)r * r);
        const double y = std::exp(-(double)d * d / (2.0 * sigma * sigma));
        const double pw[3] = {1.0, t, t * t};
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

struct GaussAxis {
    int D = 0;
    double beta[3] = {0, 0, 0};  // Bernstein coefficients of the fitted polynomial
    double mass = 0;             // sum over d = -r..r of P(d^2 / r^2)
};

bool gauss_axis(int r, double sigma, int D_req, GaussAxis &g, std::string &why)
{
    g.D = gauss_axis_degree(r, D_req);
    double c[3] = {0, 0, 0};
    if (g.D < 1) {
        why = "Gaussian window half-size must be >= 1";
        return false;
    }
    if (!gauss_fit(r, sigma, g.D, c)) {
        why = "Gaussian least-squares system is singular";
        return false;
    }
    // power basis -> Bernstein basis: beta_i = sum_{k<=i} C(i,k)/C(D,k) c_k
    if (g.D == 1) {
        g.beta[0] = c[0];
        g.beta[1] = c[0] + c[1];
    } else {
        g.beta[0] = c[0];
        g.beta[1] = c[0] + 0.5 * c[1];
        g.beta[2] = c[0] + c[1] + c[2];
    }
    for (int i = 0; i <= g.D; ++i)
        if (!(g.beta[i] >= 0.0)) {
            why = "Gaussian approximant has a negative Bernstein coefficient for this window";
            return false;
        }
    g.mass = 0.0;
    for (int d = -r; d <= r; ++d) {
        const double t = (double)d * d / ((double)r * r);
        g.mass += c[0] + t * (c[1] + t * c[2]);
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
    if (d->kernel_mask == 0 || (d->kernel_mask & ~0xFu))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "kernel_mask must name kernels 0..3");
    if (!odd_window(d->max_win_w) || !odd_window(d->max_win_h))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "max window sides must be odd and >= 3");
    if (d->max_win_w > d->width || d->max_win_h > d->height)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "max window larger than the image");
    if (d->precision < SWIH_PREC_AUTO || d->precision > SWIH_PREC_RING64)
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "precision out of range");
    if (d->band_rows < 0) return fail(nullptr, SWIH_ERR_INVALID_ARG, "band_rows must be >= 0");
    const int D = d->gauss_degree == 0 ? 2 : d->gauss_degree;
    if (D < 1 || D > 2) return fail(nullptr, SWIH_ERR_UNSUPPORTED, "gauss_degree must be 1 or 2");
    const double sf = d->gauss_sigma_frac == 0.0 ? 0.25 : d->gauss_sigma_frac;
    if (!(sf > 0.0) || !std::isfinite(sf))
        return fail(nullptr, SWIH_ERR_INVALID_ARG, "gauss_sigma_frac must be positive");

    pl->desc = *d;
    pl->gauss_degree = D;
    pl->sigma_frac = sf;
    bool mark[5][5] = {};
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
    for (int q = 0; q < 5; ++q) {
        int cnt = 0;
        for (int p = 0; p < 5; ++p) {
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
    const bool fits32 = !want_gau && need < 4294967296.0L;
    if (want_gau && gauss_bound(d->max_win_w, d->max_win_h, D) >= 18446744073709551616.0L)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED,
                    "Gaussian window too large for exact 64-bit moments (w*h*rx^2D*ry^2D >= 2^64)");
    if (d->precision == SWIH_PREC_RING32 && !fits32)
        return fail(nullptr, SWIH_ERR_UNSUPPORTED,
                    "RING32 is not exact for these kernels and windows; use AUTO or RING64");
    pl->elem_bytes = (d->precision == SWIH_PREC_RING64 || !fits32) ? 8 : 4;

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
    take((uint64_t)H * pl->bins_pitch);  // bins at offset 0
    pl->off_ih = take((uint64_t)pl->n_terms * d->bins * pl->plane * es);
    pl->off_agg = take(n_chains * pl->n_bands * pl->ih_pitch * es);
    pl->off_incl = take(n_chains * pl->n_bands * pl->ih_pitch * es);
    pl->flags_bytes = (n_chains * pl->n_bands + 1) * sizeof(int);  // flags + ticket
    pl->off_flags = take(pl->flags_bytes);
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
    if (kernel < SWIH_KERNEL_PLAIN || kernel > SWIH_KERNEL_GAUSSIAN)
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

swih_status make_gather(swih_plan_s *pl, int kernel, int w, int h, GatherParams &g, int &kind)
{
    std::memset(&g, 0, sizeof g);
    g.ih = pl->d_mem + pl->off_ih;
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
    g.want_tx = pl->cfg_tx[kernel];
    g.want_stages = pl->cfg_stages[kernel];
    g.want_bb = pl->cfg_bb[kernel];
    if (kernel == SWIH_KERNEL_GAUSSIAN) {
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

}  // namespace

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

swih_status swih_build_ih(swih_plan_t pl, const void *d_image, void *stream)
{
    if (!pl) return fail(nullptr, SWIH_ERR_INVALID_ARG, "plan is NULL");
    if (!d_image) return fail(pl, SWIH_ERR_INVALID_ARG, "d_image is NULL");
    const swih_plan_desc &d = pl->desc;
    if (d.pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_image) & 1))
        return fail(pl, SWIH_ERR_INVALID_ARG, "a U16 image must be 2-byte aligned");
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

    e = cudaMemsetAsync(pl->d_mem + pl->off_flags, 0, pl->flags_bytes, s);
    if (e != cudaSuccess) return cuda_fail(pl, "cudaMemsetAsync(scan flags)", e);

    ScanParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.bins = qp.bins;
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
    if (pl->inject == SWIH_INJECT_STALL_SCAN_TILE) {
        sp.stall_tile = 0;        // chain 0, band 0 never publishes
        sp.spin_limit = 1LL << 12;
        pl->inject = 0;
    }
    e = launch_ih_scan(sp, pl->elem_bytes, pl->scan_E, pl->scan_threads, s);
    if (e != cudaSuccess) return cuda_fail(pl, "ih_scan launch", e);
    pl->built = true;
    return SWIH_OK;
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
    if (kernel < SWIH_KERNEL_PLAIN || kernel > SWIH_KERNEL_GAUSSIAN)
        return fail(pl, SWIH_ERR_INVALID_ARG, "unknown kernel");
    if (tile_cols != 0 && tile_cols != 128 && tile_cols != 256)
        return fail(pl, SWIH_ERR_INVALID_ARG, "tile_cols must be 0, 128 or 256");
    if (stages != 0 && (stages < 2 || stages > 8))
        return fail(pl, SWIH_ERR_INVALID_ARG, "stages must be 0 or 2..8");
    if (bins_per_step != 0 && bins_per_step != 4 && bins_per_step != 8)
        return fail(pl, SWIH_ERR_INVALID_ARG, "bins_per_step must be 0, 4 or 8");
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
    return SWIH_OK;
}

}  // extern "C"

// ============================================================================
// Batches: many regions of interest of one frame in a fixed set of launches
// (see swih.h). Built from the same layout rules and job parameters as plans.
// ============================================================================
#include <vector>

struct swih_batch_s {
    swih_batch_desc desc;
    std::vector<swih_roi_desc> rois;
    swih_plan_s tmpl;  // term set, ring and Gaussian settings shared by every ROI
    struct Roi {
        int H, W, n_bands;
        int64_t bins_pitch, ih_pitch, plane;
        uint64_t off_bins, off_ih, off_agg, off_incl, off_flags;
        int ticket0;
        long long chunk0;
    };
    std::vector<Roi> r;
    int scan_E = 4, scan_threads = 32, band_rows = 32;
    long long scan_tiles = 0, quant_chunks = 0;
    uint64_t flags_ints = 0;
    uint64_t off_flags_all = 0, off_quant = 0, off_scan = 0, off_jobs = 0, off_items = 0, off_status = 0;
    uint64_t total = 0;
    struct Group {
        int kind, gdx, gdy;
        int job_begin, job_end;  // jobs[job_begin, job_end)
        bool tiled;
        GatherShape shape;
        int n_items;
        int want_tx = 0, want_stages = 0, want_bb = 0;
    };
    std::vector<Group> groups;
    std::vector<GatherParams> jobs;
    std::vector<int> items;  // per group: item_start of its jobs (job_end - job_begin + 1 entries), concatenated
    std::vector<int> items_off;
    char *d_mem = nullptr;
    uint32_t *d_status = nullptr;
    const void *d_frame = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
};

namespace {

swih_status bfail(swih_batch_s *b, swih_status st, const std::string &msg)
{
    if (b) b->err = msg;
    g_err = msg;
    return st;
}

swih_status bcuda(swih_batch_s *b, const char *what, cudaError_t e)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return bfail(b, e == cudaErrorMemoryAllocation ? SWIH_ERR_OOM : SWIH_ERR_CUDA, m);
}

// Lay out a batch (host only). One template layout, built for the largest ROI
// and the largest window of any ROI, fixes the term set and the ring for all;
// each ROI then gets its own pitches and bands. On success b->total holds the
// workspace size.
swih_status batch_layout(const swih_batch_desc *d, const swih_roi_desc *rois, int n, swih_batch_s *b)
{
    if (!d || !rois || n < 1) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "desc, rois and n_rois >= 1 required");
    if (n > (1 << 20)) return bfail(nullptr, SWIH_ERR_UNSUPPORTED, "more than 2^20 ROIs in one batch");
    if (d->height < 3 || d->width < 3) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "frame must be at least 3 x 3");
    const int pb = d->pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    if (d->pitch_bytes < (int64_t)d->width * pb)
        return bfail(nullptr, SWIH_ERR_INVALID_ARG, "pitch_bytes smaller than a frame row");
    if (d->band_rows < 0) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "band_rows must be >= 0");
    b->desc = *d;
    b->rois.assign(rois, rois + n);
    int maxH = 3, maxW = 3, mw = 3, mh = 3;
    for (int i = 0; i < n; ++i) {
        const swih_roi_desc &ro = rois[i];
        const std::string tag = "ROI " + std::to_string(i);
        if (ro.width < 3 || ro.height < 3 || ro.x0 < 0 || ro.y0 < 0 ||
            (int64_t)ro.x0 + ro.width > d->width || (int64_t)ro.y0 + ro.height > d->height)
            return bfail(nullptr, SWIH_ERR_INVALID_ARG, tag + " is not inside the frame");
        if (ro.kernel < SWIH_KERNEL_PLAIN || ro.kernel > SWIH_KERNEL_GAUSSIAN ||
            !(d->kernel_mask & SWIH_KERNEL_BIT(ro.kernel)))
            return bfail(nullptr, SWIH_ERR_INVALID_ARG, tag + ": kernel not in kernel_mask");
        if (ro.n_windows < 1 || ro.n_windows > SWIH_MAX_SCALES)
            return bfail(nullptr, SWIH_ERR_INVALID_ARG, tag + ": n_windows out of range");
        if (!ro.d_target) return bfail(nullptr, SWIH_ERR_INVALID_ARG, tag + ": d_target is NULL");
        for (int k = 0; k < ro.n_windows; ++k) {
            if (!odd_window(ro.win_w[k]) || !odd_window(ro.win_h[k]) || ro.win_w[k] > ro.width ||
                ro.win_h[k] > ro.height || !ro.d_map[k])
                return bfail(nullptr, SWIH_ERR_INVALID_ARG, tag + ": window " + std::to_string(k) + " invalid");
            mw = std::max(mw, ro.win_w[k]);
            mh = std::max(mh, ro.win_h[k]);
        }
        maxH = std::max(maxH, ro.height);
        maxW = std::max(maxW, ro.width);
    }
    swih_plan_desc pd;
    std::memset(&pd, 0, sizeof pd);
    pd.height = maxH;
    pd.width = maxW;
    pd.pitch_bytes = d->pitch_bytes;
    pd.pixel_type = d->pixel_type;
    pd.bitdepth = d->bitdepth;
    pd.bins = d->bins;
    pd.kernel_mask = d->kernel_mask;
    pd.gauss_degree = d->gauss_degree;
    pd.gauss_sigma_frac = d->gauss_sigma_frac;
    pd.max_win_w = mw;
    pd.max_win_h = mh;
    pd.precision = d->precision;
    pd.band_rows = 0;
    const swih_status st = build_layout(&pd, &b->tmpl);
    if (st != SWIH_OK) return st;
    // scan launch shape (the widest ROI decides) and one band height for all
    b->scan_E = b->tmpl.scan_E;
    b->scan_threads = b->tmpl.scan_threads;
    b->band_rows = d->band_rows > 0 ? d->band_rows : 32;
    // arena
    const uint64_t es = (uint64_t)b->tmpl.elem_bytes;
    const uint64_t n_chains = (uint64_t)d->bins * b->tmpl.n_q;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    long long ticket = 0, chunk = 0;
    uint64_t flag_ints = 0;
    b->r.clear();
    for (int i = 0; i < n; ++i) {
        swih_batch_s::Roi R;
        R.H = rois[i].height;
        R.W = rois[i].width;
        R.n_bands = (R.H + b->band_rows - 1) / b->band_rows;
        R.bins_pitch = round_up(R.W, 128);
        R.ih_pitch = round_up(R.W, 32);
        R.plane = (int64_t)R.H * R.ih_pitch;
        R.off_bins = take((uint64_t)R.H * R.bins_pitch);
        R.off_ih = take((uint64_t)b->tmpl.n_terms * d->bins * R.plane * es);
        R.off_agg = take(n_chains * R.n_bands * R.ih_pitch * es);
        R.off_incl = take(n_chains * R.n_bands * R.ih_pitch * es);
        R.off_flags = flag_ints;  // index into the shared flag array
        flag_ints += n_chains * R.n_bands;
        R.ticket0 = (int)ticket;
        ticket += (long long)(n_chains * R.n_bands);
        R.chunk0 = chunk;
        chunk += (long long)((R.W + 15) / 16) * R.H;
        if (ticket > (1LL << 30)) return bfail(nullptr, SWIH_ERR_UNSUPPORTED, "too many scan tiles in one batch");
        b->r.push_back(R);
    }
    b->scan_tiles = ticket;
    b->quant_chunks = chunk;
    b->flags_ints = flag_ints + 1;  // + the ticket counter
    b->off_flags_all = take(b->flags_ints * sizeof(int));
    b->off_quant = take(sizeof(QuantRoi) * n);
    b->off_scan = take(sizeof(ScanRoi) * n);
    size_t n_jobs = 0;
    for (int i = 0; i < n; ++i) n_jobs += rois[i].n_windows;
    b->off_jobs = take(sizeof(GatherParams) * n_jobs);
    b->off_items = take(sizeof(int) * (n_jobs + 16) * 2);
    b->off_status = take(sizeof(uint32_t) * 64);
    b->total = off;
    if (d->hbm_budget_bytes && b->total > d->hbm_budget_bytes) {
        char m[160];
        std::snprintf(m, sizeof m, "batch workspace %llu bytes exceeds the budget of %llu bytes",
                      (unsigned long long)b->total, (unsigned long long)d->hbm_budget_bytes);
        return bfail(nullptr, SWIH_ERR_BUDGET, m);
    }
    return SWIH_OK;
}

// Build the gather jobs and groups (host), with the groups' current wants.
swih_status batch_jobs(swih_batch_s *b)
{
    const int n = (int)b->rois.size();
    std::vector<GatherParams> jobs;
    std::vector<int> job_kind;
    for (int i = 0; i < n; ++i) {
        const swih_roi_desc &ro = b->rois[i];
        const swih_batch_s::Roi &R = b->r[i];
        swih_plan_s fake = b->tmpl;  // term indices, ring, Gaussian settings
        fake.desc.height = R.H;
        fake.desc.width = R.W;
        fake.desc.bins = b->desc.bins;
        fake.plane = R.plane;
        fake.ih_pitch = R.ih_pitch;
        fake.d_mem = b->d_mem + R.off_ih;
        fake.off_ih = 0;
        fake.d_status = b->d_status;
        for (int k = 0; k < ro.n_windows; ++k) {
            GatherParams g;
            int kind = 0;
            const swih_status st = make_gather(&fake, ro.kernel, ro.win_w[k], ro.win_h[k], g, kind);
            if (st != SWIH_OK) return bfail(b, st, "ROI " + std::to_string(i) + ": " + fake.err);
            g.cx0 = g.rx;
            g.cy0 = g.ry;
            g.ncx = R.W - ro.win_w[k] + 1;
            g.ncy = R.H - ro.win_h[k] + 1;
            g.target = ro.d_target;
            g.map = ro.d_map[k];
            g.hist = nullptr;
            jobs.push_back(g);
            job_kind.push_back(kind);
        }
    }
    // group by (kind, fitted degrees), keeping the previous wants
    std::vector<swih_batch_s::Group> old = b->groups;
    b->groups.clear();
    b->jobs.clear();
    std::vector<int> order(jobs.size());
    for (size_t j = 0; j < jobs.size(); ++j) order[j] = (int)j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int kx = job_kind[x] * 16 + jobs[x].gdx * 4 + jobs[x].gdy;
        const int ky = job_kind[y] * 16 + jobs[y].gdx * 4 + jobs[y].gdy;
        return kx < ky;
    });
    for (size_t idx = 0; idx < order.size(); ++idx) {
        const GatherParams &g = jobs[order[idx]];
        const int kind = job_kind[order[idx]];
        if (b->groups.empty() || b->groups.back().kind != kind || b->groups.back().gdx != g.gdx ||
            b->groups.back().gdy != g.gdy) {
            swih_batch_s::Group G;
            G.kind = kind;
            G.gdx = g.gdx;
            G.gdy = g.gdy;
            G.job_begin = (int)b->jobs.size();
            G.job_end = G.job_begin;
            G.tiled = true;
            G.n_items = 0;
            for (auto &o : old)
                if (o.kind == kind && o.gdx == g.gdx && o.gdy == g.gdy) {
                    G.want_tx = o.want_tx;
                    G.want_stages = o.want_stages;
                    G.want_bb = o.want_bb;
                }
            b->groups.push_back(G);
        }
        b->jobs.push_back(g);
        b->groups.back().job_end = (int)b->jobs.size();
    }
    // shapes and work items per group
    b->items.clear();
    b->items_off.clear();
    for (auto &G : b->groups) {
        int max_w = 3;
        for (int j = G.job_begin; j < G.job_end; ++j) max_w = std::max(max_w, 2 * b->jobs[j].rx + 1);
        const GatherParams &g0 = b->jobs[G.job_begin];
        const cudaError_t e = tiled_shape(G.kind, b->tmpl.elem_bytes, G.gdx, G.gdy, max_w, b->desc.bins, g0.nl,
                                          G.want_tx, G.want_stages, G.want_bb, &G.shape);
        G.tiled = e == cudaSuccess;
        b->items_off.push_back((int)b->items.size());
        int items = 0;
        for (int j = G.job_begin; j < G.job_end; ++j) {
            b->items.push_back(items);
            if (G.tiled) {
                items += tiled_items(&b->jobs[j], G.shape);
                if ((long long)items > (1LL << 30))
                    return bfail(b, SWIH_ERR_UNSUPPORTED, "too many work items in one batch");
            }
        }
        b->items.push_back(items);
        G.n_items = items;
    }
    return SWIH_OK;
}

swih_status batch_upload(swih_batch_s *b)
{
    cudaError_t e = cudaMemcpy(b->d_mem + b->off_jobs, b->jobs.data(), sizeof(GatherParams) * b->jobs.size(),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_mem + b->off_items, b->items.data(), sizeof(int) * b->items.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, "cudaMemcpy(batch jobs)", e);
    return SWIH_OK;
}

// enqueue one gather group
cudaError_t batch_gather_group(swih_batch_s *b, size_t gi, cudaStream_t s)
{
    const swih_batch_s::Group &G = b->groups[gi];
    if (G.tiled) {
        const GatherParams *d_jobs = reinterpret_cast<const GatherParams *>(b->d_mem + b->off_jobs) + G.job_begin;
        const int *d_items = reinterpret_cast<const int *>(b->d_mem + b->off_items) + b->items_off[gi];
        return launch_gather_table(d_jobs, d_items, G.job_end - G.job_begin, G.n_items, b->jobs[G.job_begin],
                                   G.kind, b->tmpl.elem_bytes, G.gdx, G.gdy, G.shape, s);
    }
    for (int j = G.job_begin; j < G.job_end; ++j) {
        const cudaError_t e = launch_gather(b->jobs[j], G.kind, b->tmpl.elem_bytes, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// enqueue the whole batch (not captured)
swih_status batch_enqueue(swih_batch_s *b, cudaStream_t s)
{
    const swih_batch_desc &d = b->desc;
    cudaError_t e = cudaMemsetAsync(b->d_mem + b->off_flags_all, 0, b->flags_ints * sizeof(int), s);
    if (e != cudaSuccess) return bcuda(b, "cudaMemsetAsync(batch flags)", e);
    e = launch_quantize_table(reinterpret_cast<const QuantRoi *>(b->d_mem + b->off_quant), (int)b->rois.size(),
                              b->quant_chunks, d.bins, d.bitdepth, d.pixel_type == SWIH_PIXEL_U16 ? 2 : 1, s);
    if (e != cudaSuccess) return bcuda(b, "batched quantize launch", e);
    ScanParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.B = d.bins;
    sp.band_rows = b->band_rows;
    sp.n_q = b->tmpl.n_q;
    for (int i = 0; i < b->tmpl.n_q; ++i) {
        sp.q_val[i] = b->tmpl.q_val[i];
        sp.p_count[i] = b->tmpl.p_count[i];
        for (int k = 0; k < b->tmpl.p_count[i]; ++k) {
            sp.p_val[i][k] = b->tmpl.p_val[i][k];
            sp.term[i][k] = b->tmpl.term_index[b->tmpl.p_val[i][k]][b->tmpl.q_val[i]];
        }
    }
    sp.ticket = reinterpret_cast<int *>(b->d_mem + b->off_flags_all) + (b->flags_ints - 1);
    sp.status = b->d_status;
    sp.spin_limit = 1LL << 22;
    sp.stall_tile = -1;
    e = launch_ih_scan_table(sp, reinterpret_cast<const ScanRoi *>(b->d_mem + b->off_scan), (int)b->rois.size(),
                             b->scan_tiles, b->tmpl.elem_bytes, b->scan_E, b->scan_threads, s);
    if (e != cudaSuccess) return bcuda(b, "batched scan launch", e);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        e = batch_gather_group(b, gi, s);
        if (e != cudaSuccess) return bcuda(b, "batched gather launch", e);
    }
    return SWIH_OK;
}

swih_status batch_capture(swih_batch_s *b)
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
    if (e != cudaSuccess) return bcuda(b, "cudaStreamBeginCapture", e);
    const swih_status st = batch_enqueue(b, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != SWIH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return bcuda(b, "cudaStreamEndCapture", e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return bcuda(b, "cudaGraphInstantiate", e);
    return SWIH_OK;
}

}  // namespace

extern "C" {

swih_status swih_batch_workspace_bytes(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois,
                                       uint64_t *bytes)
{
    if (!bytes) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "bytes is NULL");
    swih_batch_s tmp;
    swih_batch_desc d2;
    if (desc) {
        d2 = *desc;
        d2.hbm_budget_bytes = 0;
    }
    const swih_status st = batch_layout(desc ? &d2 : nullptr, rois, n_rois, &tmp);
    if (st != SWIH_OK) return st;
    *bytes = tmp.total;
    return SWIH_OK;
}

swih_status swih_batch_plan(const swih_batch_desc *desc, const swih_roi_desc *rois, int n_rois,
                            const void *d_frame, swih_batch_t *out)
{
    if (!out) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d_frame) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "d_frame is NULL");
    if (desc && desc->pixel_type == SWIH_PIXEL_U16 && (reinterpret_cast<uintptr_t>(d_frame) & 1))
        return bfail(nullptr, SWIH_ERR_INVALID_ARG, "a U16 frame must be 2-byte aligned");
    swih_batch_s *b = new swih_batch_s();
    swih_status st = batch_layout(desc, rois, n_rois, b);
    if (st != SWIH_OK) {
        delete b;
        return st;
    }
    b->d_frame = d_frame;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_mem), b->total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bcuda(nullptr, "cudaMalloc(batch workspace)", e);
    }
    b->d_status = reinterpret_cast<uint32_t *>(b->d_mem + b->off_status);
    e = cudaMemset(b->d_status, 0, sizeof(uint32_t) * 64);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(b->d_mem);
        delete b;
        return bcuda(nullptr, "batch set-up", e);
    }
    // region tables
    const int pb = desc->pixel_type == SWIH_PIXEL_U16 ? 2 : 1;
    std::vector<QuantRoi> qt(n_rois);
    std::vector<ScanRoi> stt(n_rois);
    const uint64_t n_chains = (uint64_t)desc->bins * b->tmpl.n_q;
    for (int i = 0; i < n_rois; ++i) {
        const swih_batch_s::Roi &R = b->r[i];
        const uint8_t *img = static_cast<const uint8_t *>(d_frame) + (int64_t)rois[i].y0 * desc->pitch_bytes +
                             (int64_t)rois[i].x0 * pb;
        qt[i].image = img;
        qt[i].pitch = desc->pitch_bytes;
        qt[i].H = R.H;
        qt[i].W = R.W;
        qt[i].bins = reinterpret_cast<uint8_t *>(b->d_mem + R.off_bins);
        qt[i].bins_pitch = R.bins_pitch;
        qt[i].chunk0 = R.chunk0;
        qt[i].vec = (desc->pitch_bytes % 16 == 0) && (reinterpret_cast<uintptr_t>(img) % 16 == 0);
        stt[i].bins = qt[i].bins;
        stt[i].bins_pitch = R.bins_pitch;
        stt[i].ih = b->d_mem + R.off_ih;
        stt[i].ih_pitch = R.ih_pitch;
        stt[i].plane = R.plane;
        stt[i].agg = b->d_mem + R.off_agg;
        stt[i].incl = b->d_mem + R.off_incl;
        stt[i].flags = reinterpret_cast<int *>(b->d_mem + b->off_flags_all) + R.off_flags;
        stt[i].H = R.H;
        stt[i].W = R.W;
        stt[i].n_bands = R.n_bands;
        stt[i].ticket0 = R.ticket0;
        (void)n_chains;
    }
    e = cudaMemcpy(b->d_mem + b->off_quant, qt.data(), sizeof(QuantRoi) * n_rois, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_mem + b->off_scan, stt.data(), sizeof(ScanRoi) * n_rois, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        swih_batch_destroy(b);
        return bcuda(nullptr, "cudaMemcpy(batch tables)", e);
    }
    st = batch_jobs(b);
    if (st == SWIH_OK) st = batch_upload(b);
    if (st != SWIH_OK) {
        g_err = b->err;
        swih_batch_destroy(b);
        return st;
    }
    *out = b;
    return SWIH_OK;
}

swih_status swih_batch_run(swih_batch_t b, void *stream)
{
    if (!b) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "batch is NULL");
    if (!b->exec) {
        const swih_status st = batch_capture(b);
        if (st != SWIH_OK) return st;
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return bcuda(b, "cudaGraphLaunch", e);
    return SWIH_OK;
}

swih_status swih_batch_autotune(swih_batch_t b, void *stream)
{
    if (!b) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // integral histograms of the current frame, for the timings
    swih_status st = batch_enqueue(b, s);
    if (st != SWIH_OK) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const bool gau = b->groups[gi].kind == kGatherGaussian;
        float best = 1e30f;
        int bt = 0, bs = 0, bbb = 0;
        const int txs[2] = {128, 256};
        const int stages[4] = {2, 3, 4, 6};
        const int bbs[2] = {4, 8};
        for (int ti = 0; ti < 2; ++ti)
            for (int si = 0; si < 4; ++si)
                for (int bi = 0; bi < (gau ? 1 : 2); ++bi) {
                    b->groups[gi].want_tx = txs[ti];
                    b->groups[gi].want_stages = stages[si];
                    b->groups[gi].want_bb = gau ? 0 : bbs[bi];
                    st = batch_jobs(b);
                    if (st != SWIH_OK) break;
                    if (!b->groups[gi].tiled) continue;
                    st = batch_upload(b);
                    if (st != SWIH_OK) break;
                    cudaError_t e = batch_gather_group(b, gi, s);  // warm-up
                    cudaEventRecord(e0, s);
                    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = batch_gather_group(b, gi, s);
                    cudaEventRecord(e1, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) {
                        st = bcuda(b, "autotune launch", e);
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
        if (st != SWIH_OK) break;
        b->groups[gi].want_tx = bt;
        b->groups[gi].want_stages = bs;
        b->groups[gi].want_bb = bbb;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SWIH_OK) return st;
    st = batch_jobs(b);
    if (st == SWIH_OK) st = batch_upload(b);
    if (st == SWIH_OK) st = batch_capture(b);
    return st;
}

swih_status swih_batch_sync_status(swih_batch_t b, void *stream)
{
    if (!b) return bfail(nullptr, SWIH_ERR_INVALID_ARG, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return bcuda(b, "cudaStreamSynchronize", e);
    uint32_t word = 0;
    e = cudaMemcpy(&word, b->d_status, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, "cudaMemcpy(status)", e);
    if (word) {
        cudaMemset(b->d_status, 0, sizeof word);
        if (word & kStatusTimeout) return bfail(b, SWIH_ERR_TIMEOUT, "a bounded device wait gave up");
    }
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
    if (e != cudaSuccess) return bcuda(nullptr, "cudaFree", e);
    return SWIH_OK;
}

}  // extern "C"
