/*
 * Brute-force spatially weighted local histograms -- CPU test oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg do. It shares no code with the CUDA library.
 *
 * What it computes is the paper's "brute-force approach" (Sec. 2, the
 * convolution-style method whose cost is O(b k^2 w h)): for every candidate
 * centre c = (xc, yc) and every bin b,
 *
 *     U_c(b) = sum_{dy=-ry..ry} sum_{dx=-rx..rx} K(dx, dy) * [bin(xc+dx, yc+dy) == b]
 *
 * visiting every pixel of the window, in FP64, in plain loop order. The
 * weight table K (h rows by w columns, K[(dy+ry)*w + (dx+rx)]) is supplied
 * by the caller, so the kernel definitions live beside their citations in
 * swih_oracle.py. Normalisation divides by the window's actual total
 * sum_b U_c(b), and the similarity is the Bhattacharyya coefficient
 * sum_b sqrt(H_c(b) q(b)).
 *
 * Bins are one byte per pixel, row-major H x W, values in [0, B).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int swih_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* U for one centre into u[0..B) (zeroed here). */
static void window_hist(const uint8_t *bins, int W, int B, const double *K, int w, int h,
                        int xc, int yc, double *u)
{
    const int rx = (w - 1) / 2, ry = (h - 1) / 2;
    for (int b = 0; b < B; ++b) u[b] = 0.0;
    for (int dy = -ry; dy <= ry; ++dy) {
        const uint8_t *row = bins + (size_t)(yc + dy) * (size_t)W;
        const double *krow = K + (size_t)(dy + ry) * (size_t)w;
        for (int dx = -rx; dx <= rx; ++dx) {
            u[row[xc + dx]] += krow[dx + rx];
        }
    }
}

/* Bhattacharyya coefficient of the normalised histogram u / sum(u) against q. */
static double bhattacharyya(const double *u, const double *q, int B)
{
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += u[b];
    double l = 0.0;
    for (int b = 0; b < B; ++b) l += sqrt((u[b] / s) * q[b]);
    return l;
}

/* Unnormalised histograms U for the centres (cx[i], cy[i]), i < n, into U[i*B + b]. */
void swih_oracle_hist_at(const uint8_t *bins, int H, int W, int B, const double *K, int w,
                         int h, const int *cx, const int *cy, long n, double *U)
{
    (void)H;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) window_hist(bins, W, B, K, w, h, cx[i], cy[i], U + i * B);
}

/* Unnormalised histograms for a rectangle of centres: xc in [cx0, cx0+ncx),
 * yc in [cy0, cy0+ncy); U[((yc-cy0)*ncx + (xc-cx0))*B + b]. */
void swih_oracle_hist_rect(const uint8_t *bins, int H, int W, int B, const double *K, int w,
                           int h, int cx0, int cy0, int ncx, int ncy, double *U)
{
    (void)H;
    const long n = (long)ncx * (long)ncy;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
        const int xc = cx0 + (int)(i % ncx), yc = cy0 + (int)(i / ncx);
        window_hist(bins, W, B, K, w, h, xc, yc, U + i * B);
    }
}

/* Likelihood L[i] = Bhattacharyya(U_ci / sum U_ci, q) for listed centres. */
void swih_oracle_likelihood_at(const uint8_t *bins, int H, int W, int B, const double *K,
                               int w, int h, const int *cx, const int *cy, long n,
                               const double *q, double *L)
{
    (void)H;
#pragma omp parallel
    {
        double *u = (double *)malloc(sizeof(double) * (size_t)B);
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < n; ++i) {
            window_hist(bins, W, B, K, w, h, cx[i], cy[i], u);
            L[i] = bhattacharyya(u, q, B);
        }
        free(u);
    }
}

/* Likelihood over a rectangle of centres, L[(yc-cy0)*ncx + (xc-cx0)]. */
void swih_oracle_likelihood_rect(const uint8_t *bins, int H, int W, int B, const double *K,
                                 int w, int h, int cx0, int cy0, int ncx, int ncy,
                                 const double *q, double *L)
{
    (void)H;
    const long n = (long)ncx * (long)ncy;
#pragma omp parallel
    {
        double *u = (double *)malloc(sizeof(double) * (size_t)B);
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < n; ++i) {
            const int xc = cx0 + (int)(i % ncx), yc = cy0 + (int)(i / ncx);
            window_hist(bins, W, B, K, w, h, xc, yc, u);
            L[i] = bhattacharyya(u, q, B);
        }
        free(u);
    }
}
