// K3 for the Gaussian approximant of any fitted degree (1..4 per axis), in the
// 64- or 128-bit ring: one thread per window centre, corner values read from
// the integral histograms in global memory.
//
// Per centre and bin (Sec. 2.1, Fig. 4(b): rectangle sums of the weighted
// integral histograms, translated from the image origin to the window centre):
//   1. the exact window count from the x^0 y^0 plane; a bin absent from the
//      window contributes nothing and is skipped;
//   2. for each y-power b, the window sums S_a = sum x^a y^b (a <= 2 dx) from
//      four corners each, shifted in place to the centre column, S_a <- sum
//      (x - xc)^a y^b (a Taylor shift: S_i -= xc S_{i-1}, repeated), then
//      added into the centred even moments M_kl = sum dx^2k dy^2l with the
//      binomial row shift coefficients C(2l, b) (-yc)^(2l-b);
//   3. the Bernstein moments F_ij = sum_kl ax[i][k] ay[j][l] M_kl, where
//      A_i(d) = C(D, i) d^2i (r^2 - d^2)^(D-i) = sum_k ax[i][k] d^2k; each F_ij
//      is a non-negative integer below 2^64 (or 2^128), so the ring gives it
//      exactly;
//   4. U = sum_ij gamma_ij F_ij in double (non-negative terms: no
//      cancellation), the normalised bin value, and the Bhattacharyya sums.
#include "ring128.h"
#include "swih_internal.h"

namespace swih {
namespace {

constexpr int kWThreads = 128;

template <typename T>
__device__ __forceinline__ T lohi(unsigned long long lo, unsigned long long hi)
{
    if constexpr (sizeof(T) == 16) {
        return T(lo, hi);
    } else {
        (void)hi;
        return (T)lo;
    }
}

template <typename T>
__device__ __forceinline__ T mul_u64(T a, unsigned long long f)
{
    if constexpr (sizeof(T) == 16) {
        return mul64(a, f);
    } else {
        return a * f;
    }
}

template <typename T>
__device__ __forceinline__ bool is_zero(T a)
{
    if constexpr (sizeof(T) == 16) {
        return (a.lo | a.hi) == 0ull;
    } else {
        return a == 0;
    }
}

template <typename T>
__device__ __forceinline__ double to_double(T a)
{
    if constexpr (sizeof(T) == 16) {
        return u128_to_double(a);
    } else {
        return (double)a;
    }
}

// a read-only load of one ring element (two 64-bit halves for the 128-bit ring)
template <typename T>
__device__ __forceinline__ T ld_ro(const T *p)
{
    if constexpr (sizeof(T) == 16) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        return T(v.x, v.y);
    } else {
        return __ldg(p);
    }
}

template <typename T>
__device__ __forceinline__ T select(bool c, T a)
{
    return c ? a : T(0);
}

// sum over columns (xa, xb] and rows (ra, rb] of one plane; ra, rb are stored
// rows (-1: above the image or an all-zero row), xa = -1 is left of the image.
// The four loads are unconditional (clamped to row or column 0 and masked
// afterwards), so a thread's loads of several planes can all be in flight.
template <typename T>
__device__ __forceinline__ T rect_sum(const T *__restrict__ plane, int64_t pitch, int ra, int rb, int xa, int xb)
{
    const bool va = ra >= 0, vb = rb >= 0, vx = xa >= 0;
    const T *row_a = plane + (int64_t)(va ? ra : 0) * pitch;
    const T *row_b = plane + (int64_t)(vb ? rb : 0) * pitch;
    const int xc = vx ? xa : 0;
    const T b1 = ld_ro(row_b + xb), b0 = ld_ro(row_b + xc), a1 = ld_ro(row_a + xb), a0 = ld_ro(row_a + xc);
    return select(vb, b1 - select(vx, b0)) - select(va, a1 - select(vx, a0));
}

__device__ __forceinline__ int binom_small(int n, int k)
{
    int v = 1;
    for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
    return v;
}

template <typename T, int DM>
__device__ __forceinline__ void centre(const GaussWideParams &p, const T (*s_cy)[2 * DM + 1], const float *s_sq,
                                       int nq, int ix, int iy, int cy)
{
    constexpr int NA = 2 * DM + 1;
    const int cx = p.cx0 + ix;
    const int xa = cx - p.rx - 1, xb = cx + p.rx;
    const int ya = cy - p.ry - 1, yb = cy + p.ry;
    const T *ih = static_cast<const T *>(p.ih);
    float L[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) L[t] = 0.f;
    float *hist = p.hist ? p.hist + ((int64_t)iy * p.ncx + ix) * p.B : nullptr;

    for (int b = 0; b < p.B; ++b) {
        int ra = ya, rb = yb;
        if (p.row_map) {
            ra = ya >= 0 ? p.row_map[(int64_t)b * p.H + ya] : -1;
            rb = p.row_map[(int64_t)b * p.H + yb];
        }
        const T count = rect_sum<T>(ih + ((int64_t)p.tg[0][0] * p.B + b) * p.plane, p.pitch, ra, rb, xa, xb);
        if (is_zero(count)) {
            if (hist) hist[b] = 0.f;
            continue;
        }
        T M[DM + 1][DM + 1];
#pragma unroll
        for (int k = 0; k <= DM; ++k)
#pragma unroll
            for (int l = 0; l <= DM; ++l) M[k][l] = 0;
#pragma unroll
        for (int yb_pow = 0; yb_pow < NA; ++yb_pow) {
            if (yb_pow > 2 * p.dy) break;
            T S[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a)
                S[a] = a <= 2 * p.dx ? rect_sum<T>(ih + ((int64_t)p.tg[a][yb_pow] * p.B + b) * p.plane, p.pitch, ra,
                                                   rb, xa, xb)
                                     : T(0);
            // Taylor shift to the centre column: S_a = sum (x - xc)^a y^b
#pragma unroll
            for (int j = 0; j < NA - 1; ++j)
#pragma unroll
                for (int i = NA - 1; i > j; --i) S[i] = S[i] - mul_u64<T>(S[i - 1], (unsigned long long)cx);
#pragma unroll
            for (int l = 0; l <= DM; ++l) {
                if (2 * l < yb_pow) continue;
                const T c = s_cy[l][yb_pow];
#pragma unroll
                for (int k = 0; k <= DM; ++k) M[k][l] = M[k][l] + c * S[2 * k];
            }
        }
        // Bernstein moments and the kernel-weighted, normalised bin value
        double U = 0.0;
#pragma unroll
        for (int i = 0; i <= DM; ++i) {
            if (i > p.dx) break;
            T G[DM + 1];
#pragma unroll
            for (int l = 0; l <= DM; ++l) {
                G[l] = 0;
#pragma unroll
                for (int k = 0; k <= DM; ++k) G[l] = G[l] + lohi<T>(p.ax_lo[i][k], p.ax_hi[i][k]) * M[k][l];
            }
#pragma unroll
            for (int j = 0; j <= DM; ++j) {
                if (j > p.dy) break;
                T F = 0;
#pragma unroll
                for (int l = 0; l <= DM; ++l) F = F + lohi<T>(p.ay_lo[j][l], p.ay_hi[j][l]) * G[l];
                U += p.gamma[i][j] * to_double(F);
            }
        }
        const float h = (float)U;
        if (hist) hist[b] = h;
        if (nq) {
            const float sh = sqrtf(fmaxf(h, 0.f));
#pragma unroll
            for (int t = 0; t < kMaxTargets; ++t)
                if (t < p.n_targets) L[t] += sh * s_sq[t * p.B + b];
        }
    }
    if (p.map && nq) {
#pragma unroll
        for (int t = 0; t < kMaxTargets; ++t)
            if (t < p.n_targets) p.map[(int64_t)t * p.map_stride + (int64_t)iy * p.ncx + ix] = L[t];
    }
}

template <typename T, int DM>
__global__ void __launch_bounds__(kWThreads, (sizeof(T) == 16 && DM == 4) ? 3 : 4) gauss_wide_kernel(const __grid_constant__ GaussWideParams p)
{
    constexpr int NA = 2 * DM + 1;
    __shared__ T s_cy[DM + 1][NA];  // C(2l, b) (-yc)^(2l-b) for b <= 2l
    extern __shared__ float s_sq[];  // sqrt of the targets [n_targets][B]
    const int ix = blockIdx.x * kWThreads + threadIdx.x;
    const int nq = p.target ? p.n_targets * p.B : 0;
    for (int i = threadIdx.x; i < nq; i += kWThreads) {
        const int t = i / p.B, b = i - t * p.B;
        s_sq[i] = sqrtf(fmaxf(p.target[(int64_t)t * p.target_stride + b], 0.f));
    }
    // centre rows in the order 0, h, 2h, ..., 1, 1 + h, ...: the bottom corner
    // row of a window is the top corner row of the window h rows below, so
    // blocks that run one after the other read shared rows from L2
    const int h = 2 * p.ry + 1;
    const int m = (p.ncy + h - 1) / h;
    for (int j = blockIdx.y; j < m * h; j += gridDim.y) {
        const int iy = (j % m) * h + j / m;
        if (iy >= p.ncy) continue;  // uniform over the block
        const int cy = p.cy0 + iy;
        __syncthreads();  // the previous row's coefficients are no longer read
        if (threadIdx.x == 0) {
            T pw[NA];
            pw[0] = 1;
            const T mcy = T(0) - T((unsigned long long)cy);
#pragma unroll
            for (int k = 1; k < NA; ++k) pw[k] = pw[k - 1] * mcy;
#pragma unroll
            for (int l = 0; l <= DM; ++l)
#pragma unroll
                for (int b = 0; b < NA; ++b)
                    s_cy[l][b] =
                        b <= 2 * l ? mul_u64<T>(pw[2 * l - b], (unsigned long long)binom_small(2 * l, b)) : T(0);
        }
        __syncthreads();
        if (ix < p.ncx) centre<T, DM>(p, s_cy, s_sq, nq, ix, iy, cy);
    }
}

template <typename T, int DM>
cudaError_t launch_dm(const GaussWideParams &p, cudaStream_t s)
{
    const long long rows = (long long)((p.ncy + 2 * p.ry) / (2 * p.ry + 1)) * (2 * p.ry + 1);
    const dim3 grid((unsigned)((p.ncx + kWThreads - 1) / kWThreads), (unsigned)(rows < 65535 ? rows : 65535));
    const size_t smem = p.target ? sizeof(float) * (size_t)p.n_targets * p.B : 0;
    gauss_wide_kernel<T, DM><<<grid, kWThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const GaussWideParams &p, cudaStream_t s)
{
    const int dm = p.dx > p.dy ? p.dx : p.dy;
    switch (dm) {
    case 1: return launch_dm<T, 1>(p, s);
    case 2: return launch_dm<T, 2>(p, s);
    case 3: return launch_dm<T, 3>(p, s);
    case 4: return launch_dm<T, 4>(p, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_gauss_wide(const GaussWideParams &p, int elem_bytes, cudaStream_t s)
{
    if (p.ncx <= 0 || p.ncy <= 0) return cudaSuccess;
    if (p.n_targets < 0 || p.n_targets > kMaxTargets) return cudaErrorInvalidValue;
    if (elem_bytes == 8) return launch_t<unsigned long long>(p, s);
    if (elem_bytes == 16) return launch_t<u128>(p, s);
    return cudaErrorInvalidValue;
}

}  // namespace swih
