// K3: per-window gather, translation, normalisation and matching
// (Sec. 1 steps (3)-(5), Sec. 2.1, Fig. 4(b)).
//
// One thread per window centre c = (xc, yc); a warp covers 32 consecutive
// centres of a row, so every integral-histogram read is a coalesced row
// segment of one (term, bin) plane. Corner lattice of a window:
//   X0 = xc-rx-1, X1 = xc, X2 = xc+rx,   Y0 = yc-ry-1, Y1 = yc, Y2 = yc+ry
// (IH at a -1 coordinate is 0). Rows of a bin that the scan did not store
// (no pixel of the bin) are read at the stored row that holds them, through
// the plan's row map. Rectangle sums over half-open lattice cells
// give the sums of [bin = b] * x^k y^l over each quadrant / half / window.
//
// All integer work happens in the ring T (uint32 or uint64, wrapping):
//   Manhattan  K = (rx-|dx|) + (ry-|dy|). Split at the centre column into the
//              left half (dx <= 0) and right half (dx >= 1), and at the centre
//              row into top (dy <= 0) and bottom (dy >= 1); in each piece |dx|
//              (or |dy|) is linear, so the piece needs the plain IH and IH_x
//              (or IH_y), translated by xc (or yc). This is the quadrant
//              decomposition of Sec. 2.1 written on the basis {1, x, y}.
//   Euclidean  K = (rx^2+ry^2) - dx^2 - dy^2 over the whole window, from
//              IH_1, IH_x, IH_y, IH_xx, IH_yy by the binomial translation.
//   Gaussian   K = Px(dx^2/rx^2) Py(dy^2/ry^2). The centred even moments
//              sum dx^2i dy^2j come from IH_{x^k y^l} (k, l <= 4) by binomial
//              translation; they are then mapped, still in the ring, onto the
//              Bernstein basis of each axis polynomial,
//                r^2D B_i(d^2/r^2) = C(D,i) d^2i (r^2 - d^2)^(D-i) >= 0,
//              so every per-bin quantity F_ij is a non-negative exact integer
//              and U = sum_ij beta_i beta_j F_ij / (rx^2D ry^2D) is a sum of
//              non-negative terms (the Bernstein coefficients beta of the
//              fitted polynomial are checked non-negative on the host). That
//              sum is taken in FP32 without cancellation.
// The exact integer U(b) (Manhattan / Euclidean / plain) is converted once and
// scaled by 1/M, M the kernel's total weight over the window, which does not
// depend on the window's position (Sec. 2.1). The likelihood is the
// Bhattacharyya coefficient sum_b sqrt(H(b)) sqrt(q(b)).
#include "swih_internal.h"

namespace swih {
namespace {

template <typename T>
struct Plane {
    const T *base;
    int64_t pitch;
    __device__ __forceinline__ T at(int x, int y) const
    {
        return (x >= 0 && y >= 0) ? __ldg(base + (int64_t)y * pitch + x) : T(0);
    }
    // sum over x in (xa, xb], y in (ya, yb]
    __device__ __forceinline__ T rect(int xa, int xb, int ya, int yb) const
    {
        return at(xb, yb) - at(xa, yb) - at(xb, ya) + at(xa, ya);
    }
};

template <typename T>
__device__ __forceinline__ Plane<T> plane_of(const GatherParams &p, int t, int b)
{
    Plane<T> pl;
    pl.base = reinterpret_cast<const T *>(p.ih) + ((int64_t)t * p.B + b) * p.plane;
    pl.pitch = p.pitch;
    return pl;
}

template <typename T>
__device__ __forceinline__ float to_float(T v)
{
    if constexpr (sizeof(T) == 4)
        return __uint2float_rn((uint32_t)v);
    else
        return __ull2float_rn((unsigned long long)v);
}

// even centred moments of one axis from raw moments R[0..4] (ring), then the
// Bernstein map of degree D: out[i] = sum over the axis of C(D,i) d^2i (r^2-d^2)^(D-i)
template <typename T>
__device__ __forceinline__ void axis_bernstein(const T (&R)[5], T c1, T c2, T c3, T c4, int D,
                                               T r2, T r4, T (&out)[3])
{
    // c_m = (-centre)^m in the ring
    const T m0 = R[0];
    const T m2 = R[2] + (T)2 * c1 * R[1] + c2 * R[0];
    if (D == 1) {
        out[0] = r2 * m0 - m2;
        out[1] = m2;
        out[2] = 0;
        return;
    }
    const T m4 = R[4] + (T)4 * c1 * R[3] + (T)6 * c2 * R[2] + (T)4 * c3 * R[1] + c4 * R[0];
    out[0] = r4 * m0 - (T)2 * r2 * m2 + m4;
    out[1] = (T)2 * (r2 * m2 - m4);
    out[2] = m4;
}

template <int KIND, typename T>
__global__ void __launch_bounds__(128) gather_kernel(GatherParams p)
{
    extern __shared__ float s_sq[];  // sqrt(q_t(b)), target-major
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int NT = p.n_targets;
    if (p.target) {
        for (int i = tid; i < NT * p.B; i += blockDim.x * blockDim.y) {
            const int t = i / p.B;
            s_sq[i] = sqrtf(fmaxf(p.target[t * p.target_stride + (i - t * p.B)], 0.f));
        }
        __syncthreads();
    }
    int ix = blockIdx.x * blockDim.x + threadIdx.x;
    int iy = blockIdx.y * blockDim.y + threadIdx.y;
    const bool valid = ix < p.ncx && iy < p.ncy;
    ix = min(ix, p.ncx - 1);
    iy = min(iy, p.ncy - 1);
    const int xc = p.cx0 + ix, yc = p.cy0 + iy;
    const int X0 = xc - p.rx - 1, X1 = xc, X2 = xc + p.rx;
    const int yT = yc - p.ry - 1, yC = yc, yB = yc + p.ry;  // lattice rows (image)
    const T txc = (T)xc, tyc = (T)yc;

    float acc[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) acc[t] = 0.f;
    float *hist = p.hist ? p.hist + ((int64_t)iy * p.ncx + ix) * p.B : nullptr;
    for (int b = 0; b < p.B; ++b) {
        // the stored row holding image row y of bin b's planes (-1: zero)
        auto row = [&](int y) -> int { return (y < 0 || !p.row_map) ? y : __ldg(p.row_map + (int64_t)b * p.H + y); };
        const int Y0 = row(yT), Y1 = row(yC), Y2 = row(yB);
        float h;
        if constexpr (KIND == kGatherPlain) {
            const T U = plane_of<T>(p, p.t1, b).rect(X0, X2, Y0, Y2);
            h = to_float(U) * p.inv_mass;
        } else if constexpr (KIND == kGatherWedding) {
            // nested windows i: plain counts, weighted by c_i = w_i - w_{i+1}
            const Plane<T> P1 = plane_of<T>(p, p.t1, b);
            float u = 0.f;
            for (int i = 0; i < p.n_rings; ++i) {
                const int a = p.ring_rx[i], c = p.ring_ry[i];
                const T n = P1.rect(xc - a - 1, xc + a, row(yc - c - 1), row(yc + c));
                u = fmaf(p.ring_c[i], to_float(n), u);
            }
            h = u * p.inv_mass;
        } else if constexpr (KIND == kGatherManhattan) {
            const Plane<T> P1 = plane_of<T>(p, p.t1, b);
            const Plane<T> Px = plane_of<T>(p, p.tx, b);
            const Plane<T> Py = plane_of<T>(p, p.ty, b);
            const T a00 = P1.at(X0, Y0), a10 = P1.at(X1, Y0), a20 = P1.at(X2, Y0);
            const T a01 = P1.at(X0, Y1), a21 = P1.at(X2, Y1);
            const T a02 = P1.at(X0, Y2), a12 = P1.at(X1, Y2), a22 = P1.at(X2, Y2);
            const T R1 = a22 - a02 - a20 + a00;          // whole window
            const T R1l = a12 - a02 - a10 + a00;         // dx <= 0
            const T R1r = a22 - a12 - a20 + a10;         // dx >= 1
            const T R1t = a21 - a01 - a20 + a00;         // dy <= 0
            const T R1b = a22 - a02 - a21 + a01;         // dy >= 1
            const T Rxl = Px.rect(X0, X1, Y0, Y2);
            const T Rxr = Px.rect(X1, X2, Y0, Y2);
            const T Ryt = Py.rect(X0, X2, Y0, Y1);
            const T Ryb = Py.rect(X0, X2, Y1, Y2);
            // sum |dx| = (sum_r x - xc R1r) - (sum_l x - xc R1l); same for y
            const T sdx = (Rxr - txc * R1r) - (Rxl - txc * R1l);
            const T sdy = (Ryb - tyc * R1b) - (Ryt - tyc * R1t);
            const T U = (T)(p.rx + p.ry) * R1 - sdx - sdy;
            h = to_float(U) * p.inv_mass;
        } else if constexpr (KIND == kGatherEuclidean) {
            const T R1 = plane_of<T>(p, p.t1, b).rect(X0, X2, Y0, Y2);
            const T Rx = plane_of<T>(p, p.tx, b).rect(X0, X2, Y0, Y2);
            const T Ry = plane_of<T>(p, p.ty, b).rect(X0, X2, Y0, Y2);
            const T Rxx = plane_of<T>(p, p.txx, b).rect(X0, X2, Y0, Y2);
            const T Ryy = plane_of<T>(p, p.tyy, b).rect(X0, X2, Y0, Y2);
            // sum dx^2 = Rxx - 2 xc Rx + xc^2 R1 (same for y)
            const T sdx2 = Rxx - (T)2 * txc * Rx + txc * txc * R1;
            const T sdy2 = Ryy - (T)2 * tyc * Ry + tyc * tyc * R1;
            const T U = ((T)p.rx * (T)p.rx + (T)p.ry * (T)p.ry) * R1 - sdx2 - sdy2;
            h = to_float(U) * p.inv_mass;
        } else {
            // Gaussian approximant, T = 64-bit ring
            const T cx1 = (T)0 - txc, cx2 = cx1 * cx1, cx3 = cx2 * cx1, cx4 = cx2 * cx2;
            const T cy1 = (T)0 - tyc, cy2 = cy1 * cy1, cy3 = cy2 * cy1, cy4 = cy2 * cy2;
            const int kx = 2 * p.gdx, ky = 2 * p.gdy;
            T E[3][5];  // x-Bernstein moments per raw y-exponent l
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                if (l > ky) break;
                T R[5] = {0, 0, 0, 0, 0};
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (k > kx) break;
                    R[k] = plane_of<T>(p, p.tg[k][l], b).rect(X0, X2, Y0, Y2);
                }
                T o[3];
                axis_bernstein<T>(R, cx1, cx2, cx3, cx4, p.gdx, (T)p.rx2, (T)p.rx4, o);
                E[0][l] = o[0];
                E[1][l] = o[1];
                E[2][l] = o[2];
            }
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i > p.gdx) break;
                T R[5] = {0, 0, 0, 0, 0};
#pragma unroll
                for (int l = 0; l < 5; ++l)
                    if (l <= ky) R[l] = E[i][l];
                T o[3];
                axis_bernstein<T>(R, cy1, cy2, cy3, cy4, p.gdy, (T)p.ry2, (T)p.ry4, o);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j <= p.gdy) s = fmaf(p.gamma[i][j], to_float(o[j]), s);
            }
            h = s;
        }
        if (hist && valid) hist[b] = h;
        if (p.target) {
            const float sq = sqrtf(h);
#pragma unroll
            for (int t = 0; t < kMaxTargets; ++t)
                if (t < NT) acc[t] = fmaf(sq, s_sq[t * p.B + b], acc[t]);
        }
    }
    if (p.map && valid) {
#pragma unroll
        for (int t = 0; t < kMaxTargets; ++t)
            if (t < NT) p.map[t * p.map_stride + (int64_t)iy * p.ncx + ix] = acc[t];
    }
}

template <typename T>
cudaError_t launch_kind(const GatherParams &p, int kind, cudaStream_t s)
{
    const dim3 block(32, 4);
    const dim3 grid((unsigned)((p.ncx + 31) / 32), (unsigned)((p.ncy + 3) / 4));
    const size_t smem = sizeof(float) * (size_t)p.B * (size_t)p.n_targets;
    switch (kind) {
    case kGatherPlain: gather_kernel<kGatherPlain, T><<<grid, block, smem, s>>>(p); break;
    case kGatherManhattan: gather_kernel<kGatherManhattan, T><<<grid, block, smem, s>>>(p); break;
    case kGatherEuclidean: gather_kernel<kGatherEuclidean, T><<<grid, block, smem, s>>>(p); break;
    case kGatherWedding: gather_kernel<kGatherWedding, T><<<grid, block, smem, s>>>(p); break;
    case kGatherGaussian:
        if constexpr (sizeof(T) == 8) {
            gather_kernel<kGatherGaussian, T><<<grid, block, smem, s>>>(p);
            break;
        } else {
            return cudaErrorInvalidValue;
        }
    default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather(const GatherParams &p, int kind, int elem_bytes, cudaStream_t s)
{
    if (p.ncx <= 0 || p.ncy <= 0) return cudaSuccess;
    if (elem_bytes == 4) return launch_kind<uint32_t>(p, kind, s);
    if (elem_bytes == 8) return launch_kind<unsigned long long>(p, kind, s);
    return cudaErrorInvalidValue;
}

}  // namespace swih
