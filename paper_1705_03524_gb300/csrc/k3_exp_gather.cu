// K3e: window gather of the exponential kernel K = exp(-lambda (|dx| + |dy|)).
//
// With q = exp(-lambda) and the directional integral histograms J_d of K2e, a
// window's quadrants (the centre row and column belong to the top-left one,
// Sec. 2.1's half-open split) are corner differences of their own direction's
// table, the decay across the window supplied by powers of q:
//
//   TL = J0(xc, yc)   - q^(rx+1) J0(xl, yc)   - q^(ry+1) [J0(xc, yu)   - q^(rx+1) J0(xl, yu)]
//   TR = q  [J1(xc+1, yc)   - q^rx J1(xr, yc)   - q^(ry+1) (J1(xc+1, yu)   - q^rx J1(xr, yu))]
//   BL = q  [J2(xc, yc+1)   - q^(rx+1) J2(xl, yc+1) - q^ry (J2(xc, yd)   - q^(rx+1) J2(xl, yd))]
//   BR = q^2 [J3(xc+1, yc+1) - q^rx J3(xr, yc+1) - q^ry (J3(xc+1, yd) - q^rx J3(xr, yd))]
//
// xl = xc-rx-1, xr = xc+rx+1, yu = yc-ry-1, yd = yc+ry+1; reads outside the image
// are 0. U(b) = TL + TR + BL + BR, normalised by the kernel's total weight M.
// Fixed-point values (one = 2^F) are combined as signed 64-bit integers; each
// bracket is a non-negative sum, so rounding noise below zero is clamped.
//
// Bins absent from a window give exactly 0: the window's pixel count of each
// bin, from the exact plain integral histogram (4 reads), gates the 16 reads of
// J. One thread per centre, consecutive centres of a row in consecutive
// threads (coalesced corner reads); the Bhattacharyya sum accumulates over the
// bins in a register.
#include "swih_internal.h"

namespace swih {
namespace {

using u64 = unsigned long long;

__device__ __forceinline__ long long mulq(long long v, u64 qn) { return (long long)__umul64hi((u64)v, qn); }

// max(a - q b, 0) for a, b in [0, 2^62)
__device__ __forceinline__ long long dif(long long a, long long b, u64 qn)
{
    const long long d = a - mulq(b, qn);
    return d > 0 ? d : 0;
}

__device__ __forceinline__ float u64_to_float(u64 v)
{
    return fmaf(__uint2float_rn((uint32_t)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

// compiled for 3 resident CTAs per SM (80 registers; uncapped it took 96 and
// fitted 2): 0.25-0.31 ms against 0.36-0.45 ms per benchmark map
template <typename T>
__global__ void __launch_bounds__(256, 3) exp_gather_kernel(const ExpGatherParams p)
{
    extern __shared__ float s_sq[];  // sqrt(q(b))
    for (int i = threadIdx.x; i < p.B; i += blockDim.x)
        s_sq[i] = p.target ? sqrtf(fmaxf(p.target[i], 0.f)) : 0.f;
    __syncthreads();

    const int64_t n = (int64_t)p.ncx * p.ncy;
    const int64_t dplane = (int64_t)p.B * p.plane;  // between direction groups
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int yc = p.cy0 + (int)(i / p.ncx);
        const int xc = p.cx0 + (int)(i % p.ncx);
        const int xl = xc - p.rx - 1, xr = xc + p.rx + 1, yu = yc - p.ry - 1, yd = yc + p.ry + 1;
        const int x2 = xc + p.rx, y2 = yc + p.ry;
        // row offsets; a corner outside the image reads 0
        const bool in_l = xl >= 0, in_r = xr < p.W, in_u = yu >= 0, in_d = yd < p.H;
        const int64_t oc = (int64_t)yc * p.pitch, ou = (int64_t)yu * p.pitch;
        const int64_t oc1 = (int64_t)(yc + 1) * p.pitch, od = (int64_t)yd * p.pitch;
        float acc = 0.f;
        for (int b = 0; b < p.B; ++b) {
            const T *cnt = reinterpret_cast<const T *>(p.count) + (int64_t)b * p.plane;
            // rows of the count plane without a pixel of the bin are read at the stored row holding them
            int r2 = y2, ru = yu;
            if (p.row_map) {
                r2 = __ldg(p.row_map + (int64_t)b * p.H + y2);
                ru = in_u ? __ldg(p.row_map + (int64_t)b * p.H + yu) : -1;
            }
            const int64_t q2 = (int64_t)r2 * p.pitch, qu = (int64_t)ru * p.pitch;
            const T c22 = r2 >= 0 ? cnt[q2 + x2] : T(0);
            const T c02 = (in_l && r2 >= 0) ? cnt[q2 + xl] : T(0);
            const T c20 = ru >= 0 ? cnt[qu + x2] : T(0);
            const T c00 = (in_l && ru >= 0) ? cnt[qu + xl] : T(0);
            float h = 0.f;
            if ((T)(c22 - c02 - c20 + c00) != T(0)) {
                const u64 *J0 = p.J + (int64_t)b * p.plane;
                const u64 *J1 = J0 + dplane, *J2 = J1 + dplane, *J3 = J2 + dplane;
                auto at = [](const u64 *J, int64_t o, int x, bool ok) -> long long {
                    return ok ? (long long)J[o + x] : 0ll;
                };
                // top-left: x' in [xl+1, xc], y' in [yu+1, yc]
                const long long tl = dif(dif(at(J0, oc, xc, true), at(J0, oc, xl, in_l), p.qx1),
                                         dif(at(J0, ou, xc, in_u), at(J0, ou, xl, in_l && in_u), p.qx1), p.qy1);
                // top-right: x' in [xc+1, xr-1]
                const long long tr = dif(dif(at(J1, oc, xc + 1, true), at(J1, oc, xr, in_r), p.qx0),
                                         dif(at(J1, ou, xc + 1, in_u), at(J1, ou, xr, in_r && in_u), p.qx0), p.qy1);
                // bottom-left: y' in [yc+1, yd-1]
                const long long bl = dif(dif(at(J2, oc1, xc, true), at(J2, oc1, xl, in_l), p.qx1),
                                         dif(at(J2, od, xc, in_d), at(J2, od, xl, in_l && in_d), p.qx1), p.qy0);
                const long long br = dif(dif(at(J3, oc1, xc + 1, true), at(J3, oc1, xr, in_r), p.qx0),
                                         dif(at(J3, od, xc + 1, in_d), at(J3, od, xr, in_r && in_d), p.qx0), p.qy0);
                const long long U = tl + mulq(tr + bl + mulq(br, p.q1), p.q1);
                h = u64_to_float((u64)U) * p.scale;
            }
            if (p.hist) p.hist[i * p.B + b] = h;
            if (h != 0.f) acc = fmaf(sqrtf(h), s_sq[b], acc);
        }
        if (p.map) p.map[i] = acc;
    }
}

}  // namespace

cudaError_t launch_exp_gather(const ExpGatherParams &p, int elem_bytes, cudaStream_t s)
{
    const int64_t n = (int64_t)p.ncx * p.ncy;
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (1 << 20) ? want : (1 << 20));
    const size_t smem = sizeof(float) * (size_t)p.B;
    if (elem_bytes == 4)
        exp_gather_kernel<uint32_t><<<blocks, 256, smem, s>>>(p);
    else
        exp_gather_kernel<unsigned long long><<<blocks, 256, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace swih
