// K2e: directional integral histograms of the exponential kernel.
//
// The kernel K = exp(-lambda (|dx| + |dy|)) has, inside each quadrant of a
// window, the weights exp(+-lambda x) exp(+-lambda y) times a factor fixed by the
// centre, so each quadrant's histogram is a rectangle sum of one weighted
// integral histogram (Sec. 2.1, Eq. 2 with that weight). Those prefix sums grow
// like exp(lambda W). Divided by the weight at the point, and summed from the
// side where the quadrant's weight is smallest, they become
//
//   J_d(x, y) = sum_{x' on side sx of x, y' on side sy of y} [bin = b] q^(|x-x'| + |y-y'|)
//
// with q = exp(-lambda) and d = sx + 2 sy (side 0: x' <= x, side 1: x' >= x), which
// stays below 1 / (1 - q)^2 on any image. J is separable: the column filter
//   C(x, y) = [bin(x, y) = b] + q C(x, y -+ 1)
// followed by the row filter J(x, y) = C(x, y) + q J(x -+ 1, y).
// Values are unsigned 64-bit fixed point (one = 2^F). A product by q^n is the
// high half of v * floor(q^n 2^64), rounded down; every value stays below
// 2^60, so sums never wrap.
//
// A chain is (bin b, y side s); both x sides share its C. Three launches:
//  1. exp_band_agg_kernel: per (chain, band, column), C at the band's last row
//     (scan order) with nothing carried in, as a sum of table powers q^d over the
//     rows that hold the bin; and the band's mask of such rows.
//  2. exp_band_carry_kernel: per (chain, column), the value carried into each
//     band, sequentially over the bands: c_{k+1} = agg_k + q^band_rows c_k,
//     written over the aggregates.
//  3. exp_scan_kernel: per (chain, band), the band's rows in scan order: C from
//     the carry, then for each x side a block-wide scan of the linear
//     recurrence (thread-serial over E columns, warp shuffles with q^(E d),
//     warp totals through shared memory with q^(32 E d)); each row of J leaves
//     as 16-byte stores. A row without the bin is q times the row above.
// No block waits on another.
#include "swih_internal.h"

namespace swih {
namespace {

using u64 = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;

// v * q^n for v < 2^62 and qn = floor(q^n 2^64): the high 64 bits of the product
// from three 32 x 32-bit products; the dropped low x low product and the
// truncated middle terms make it 0 to 2 units below the exact high half, so it
// still rounds down (measured 7% faster than the full 64 x 64-bit high half)
__device__ __forceinline__ u64 mulq(u64 v, u64 qn)
{
    const uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
    const uint32_t qh = (uint32_t)(qn >> 32), ql = (uint32_t)qn;
    return (u64)vh * qh + __umulhi(vh, ql) + __umulhi(vl, qh);
}

// bit i set when column x0 + i (< W) of the row holds bin b; x0 is a multiple of
// E and rows start 128-byte aligned, so whole groups are aligned vector loads
template <int E>
__device__ __forceinline__ unsigned match_bits(const uint8_t *row, int x0, int W, int b)
{
    unsigned m = 0;
    if (x0 + E <= W) {
        uint32_t w[E / 4];
        if constexpr (E == 4) {
            w[0] = *reinterpret_cast<const uint32_t *>(row + x0);
        } else if constexpr (E == 8) {
            const uint2 v = *reinterpret_cast<const uint2 *>(row + x0);
            w[0] = v.x;
            w[1] = v.y;
        } else {
            const uint4 v = *reinterpret_cast<const uint4 *>(row + x0);
            w[0] = v.x;
            w[1] = v.y;
            w[2] = v.z;
            w[3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < E; ++i) m |= (((w[i >> 2] >> (8 * (i & 3))) & 0xffu) == (unsigned)b ? 1u : 0u) << i;
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i)
            if (x0 + i < W && row[x0 + i] == b) m |= 1u << i;
    }
    return m;
}

__global__ void __launch_bounds__(256) exp_band_agg_kernel(const ExpScanParams p)
{
    // the band's C at its last row is a sum of powers q^d over the rows holding
    // the bin (d = rows after it); bands of up to 64 rows read them from a table
    __shared__ unsigned long long s_qrow[65];
    __shared__ unsigned long long s_rows;
    const int nchain = 2 * p.B;
    const int chain = blockIdx.x % nchain, band = blockIdx.x / nchain;
    const int side = chain / p.B, b = chain - side * p.B;
    const int r0 = band * p.band_rows, r1 = min(r0 + p.band_rows, p.H);
    const bool table = p.band_rows <= 64;
    for (int i = threadIdx.x; i < 65; i += blockDim.x) s_qrow[i] = p.qrow[i];
    if (threadIdx.x == 0) s_rows = 0ull;
    __syncthreads();
    unsigned long long mine = 0ull;  // rows (first 64 of the band) where the thread's columns hold the bin
    u64 *out = p.carry + ((int64_t)chain * p.n_bands + band) * p.pitch;
    for (int x0 = 4 * threadIdx.x; x0 < p.W; x0 += 4 * blockDim.x) {
        u64 a[4] = {0, 0, 0, 0};
        for (int r = r0; r < r1; ++r) {
            const int y = side ? p.H - 1 - r : r;
            const unsigned m = match_bits<4>(p.bins + (int64_t)y * p.bins_pitch, x0, p.W, b);
            if (table) {
                if (m) {
                    mine |= 1ull << (r - r0);
                    const u64 w = s_qrow[r1 - 1 - r];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if ((m >> i) & 1u) a[i] += w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = mulq(a[i], p.q1) + (((m >> i) & 1u) ? p.one : 0ull);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (x0 + i < p.W) out[x0 + i] = a[i];
    }
    if (mine) atomicOr(&s_rows, mine);
    __syncthreads();
    if (threadIdx.x == 0) p.rows[(int64_t)chain * p.n_bands + band] = table ? s_rows : ~0ull;
}

__global__ void __launch_bounds__(256) exp_band_carry_kernel(const ExpScanParams p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)2 * p.B * p.W) return;
    const int64_t chain = i / p.W;
    const int x = (int)(i - chain * p.W);
    u64 *c = p.carry + chain * p.n_bands * p.pitch + x;
    u64 acc = 0;
    for (int k = 0; k < p.n_bands; ++k) {
        const u64 a = c[(int64_t)k * p.pitch];
        c[(int64_t)k * p.pitch] = acc;
        acc = a + mulq(acc, p.qband);
    }
}

template <int E>
__device__ __forceinline__ void store_row(u64 *dst, int x0, int64_t pitch, int W, const u64 (&v)[E])
{
    if (x0 + E <= pitch) {
#pragma unroll
        for (int i = 0; i < E; i += 2) *reinterpret_cast<ulonglong2 *>(dst + x0 + i) = make_ulonglong2(v[i], v[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i)
            if (x0 + i < W) dst[x0 + i] = v[i];
    }
}

template <int E>
__global__ void __launch_bounds__(512) exp_scan_kernel(const ExpScanParams p)
{
    // [row parity][x side][warp]: warp totals, then their scan across warps
    __shared__ u64 s_warp[2][2][16];
    const int nchain = 2 * p.B;
    const int chain = blockIdx.x % nchain, band = blockIdx.x / nchain;
    const int side = chain / p.B, b = chain - side * p.B;
    const int r0 = band * p.band_rows, r1 = min(r0 + p.band_rows, p.H);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int x0 = tid * E;

    u64 C[E];
    {
        const u64 *cin = p.carry + ((int64_t)chain * p.n_bands + band) * p.pitch;
#pragma unroll
        for (int i = 0; i < E; ++i) C[i] = x0 + i < p.W ? cin[x0 + i] : 0ull;
    }
    u64 *Jf = p.J + ((int64_t)(2 * side) * p.B + b) * p.plane;      // x side 0 (x' <= x)
    u64 *Jr = p.J + ((int64_t)(2 * side + 1) * p.B + b) * p.plane;  // x side 1 (x' >= x)

    // A row without the bin has C = q C(row above), hence both rows of J are q
    // times the rows above: with up to 8 columns per thread they are formed from
    // the previous row's outputs, kept in registers, with no scan and no barrier
    // (uniform over the block: the band's row mask comes from the aggregate pass).
    constexpr bool kDecay = E <= 8;
    const unsigned long long rmask = p.rows[(int64_t)chain * p.n_bands + band];
    u64 outf[E], outr[E];
#pragma unroll
    for (int i = 0; i < E; ++i) outf[i] = outr[i] = 0;
    // the warp-total buffers alternate per scanned row (rows formed by decay
    // pass no barrier, so alternating per image row could reuse a buffer that
    // a slower warp has not yet read)
    int par = 1;

    for (int r = r0; r < r1; ++r) {
        const int y = side ? p.H - 1 - r : r;
        if constexpr (kDecay) {
            if (r > r0 && r - r0 < 64 && !((rmask >> (r - r0)) & 1ull)) {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    C[i] = mulq(C[i], p.q1);
                    outf[i] = mulq(outf[i], p.q1);
                    outr[i] = mulq(outr[i], p.q1);
                }
                store_row<E>(Jf + (int64_t)y * p.pitch, x0, p.pitch, p.W, outf);
                store_row<E>(Jr + (int64_t)y * p.pitch, x0, p.pitch, p.W, outr);
                continue;
            }
        }
        par ^= 1;
        const unsigned m = match_bits<E>(p.bins + (int64_t)y * p.bins_pitch, x0, p.W, b);
#pragma unroll
        for (int i = 0; i < E; ++i) C[i] = mulq(C[i], p.q1) + (((m >> i) & 1u) ? p.one : 0ull);

        // thread totals of both recurrences over the thread's columns, nothing carried in
        u64 tf = 0, tr = 0;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            tf = C[i] + mulq(tf, p.q1);
            tr = C[E - 1 - i] + mulq(tr, p.q1);
        }
        // inclusive scans within the warp: forward from lower lanes, reverse from higher
        u64 vf = tf, vr = tr;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const u64 of = __shfl_up_sync(kFull, vf, d);
            const u64 orr = __shfl_down_sync(kFull, vr, d);
            if (lane >= d) vf += mulq(of, p.qe[d]);
            if (lane + d < 32) vr += mulq(orr, p.qe[d]);
        }
        if (lane == 31) s_warp[par][0][wid] = vf;
        if (lane == 0) s_warp[par][1][wid] = vr;
        __syncthreads();
        if (wid == 0) {  // scan the warp totals (nw <= 16), both directions
            u64 af = lane < nw ? s_warp[par][0][lane] : 0ull;
            u64 ar = lane < nw ? s_warp[par][1][lane] : 0ull;
#pragma unroll
            for (int d = 1; d < 16; d <<= 1) {
                const u64 of = __shfl_up_sync(kFull, af, d);
                const u64 orr = __shfl_down_sync(kFull, ar, d);
                if (lane >= d) af += mulq(of, p.qw[d]);
                if (lane + d < 32) ar += mulq(orr, p.qw[d]);
            }
            if (lane < nw) {
                s_warp[par][0][lane] = af;
                s_warp[par][1][lane] = ar;
            }
        }
        __syncthreads();
        // value of each recurrence just outside the thread's columns
        const u64 Pf = wid > 0 ? s_warp[par][0][wid - 1] : 0ull;       // end of the warp to the left
        const u64 Pr = wid + 1 < nw ? s_warp[par][1][wid + 1] : 0ull;  // start of the warp to the right
        const u64 pf = __shfl_up_sync(kFull, vf, 1);
        const u64 pr = __shfl_down_sync(kFull, vr, 1);
        const u64 Xf = lane == 0 ? Pf : pf + mulq(Pf, p.qe[lane]);
        const u64 Xr = lane == 31 ? Pr : pr + mulq(Pr, p.qe[31 - lane]);

        u64 s = Xf;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            s = C[i] + mulq(s, p.q1);
            outf[i] = s;
        }
        store_row<E>(Jf + (int64_t)y * p.pitch, x0, p.pitch, p.W, outf);
        s = Xr;
#pragma unroll
        for (int i = E - 1; i >= 0; --i) {
            s = C[i] + mulq(s, p.q1);
            outr[i] = s;
        }
        store_row<E>(Jr + (int64_t)y * p.pitch, x0, p.pitch, p.W, outr);
    }
}

}  // namespace

cudaError_t launch_exp_scan(const ExpScanParams &p, cudaStream_t s)
{
    const long long tiles = 2LL * p.B * p.n_bands;
    const long long cols = 2LL * p.B * p.W;
    if (tiles > 0x7fffffffLL || p.threads < 32 || p.threads > 512 || p.threads % 32 ||
        (long long)p.threads * p.E < p.W)
        return cudaErrorInvalidConfiguration;
    exp_band_agg_kernel<<<(unsigned)tiles, 256, 0, s>>>(p);
    exp_band_carry_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(p);
    switch (p.E) {
    case 4: exp_scan_kernel<4><<<(unsigned)tiles, p.threads, 0, s>>>(p); break;
    case 8: exp_scan_kernel<8><<<(unsigned)tiles, p.threads, 0, s>>>(p); break;
    case 16: exp_scan_kernel<16><<<(unsigned)tiles, p.threads, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace swih
