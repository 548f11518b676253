// K3 (tiled): the window gather of Sec. 2.1 with lattice-row reuse.
//
// Computes exactly what k3_gather.cu computes (same ring arithmetic, same
// translation, same normalisation and Bhattacharyya sum), organised so that each
// integral-histogram element is fetched about once per launch instead of four
// to nine times:
//
// * A CTA owns TX consecutive centre columns (one thread per column) and a
//   chain of up to KMAX centre rows spaced exactly one window height h apart.
//   Window k's bottom corner row is window k+1's top corner row, so the chain
//   walks K+1 lattice rows for K windows (Manhattan adds each window's centre
//   row, which splits it into top and bottom halves: 2K+1 rows).
// * Work is a sequence of pipeline steps (bin block, lattice row, plane group).
//   A step carries BB bins (several for the cheap kernels, one for the
//   Gaussian) and, for the Gaussian, one y-exponent l, i.e. the planes
//   x^0..x^2Dx y^l. A dedicated producer warp issues, for each step, TMA bulk
//   copies (cp.async.bulk, completion counted on a "full" mbarrier) of the row
//   segments [xs-rx-1, xs+TX+rx) into one stage of a ring of NS shared-memory
//   stages, up to NS steps ahead of the consumers; its lanes share the step's
//   copies, and lane 0 posts their byte count on the barrier first. Each consumer
//   warp releases a stage through an "empty" mbarrier, and the producer refills
//   a stage only after every consumer warp has released it.
// * Every thread forms its horizontal differences I(X2) - I(X0) (and the
//   centre split for Manhattan) from shared memory; the vertical difference is
//   taken against the previous lattice row's values held in registers.
//   For the Gaussian the carried values are already translated to the centre
//   column and mapped to the Bernstein basis along x (a linear map, so it
//   commutes with the vertical difference).
// * The likelihood of each of the K windows accumulates over bins in shared
//   memory (one slot per window and column) and is written once at the end.
// CTAs are ordered with the column tiles fastest and the chains of one phase
// adjacent, so the halo columns of neighbouring tiles and the boundary row of
// neighbouring chains are shared through L2 while both are resident.
// Every mbarrier wait is bounded; a wait that gives up sets the status word and
// stops the waiting warp. Copies already issued always land in shared memory
// that stays allocated until the consumer warps, which wait for them, exit.
//
// This header holds the device code; k3_tiled_<kind>.cu instantiate it, one
// kernel kind per translation unit, and k3_gather_tiled.cu holds the host side.
#pragma once

#include "k3_tiled.h"

namespace swih {
namespace {


constexpr int KMAX = kTiledChainMax;
constexpr int kRowSlots = kTiledRowSlots;  // lattice rows per chain: K + 1, or 2 K + 1 with K <= KMAX / 2 (Manhattan)
static_assert(2 * (KMAX / 2) + 1 <= kRowSlots, "row slots");
constexpr int kMaxStages = kTiledMaxStages;

template <typename T>
struct template_tag {
    using type = T;
};
template <int V>
struct int_tag {
    static constexpr int value = V;
};
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr uint32_t kSuspendHintNs = 200000;                   // sleep up to 0.2 ms per try

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// test the phase; the thread may sleep (up to the hint) until it completes
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (about 2 s of wall time); false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// a * b for a 64-bit ring element and a 32-bit factor (two IMADs)
__device__ __forceinline__ unsigned long long mul_u32(unsigned long long a, uint32_t b)
{
    const unsigned long long lo = (unsigned long long)(uint32_t)a * b;
    const uint32_t hi = (uint32_t)(a >> 32) * b;
    return lo + ((unsigned long long)hi << 32);
}

// non-negative 64-bit integer to float via two 32-bit conversions
__device__ __forceinline__ float u64_to_float(unsigned long long v)
{
    return fmaf(__uint2float_rn((uint32_t)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

template <typename T>
__device__ __forceinline__ float ring_to_float(T v)
{
    if constexpr (sizeof(T) == 4)
        return __uint2float_rn((uint32_t)v);
    else
        return u64_to_float((unsigned long long)v);
}

// Even centred moments of one axis from raw moments R[0..2D] (Horner in the
// centre c: sum_k C(m,k) (-c)^(m-k) R_k), then the Bernstein map of degree D:
//   out_i = sum over the axis of C(D,i) d^2i (r^2 - d^2)^(D-i).
// c (a centre coordinate) and r2 = r^2 fit 32 bits; r4 = r^4 may not (r > 255).
template <int D>
__device__ __forceinline__ void axis_bernstein(const unsigned long long (&R)[5], uint32_t c, uint32_t r2,
                                               unsigned long long r4, unsigned long long (&out)[3])
{
    using u64 = unsigned long long;
    // m2 = R2 - 2c R1 + c^2 R0
    u64 t = R[0];
    t = 2 * R[1] - mul_u32(t, c);
    const u64 m2 = R[2] - mul_u32(t, c);
    if constexpr (D == 1) {
        out[0] = mul_u32(R[0], r2) - m2;
        out[1] = m2;
        out[2] = 0;
    } else {
        // m4 = R4 - 4c R3 + 6c^2 R2 - 4c^3 R1 + c^4 R0
        u64 v = R[0];
        v = 4 * R[1] - mul_u32(v, c);
        v = 6 * R[2] - mul_u32(v, c);
        v = 4 * R[3] - mul_u32(v, c);
        const u64 m4 = R[4] - mul_u32(v, c);
        const u64 r2m2 = mul_u32(m2, r2);
        out[0] = R[0] * r4 - 2 * r2m2 + m4;
        out[1] = 2 * (r2m2 - m4);
        out[2] = m4;
    }
}

// One work item: column tile `tile` and chain `cy` (phase-major) of job p.
template <int KIND, typename T, int TX, int DX, int DY, int BB, bool SPLIT, bool ROWMAP>
__device__ __forceinline__ void gather_tiled_body(const GatherParams &p, const int tile, const int cy, const int bg)
{
    using u64 = unsigned long long;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);
    uint64_t *empty = full + kMaxStages;
    float *s_sq = reinterpret_cast<float *>(sm + 16 * kMaxStages);
    float *s_acc = s_sq + p.n_targets * p.B;
    T *stages = reinterpret_cast<T *>(sm + p.stage_off);

    constexpr int NWARP = TX / 32;
    constexpr bool kMan = KIND == kGatherManhattan;
    constexpr bool kGau = KIND == kGatherGaussian;
    constexpr int KX = 2 * DX, KY = 2 * DY;  // Gaussian raw-moment orders
    constexpr int G = kGau ? KY + 1 : 1;     // plane groups per lattice row
    static_assert(!kGau || BB == 1, "the Gaussian carries one bin per step");

    const int tid = threadIdx.x;  // threads [0, TX): consumers; warp TX/32: producer
    const int lane = tid & 31;
    const bool producer = tid >= TX;
    const int h = 2 * p.ry + 1;
    const int blk = cy % p.nblk;
    const int phase = cy / p.nblk;
    const int n_slots = (p.ncy - phase + h - 1) / h;
    const int slot0 = blk * p.kchain;
    const int K = min(p.kchain, n_slots - slot0);
    // bin blocks [bb0, bb1): all of them, or bin group bg's share of a split launch
    const int NBB = (p.B + BB - 1) / BB;
    int bb0 = 0, bb1 = NBB;
    if constexpr (SPLIT) {
        const int per_group = (NBB + p.nbg - 1) / p.nbg;
        bb0 = bg * per_group;
        bb1 = min(NBB, bb0 + per_group);
    }
    if (K <= 0 || bb0 >= bb1) return;  // whole CTA, before any barrier

    const int xs = p.cx0 + tile * TX;
    int xc = xs + (producer ? 0 : tid);
    const bool valid_x = xc < p.cx0 + p.ncx;
    xc = min(xc, p.cx0 + p.ncx - 1);
    const int yc0 = p.cy0 + phase + slot0 * h;
    const int S = kMan ? 2 * K + 1 : K + 1;  // lattice rows
    // bin blocks this CTA walks: [bb0, bb1), less those without a pixel in the
    // union of its windows (see below); the list sits just below the carry area
    int *s_list = reinterpret_cast<int *>(sm + p.dtop_off) - 2 * (p.B + 1);
    int *s_rows = s_list + (p.B + 1);  // per listed bin block: the lattice rows to load (bit s)
    // per bin and lattice row: the stored row that holds it (-1: the zero row),
    // through the row map when empty rows are not stored. Images taller than
    // 32767 rows never reach the tiled gather (the host sends them to the direct
    // one), so int16 holds every row.
    int16_t *s_rmap = reinterpret_cast<int16_t *>(s_list) - p.B * kRowSlots;
    const int NS = p.nstage;

    // row segment [xs-rx-1, xs+TX+rx) of every plane, copied from a 16-byte boundary
    constexpr int A = 16 / (int)sizeof(T);
    const int xlo = xs - p.rx - 1;  // >= -1
    const int xo = xlo >= 0 ? (xlo / A) * A : -A;
    const int x_begin = xo > 0 ? xo : 0;
    const int x_end = min(xs + TX + p.rx, p.W);
    const uint32_t seg_bytes = (uint32_t)(((x_end - x_begin) * (int)sizeof(T) + 15) & ~15);
    const int land = x_begin - xo;
    const int stage_elems = p.nl * p.seg;  // nl = slots per stage (BB * planes per step)

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NWARP);  // consumer warps
        }
        mbar_init_fence();
    }
    // sqrt(q_t(b)) of every target; one accumulator per (target, window, column)
    const int NT = p.n_targets;
    const int KC = p.kchain;
    for (int i = tid; i < NT * p.B; i += TX + 32) {
        const int t = i / p.B;
        s_sq[i] = p.target ? sqrtf(fmaxf(p.target[t * p.target_stride + (i - t * p.B)], 0.f)) : 0.f;
    }
    if (!producer)
        for (int k = 0; k < NT * KC; ++k) s_acc[k * TX + tid] = 0.f;
    if (xlo < 0) {  // column -1 of the integral histogram is 0; copies never land there
        for (int i = tid; i < NS * p.nl; i += TX + 32) stages[(size_t)i * p.seg + (A - 1)] = T(0);
    }
    // A window with no pixel of bin b has every moment of b zero, so the
    // integral histograms' differences at its bottom lattice row equal those at
    // its top: the row after such a window need not be copied, and a bin absent
    // from all the CTA's windows needs no row at all. Per bin, the pixel count
    // of window k over the tile's columns is c(bottom_k) - c(top_k), with
    // c(y) = I(y, xb) - I(y, xa) on the count plane (x^0 y^0), exact in the
    // ring: 2 reads per lattice row. The rows to load are those of the present
    // windows (Manhattan: top, centre and bottom rows). Histogram output needs
    // every bin and row, so then all are loaded.
    auto row_of = [&](int s) -> int {
        if constexpr (kMan) {
            const int k = s >> 1;
            return (s & 1) ? yc0 + k * h : yc0 + k * h - p.ry - 1;
        } else {
            return yc0 + s * h - p.ry - 1;
        }
    };
    const bool sparse = p.hist == nullptr;
    const int all_rows = (int)((1u << S) - 1u);
    // the CTA's bins: all of them, or bin group bg's share of a split launch
    const int bin0 = bb0 * BB, bin1 = min(p.B, bb1 * BB);
    if constexpr (ROWMAP) {  // all threads: the row map reads overlap
        for (int i = tid; i < (bin1 - bin0) * S; i += TX + 32) {
            const int b = bin0 + i / S, s = i % S;
            const int Y = row_of(s);
            s_rmap[b * kRowSlots + s] = (int16_t)((Y < 0 || !p.row_map) ? Y : __ldg(p.row_map + (int64_t)b * p.H + Y));
        }
        __syncthreads();
    }
    // image row s of bin b's planes is stored at this row (-1: zero); without a
    // row map every row is stored
    auto stored_row = [&](int b, int s) -> int {
        if constexpr (ROWMAP)
            return s_rmap[b * kRowSlots + s];
        else
            return row_of(s);
    };
    {
        const int xa = xs - p.rx - 1;                           // exclusive
        const int xb = min(xs + TX, p.cx0 + p.ncx) - 1 + p.rx;  // inclusive
        for (int b = bin0 + tid; b < bin1; b += TX + 32) {
            if (!sparse) continue;
            const T *pl = reinterpret_cast<const T *>(p.ih) + ((int64_t)p.t1 * p.B + b) * p.plane;
            auto at = [&](int x, int y) -> T { return (x >= 0 && y >= 0) ? __ldg(pl + (int64_t)y * p.pitch + x) : T(0); };
            auto span = [&](int s) -> T { return at(xb, stored_row(b, s)) - at(xa, stored_row(b, s)); };  // lattice row s
            unsigned rows_b = 0u;
            T prev = span(0);
            for (int k = 0; k < K; ++k) {
                const T next = span(kMan ? 2 * k + 2 : k + 1);  // window k's bottom row
                if (next != prev) rows_b |= kMan ? (7u << (2 * k)) : (3u << k);
                prev = next;
            }
            s_list[b] = (int)rows_b;
        }
    }
    __syncthreads();
    if (tid == 0) {  // compact in place: per-bin masks are read ahead of where block entries are written
        int n = 0, total = 0;
        for (int bb = bb0; bb < bb1; ++bb) {
            unsigned m = sparse ? 0u : (unsigned)all_rows;
            for (int j = 0; j < BB && sparse; ++j)
                if (bb * BB + j < p.B) m |= (unsigned)s_list[bb * BB + j];
            if (m) {
                s_list[n] = bb;
                s_rows[n] = (int)m;
                ++n;
                total += __popc(m);
            }
        }
        s_list[p.B] = n;
        s_rows[p.B] = total;
    }
    __syncthreads();
    const int nlist = s_list[p.B];
    const int steps = s_rows[p.B] * G;

    // producer warp: steps in order, each into stage m % NS once the consumers
    // have released that stage's previous step. The step's copies (bin j, plane
    // t) are spread over the lanes; lane 0 posts the step's byte count on the
    // full barrier before any lane issues its copies.
    if (producer) {
        int g = 0, s = 0, li = 0;
        int bb = nlist > 0 ? s_list[0] : 0;
        unsigned rmask = nlist > 0 ? (unsigned)s_rows[0] : 0u;
        while (s < S && !((rmask >> s) & 1u)) ++s;  // the first row to load
        unsigned long long loaded = 0;  // bytes of integral histogram requested (lane 0)
        for (int m = 0; m < steps; ++m) {
            const int st_i = m % NS;
            if (m >= NS) {
                const bool ok = mbar_wait(&empty[st_i], (uint32_t)(((m / NS) - 1) & 1));
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(p.status, kStatusTimeout);
                    return;
                }
            }
            uint64_t *br = &full[st_i];
            const int b0 = bb * BB;
            const int nb = min(BB, p.B - b0);
            int nt;
            const int *list;
            if constexpr (kGau) {
                nt = KX + 1;
                list = p.load_even + g * (KX + 1);
            } else {
                const bool odd = kMan && (s & 1);
                nt = odd ? p.n_load_odd : p.n_load_even;
                list = odd ? p.load_odd : p.load_even;
            }
            // copies of bins whose row is stored (the others read as zero)
            const int n_copies = nb * nt;
            int n_valid = 0;
            for (int c0 = 0; c0 < n_copies; c0 += 32) {
                const int c = c0 + lane;
                const bool v = c < n_copies && stored_row(b0 + c / nt, s) >= 0;
                n_valid += __popc(__ballot_sync(0xffffffffu, v));
            }
            if (lane == 0) {
                if (n_valid == 0) {  // zero rows only (above the image, or before the bin's first pixel)
                    mbar_arrive(br);
                } else {
                    mbar_arrive_expect_tx(br, (uint32_t)n_valid * seg_bytes);
                    loaded += (unsigned long long)n_valid * seg_bytes;
                }
            }
            __syncwarp();
            if (n_valid > 0) {
                T *dst = stages + (size_t)st_i * stage_elems + land;
                for (int c = lane; c < n_copies; c += 32) {
                    const int j = c / nt, t = c - j * nt;
                    const int Y = stored_row(b0 + j, s);
                    if (Y < 0) continue;
                    const T *src = reinterpret_cast<const T *>(p.ih) + (int64_t)Y * p.pitch + x_begin +
                                   ((int64_t)list[t] * p.B + b0 + j) * p.plane;
                    fence_proxy_async_smem();
                    bulk_copy_g2s(dst + (size_t)c * p.seg, src, seg_bytes, br);
                }
            }
            if (++g == G) {
                g = 0;
                do {
                    ++s;
                } while (s < S && !((rmask >> s) & 1u));
                if (s == S && ++li < nlist) {
                    bb = s_list[li];
                    rmask = (unsigned)s_rows[li];
                    s = 0;
                    while (s < S && !((rmask >> s) & 1u)) ++s;
                }
            }
        }
        if (lane == 0 && p.load_bytes) atomicAdd(p.load_bytes, loaded);
        return;
    }

    const int i0 = xc - p.rx - 1 - xo;  // smem index of X0 (column -1 reads the zeroed word)
    const int i1 = xc - xo;
    const int i2 = xc + p.rx - xo;
    const T txc = (T)xc;

    // carried values of the previous lattice row, per bin of the block
    T top[BB][4];
    T mid1[BB], midy[BB];
#pragma unroll
    for (int j = 0; j < BB; ++j) {
        mid1[j] = midy[j] = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) top[j][i] = 0;
    }
    // Gaussian: raw row differences of the previous lattice row (shared memory,
    // one column per thread), and the current window's x-translated Bernstein
    // moments per y-exponent (registers)
    u64 *dtop = reinterpret_cast<u64 *>(sm + p.dtop_off) + tid;
    if constexpr (kGau) {
#pragma unroll
        for (int i = 0; i < (KX + 1) * (KY + 1); ++i) dtop[i * TX] = 0;
    }
    u64 E[3][5];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 5; ++l) E[i][l] = 0;
    bool occupied = false;  // Gaussian: the bin has pixels in the current window

    bool stop = false;
    int n = 0;          // step index
    int cs = 0;         // consumer stage
    uint32_t cpar = 0;  // its parity
    for (int li = 0; li < nlist && !stop; ++li) {
        const int bb = s_list[li];
        const unsigned rmask = (unsigned)s_rows[li];
        bool first = true;  // the first row loaded for this bin completes no window
        const int b0 = bb * BB;
        const int nb = min(BB, p.B - b0);
        for (int s = 0; s < S && !stop; ++s) {
            if (!((rmask >> s) & 1u)) continue;  // after an absent window: same values as the carried ones
            // bin b0's row s reads as zero (above the image, or before the bin's
            // first pixel); the Gaussian carries one bin, the others test each bin
            const bool zero_row = stored_row(b0, s) < 0;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (!mbar_wait(&full[cs], cpar)) stop = true;
                if (stop) break;
                const T *st = stages + (size_t)cs * stage_elems;

                if constexpr (kGau) {
                    // planes x^0..x^KX of y^g: window sums R = this row's horizontal
                    // differences minus the previous lattice row's
                    u64 R[5] = {0, 0, 0, 0, 0};
#pragma unroll
                    for (int k = 0; k <= KX; ++k) {
                        const u64 d = zero_row ? 0ull : (u64)st[k * p.seg + i2] - (u64)st[k * p.seg + i0];
                        R[k] = d - dtop[(g * (KX + 1) + k) * TX];
                        dtop[(g * (KX + 1) + k) * TX] = d;
                    }
                    // a bin with no pixel in the window has every moment zero: its
                    // translation is skipped (the pixel count is the x^0 y^0 plane)
                    if (g == 0) occupied = !first && R[0] != 0;
                    if (occupied) {
                        u64 ex[3] = {0, 0, 0};
                        axis_bernstein<DX>(R, (uint32_t)xc, (uint32_t)p.rx2, p.rx4, ex);
#pragma unroll
                        for (int i = 0; i <= DX; ++i) E[i][g] = ex[i];
                    }
                } else {
                    // the window completed by this lattice row (if any); its
                    // likelihood terms for the step's bins are summed in a register
                    const int done_k = first ? -1 : (kMan ? ((s & 1) ? -1 : (s >> 1) - 1) : s - 1);
                    float step_acc = 0.f;
#pragma unroll
                    for (int j = 0; j < BB; ++j) {
                        if (j >= nb) break;
                        const int b = b0 + j;
                        const bool zr = stored_row(b, s) < 0;
                        // h stays 0 for a bin with no pixel in the window: the
                        // combination, conversion and square root are skipped
                        float hval = 0.f;
                        if constexpr (KIND == kGatherPlain) {
                            const T *q = st + (size_t)j * p.seg;
                            const T d = zr ? T(0) : (T)(q[i2] - q[i0]);
                            if (done_k >= 0) {
                                const T U = d - top[j][0];
                                if (U != 0) hval = ring_to_float<T>(U) * p.inv_mass;
                            }
                            top[j][0] = d;
                        } else if constexpr (kMan) {
                            if (s & 1) {  // centre row: full-width sums of IH_1 and IH_y
                                const T *q = st + (size_t)(j * 2) * p.seg;
                                mid1[j] = zr ? T(0) : (T)(q[i2] - q[i0]);
                                midy[j] = zr ? T(0) : (T)(q[p.seg + i2] - q[p.seg + i0]);
                            } else {
                                // per lattice row, of the left (dx <= 0) and right (dx > 0)
                                // halves of the window's columns: the count of both (d1),
                                // right minus left of the count (dd1) and of IH_x (ddx), and
                                // the full-width IH_y difference (dyf)
                                T d1 = 0, dd1 = 0, ddx = 0, dyf = 0;
                                if (!zr) {
                                    const T *q = st + (size_t)(j * 3) * p.seg;
                                    const T a0 = q[i0], a1 = q[i1], a2 = q[i2];
                                    const T *sx = q + p.seg;
                                    const T *sy = q + 2 * p.seg;
                                    d1 = a2 - a0;
                                    dd1 = (a2 + a0) - (a1 + a1);
                                    ddx = (sx[i2] + sx[i0]) - (sx[i1] + sx[i1]);
                                    dyf = sy[i2] - sy[i0];
                                }
                                if (done_k >= 0) {
                                    const T R1 = d1 - top[j][0];  // pixel count of the bin in the window
                                    if (R1 != 0) {
                                        const T tyc = (T)(yc0 + done_k * h);
                                        const T R1t = mid1[j] - top[j][0];
                                        const T R1b = d1 - mid1[j];
                                        const T Ryt = midy[j] - top[j][3], Ryb = dyf - midy[j];
                                        // sum over the window of |dx|: right half minus left half of
                                        // (x - xc); likewise |dy| with the centre row
                                        const T sdx = (ddx - top[j][2]) - txc * (dd1 - top[j][1]);
                                        const T sdy = (Ryb - tyc * R1b) - (Ryt - tyc * R1t);
                                        const T U = (T)(p.rx + p.ry) * R1 - sdx - sdy;
                                        hval = ring_to_float<T>(U) * p.inv_mass;
                                    }
                                }
                                top[j][0] = d1;
                                top[j][1] = dd1;
                                top[j][2] = ddx;
                                top[j][3] = dyf;
                            }
                        } else {  // Euclidean
                            // full-width differences of the planes 1, y, y^2 and of
                            // x^2 - 2 xc x + xc^2 (centred on this thread's column, a
                            // linear map, so it commutes with the vertical difference)
                            T d[4] = {0, 0, 0, 0};
                            if (!zr) {
                                const T *q = st + (size_t)(j * 5) * p.seg;
                                auto dif = [&](int t) -> T { return q[t * p.seg + i2] - q[t * p.seg + i0]; };
                                d[0] = dif(0);
                                d[1] = dif(3) - (T)2 * txc * dif(1) + txc * txc * d[0];
                                d[2] = dif(2);
                                d[3] = dif(4);
                            }
                            if (done_k >= 0) {
                                const T R1 = d[0] - top[j][0];
                                if (R1 != 0) {
                                    const T tyc = (T)(yc0 + done_k * h);
                                    const T sdx2 = d[1] - top[j][1];
                                    const T Ry = d[2] - top[j][2], Ryy = d[3] - top[j][3];
                                    const T sdy2 = Ryy - (T)2 * tyc * Ry + tyc * tyc * R1;
                                    const T U = ((T)p.rx * (T)p.rx + (T)p.ry * (T)p.ry) * R1 - sdx2 - sdy2;
                                    hval = ring_to_float<T>(U) * p.inv_mass;
                                }
                            }
#pragma unroll
                            for (int t = 0; t < 4; ++t) top[j][t] = d[t];
                        }
                        if (done_k >= 0) {
                            if (p.hist && valid_x) {
                                const int yc = yc0 + done_k * h;
                                p.hist[((int64_t)(yc - p.cy0) * p.ncx + (xc - p.cx0)) * p.B + b] = hval;
                            }
                            if (hval != 0.f) {
                                const float sq = sqrtf(hval);
                                step_acc += sq * s_sq[b];
                                for (int t = 1; t < NT; ++t)
                                    s_acc[(t * KC + done_k) * TX + tid] += sq * s_sq[t * p.B + b];
                            }
                        }
                    }
                    if (done_k >= 0 && p.target) s_acc[done_k * TX + tid] += step_acc;
                }
                // release the stage: every lane of the warp is done reading it
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[cs]);
                if (++cs == NS) {
                    cs = 0;
                    cpar ^= 1u;
                }
                ++n;
            }
            if (stop) break;
            if constexpr (kGau) {
                if (!first) {  // the window above this lattice row is complete
                    const int k = s - 1;
                    const uint32_t yc = (uint32_t)(yc0 + k * h);
                    float acc = 0.f;
#pragma unroll
                    for (int i = 0; i <= DX; ++i) {
                        if (!occupied) break;
                        u64 R[5] = {0, 0, 0, 0, 0};
#pragma unroll
                        for (int l = 0; l <= KY; ++l) R[l] = E[i][l];
                        u64 o[3] = {0, 0, 0};
                        axis_bernstein<DY>(R, yc, (uint32_t)p.ry2, p.ry4, o);
#pragma unroll
                        for (int j = 0; j <= DY; ++j) acc = fmaf(p.gamma[i][j], u64_to_float(o[j]), acc);
                    }
                    if (p.hist && valid_x)
                        p.hist[((int64_t)(yc - p.cy0) * p.ncx + (xc - p.cx0)) * p.B + b0] = acc;
                    if (p.target && occupied) {
                        const float sq = sqrtf(acc);
                        for (int t = 0; t < NT; ++t) s_acc[(t * KC + k) * TX + tid] += sq * s_sq[t * p.B + b0];
                    }
                }
            }
            first = false;
        }
    }
    if (stop) {
        if (lane == 0) atomicOr(p.status, kStatusTimeout);
        return;
    }
    if (p.map && valid_x) {
        for (int t = 0; t < NT; ++t)
            for (int k = 0; k < K; ++k) {
                const int yc = yc0 + k * h;
                const int64_t at = (int64_t)(yc - p.cy0) * p.ncx + (xc - p.cx0);
                const float v = s_acc[(t * KC + k) * TX + tid];
                if constexpr (SPLIT)  // this group's share, summed over the groups by gather_reduce_kernel
                    p.partial[((int64_t)bg * NT + t) * p.ncy * p.ncx + at] = v;
                else
                    p.map[t * p.map_stride + at] = v;
            }
    }
}

// A single job: the grid is (column tiles, chains).
template <int KIND, typename T, int TX, int DX, int DY, int BB, bool SPLIT>
__global__ void __launch_bounds__(TX + 32) gather_tiled_kernel(const __grid_constant__ GatherParams p)
{
    if constexpr (SPLIT)
        gather_tiled_body<KIND, T, TX, DX, DY, BB, true, true>(p, blockIdx.x, blockIdx.y / p.nbg, blockIdx.y % p.nbg);
    else
        gather_tiled_body<KIND, T, TX, DX, DY, BB, false, true>(p, blockIdx.x, blockIdx.y, 0);
}

// The same for the 128-column Gaussian, compiled for 5 resident CTAs: 72
// registers instead of 86 and no spills. Its 3-stage ring fits 4 CTAs in shared
// memory; the leaner code measured 2-5% faster at w = 21 and 81 and 1% slower
// at 41. (A minimum of one CTA written out for the other kernels changed their
// register allocation and slowed them, hence a kernel of its own.)
template <typename T, int DX, int DY, bool SPLIT>
__global__ void __launch_bounds__(128 + 32, 5) gather_gauss128_kernel(const __grid_constant__ GatherParams p)
{
    if constexpr (SPLIT)
        gather_tiled_body<kGatherGaussian, T, 128, DX, DY, 1, true, true>(p, blockIdx.x, blockIdx.y / p.nbg,
                                                                           blockIdx.y % p.nbg);
    else
        gather_tiled_body<kGatherGaussian, T, 128, DX, DY, 1, false, true>(p, blockIdx.x, blockIdx.y, 0);
}

// The 256-column Manhattan and Euclidean gathers in the 32-bit ring with 4 or 2
// bins per step, compiled for 4 resident CTAs (56 registers instead of 71-72, a
// few bytes of spills): 3-6% faster at the benchmark's windows.
template <int KIND, typename T, int TX, int BB>
constexpr bool is_me256 =
    (KIND == kGatherManhattan || KIND == kGatherEuclidean) && TX == 256 && (BB == 4 || BB == 2) && sizeof(T) == 4;

template <int KIND, int BB, bool SPLIT>
__global__ void __launch_bounds__(256 + 32, 4) gather_me256_kernel(const __grid_constant__ GatherParams p)
{
    if constexpr (SPLIT)
        gather_tiled_body<KIND, uint32_t, 256, 0, 0, BB, true, true>(p, blockIdx.x, blockIdx.y / p.nbg,
                                                                     blockIdx.y % p.nbg);
    else
        gather_tiled_body<KIND, uint32_t, 256, 0, 0, BB, false, true>(p, blockIdx.x, blockIdx.y, 0);
}

// the single-job kernel of an instantiation
template <int KIND, typename T, int TX, int DX, int DY, int BB, bool SPLIT>
constexpr auto single_kernel()
{
    if constexpr (KIND == kGatherGaussian && TX == 128 && BB == 1)
        return gather_gauss128_kernel<T, DX, DY, SPLIT>;
    else if constexpr (is_me256<KIND, T, TX, BB>)
        return gather_me256_kernel<KIND, BB, SPLIT>;
    else
        return gather_tiled_kernel<KIND, T, TX, DX, DY, BB, SPLIT>;
}

// A table of jobs sharing one shape: one CTA per work item, items of job j
// numbered from item_start[j] with the column tiles fastest.
template <int KIND, typename T, int TX, int DX, int DY, int BB, bool SMEM_P = false>
__device__ __forceinline__ void gather_table_body(const GatherParams *__restrict__ jobs,
                                                  const int *__restrict__ item_start, int n_jobs, int p_off = 0);

template <int KIND, typename T, int TX, int DX, int DY, int BB>
__global__ void __launch_bounds__(TX + 32)
    gather_table_kernel(const GatherParams *__restrict__ jobs, const int *__restrict__ item_start, int n_jobs)
{
    gather_table_body<KIND, T, TX, DX, DY, BB>(jobs, item_start, n_jobs);
}

// The table kernel's body, and its instantiations with the same register
// bounds as the single-job kernels (the 128-column Gaussian for 5 resident CTAs,
// the 256-column 32-bit Manhattan and Euclidean for 4). With SMEM_P the job's
// parameters are first copied to shared memory at byte p_off (past the shape's
// layout), so that fields the loop reloads come from shared memory, not L1.
template <int KIND, typename T, int TX, int DX, int DY, int BB, bool SMEM_P>
__device__ __forceinline__ void gather_table_body(const GatherParams *__restrict__ jobs,
                                                  const int *__restrict__ item_start, int n_jobs, int p_off)
{
    const int item = blockIdx.x;
    int lo = 0, hi = n_jobs - 1;  // the last job whose first item is <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const GatherParams *pp = jobs + lo;
    if constexpr (SMEM_P) {
        extern __shared__ __align__(128) unsigned char sm[];
        static_assert(sizeof(GatherParams) % 8 == 0, "copied as 8-byte words");
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(pp);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(sm + p_off);
        for (int i = threadIdx.x; i < (int)(sizeof(GatherParams) / 8); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        pp = reinterpret_cast<const GatherParams *>(sm + p_off);
    }
    const GatherParams &p = *pp;
    const int li = item - item_start[lo];
    const int tiles = (p.ncx + TX - 1) / TX;
    gather_tiled_body<KIND, T, TX, DX, DY, BB, false, true>(p, li % tiles, li / tiles, 0);
}

template <typename T, int DX, int DY>
__global__ void __launch_bounds__(128 + 32, 5)
    gather_table_gauss128_kernel(const GatherParams *__restrict__ jobs, const int *__restrict__ item_start, int n_jobs)
{
    gather_table_body<kGatherGaussian, T, 128, DX, DY, 1>(jobs, item_start, n_jobs);
}

template <int KIND, int BB>
__global__ void __launch_bounds__(256 + 32, 4)
    gather_table_me256_kernel(const GatherParams *__restrict__ jobs, const int *__restrict__ item_start, int n_jobs,
                              int p_off)
{
    gather_table_body<KIND, uint32_t, 256, 0, 0, BB, true>(jobs, item_start, n_jobs, p_off);
}

// (gather_table_me256_kernel, for the shapes is_me256 names, takes the
// parameters' shared-memory offset as a fourth argument)
template <int KIND, typename T, int TX, int DX, int DY, int BB>
constexpr auto table_kernel()
{
    if constexpr (KIND == kGatherGaussian && TX == 128 && BB == 1)
        return gather_table_gauss128_kernel<T, DX, DY>;
    else if constexpr (is_me256<KIND, T, TX, BB>)
        return gather_table_me256_kernel<KIND, BB>;
    else
        return gather_table_kernel<KIND, T, TX, DX, DY, BB>;
}

template <int KIND, typename T, int TX, int DX, int DY, int BB>
int kernel_regs()
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, single_kernel<KIND, T, TX, DX, DY, BB, false>()) != cudaSuccess) return 255;
    return fa.numRegs;
}

template <typename KernelFn>
cudaError_t set_smem(KernelFn fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K, typename T, int TX, int DX, int DY, int BB>
cudaError_t run_op(TiledOp &op)
{
    switch (op.what) {
    case TiledOp::kRegs:
        op.regs = kernel_regs<K, T, TX, DX, DY, BB>();
        return cudaSuccess;
    case TiledOp::kSingle: {
        const GatherParams &p = *op.p;
        auto fn = p.nbg > 1 ? single_kernel<K, T, TX, DX, DY, BB, true>()
                            : single_kernel<K, T, TX, DX, DY, BB, false>();
        cudaError_t e = set_smem(fn, op.sh->smem);
        if (e != cudaSuccess) return e;
        const int h = 2 * p.ry + 1;
        const dim3 grid((unsigned)((p.ncx + TX - 1) / TX), (unsigned)(h * p.nblk * p.nbg));
        fn<<<grid, TX + 32, op.sh->smem, op.s>>>(p);
        count_launches(1);
        return cudaGetLastError();
    }
    case TiledOp::kTable: {
        auto fn = table_kernel<K, T, TX, DX, DY, BB>();
        if constexpr (is_me256<K, T, TX, BB>) {
            // the job's parameters follow the shape's layout in shared memory
            const size_t smem = (size_t)op.sh->smem + sizeof(GatherParams);
            cudaError_t e = set_smem(fn, smem);
            if (e != cudaSuccess) return e;
            fn<<<(unsigned)op.n_items, TX + 32, smem, op.s>>>(op.d_jobs, op.d_items, op.n_jobs, (int)op.sh->smem);
        } else {
            cudaError_t e = set_smem(fn, op.sh->smem);
            if (e != cudaSuccess) return e;
            fn<<<(unsigned)op.n_items, TX + 32, op.sh->smem, op.s>>>(op.d_jobs, op.d_items, op.n_jobs);
        }
        count_launches(1);
        return cudaGetLastError();
    }
    }
    return cudaErrorInvalidValue;
}

// every shape of one kind: element type, tile width, bins per step (and, for
// the Gaussian, the fitted degrees)
template <int K>
cudaError_t dispatch_kind(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op)
{
    using u64 = unsigned long long;
    if constexpr (K == kGatherGaussian) {
        if (elem_bytes != 8) return cudaErrorInvalidValue;
        auto by_tx = [&](auto dx_tag, auto dy_tag) -> cudaError_t {
            constexpr int DX = decltype(dx_tag)::value, DY = decltype(dy_tag)::value;
            return tx == 128 ? run_op<K, u64, 128, DX, DY, 1>(op) : run_op<K, u64, 256, DX, DY, 1>(op);
        };
        if (gdx == 2 && gdy == 2) return by_tx(int_tag<2>{}, int_tag<2>{});
        if (gdx == 2 && gdy == 1) return by_tx(int_tag<2>{}, int_tag<1>{});
        if (gdx == 1 && gdy == 2) return by_tx(int_tag<1>{}, int_tag<2>{});
        if (gdx == 1 && gdy == 1) return by_tx(int_tag<1>{}, int_tag<1>{});
        return cudaErrorInvalidValue;
    } else {
        auto by_type = [&](auto t_tag) -> cudaError_t {
            using T = typename decltype(t_tag)::type;
            if (bb == 2) {  // the 256-column 32-bit kernels only
                if constexpr (sizeof(T) == 4)
                    if (tx == 256) return run_op<K, T, 256, 0, 0, 2>(op);
                return cudaErrorInvalidValue;
            }
            if (tx == 128) return bb == 8 ? run_op<K, T, 128, 0, 0, 8>(op) : run_op<K, T, 128, 0, 0, 4>(op);
            return bb == 8 ? run_op<K, T, 256, 0, 0, 8>(op) : run_op<K, T, 256, 0, 0, 4>(op);
        };
        if (elem_bytes == 4) return by_type(template_tag<uint32_t>{});
        if (elem_bytes == 8) return by_type(template_tag<u64>{});
        return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace swih
