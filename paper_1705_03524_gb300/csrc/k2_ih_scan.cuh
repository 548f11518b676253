// K2: weighted integral histograms (Eq. 2), one per bin b and weight term x^p y^q:
//
//   IH_pq(x, y, b) = sum_{i<=x, j<=y} [bin(i, j) = b] * i^p * j^q
//
// kept exactly in the ring of integers mod 2^32 or 2^64 (type T wraps).
//
// Factorisation used: with the column sums
//   cs_q(x, y) = sum_{j<=y} [bin(x, j) = b] * j^q,
// every term sharing q is a row prefix sum of a column scaled by x^p:
//   IH_pq(x, y) = sum_{i<=x} i^p * cs_q(i, y).
// So one "chain" per (b, q) carries cs_q down the image, and each row of the
// chain emits one block-wide row scan per p.
//
// Work decomposition: the image is cut into horizontal bands of band_rows
// full-width rows. A CTA takes one (chain, band) tile in ticket order (an
// atomic counter), so every tile it may wait for has already started.
// The column carry into a band comes from a single-pass decoupled look-back
// over the bands above it (Merrill & Garland's scheme, carried on W-wide state
// vectors instead of scalars):
//   1. sum the band's own rows into a per-column aggregate, publish it
//      (flag AGGREGATE; band 0 publishes its INCLUSIVE value directly); when
//      the band's bins fit in shared memory they arrive there first, every
//      row at once, by TMA bulk copies (bulk_rows.cuh);
//   2. walk back over earlier bands, adding aggregates until an INCLUSIVE
//      vector is found; every wait is bounded and a wait that gives up marks
//      the tile ERROR and sets the plan's status word;
//   3. publish carry + aggregate as INCLUSIVE;
//   4. sweep the band again, carrying cs_q in registers, and write each row of
//      every term of the chain with a block-wide scan (thread-serial over E
//      columns, warp shuffles, then a cross-warp pass through shared memory),
//      reading the bins from shared memory (or, for bands too tall to keep
//      there, loading the next row's bins while the current row is scanned).
// Output writes are full rows, coalesced, each IH element written once; the
// bin image (1 byte per pixel) is read once per tile when the band's bins are
// kept in shared memory, else twice, and stays in L2.
#pragma once

#include "bulk_rows.cuh"
#include "ring128.h"
#include "swih_internal.h"

namespace swih {
namespace {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T ring_pow(T base, int e)
{
    T r = 1;
    for (int i = 0; i < e; ++i) r *= base;
    return r;
}

// a warp shuffle of a ring element (two for the 128-bit ring)
template <typename T>
__device__ __forceinline__ T ring_shfl_up(T v, int o)
{
    if constexpr (sizeof(T) == 16) {
        return T(__shfl_up_sync(0xffffffffu, v.lo, o), __shfl_up_sync(0xffffffffu, v.hi, o));
    } else {
        return __shfl_up_sync(0xffffffffu, v, o);
    }
}

// v * f for a ring element v and a factor f < 2^32 (64-bit ring: two IMADs)
template <typename T>
__device__ __forceinline__ T mul_small(T v, uint32_t f)
{
    if constexpr (sizeof(T) == 4) {
        return v * f;
    } else if constexpr (sizeof(T) == 16) {
        return mul64(v, f);
    } else {
        const unsigned long long lo = (unsigned long long)(uint32_t)v * f;
        const uint32_t hi = (uint32_t)(v >> 32) * f;
        return lo + ((unsigned long long)hi << 32);
    }
}

// E consecutive bins starting at column x0 (x0 multiple of E, row 16-byte aligned)
template <int E>
__device__ __forceinline__ void load_bins(const uint8_t *row, int x0, uint8_t (&v)[E])
{
    if constexpr (E == 4) {
        const uint32_t u = *reinterpret_cast<const uint32_t *>(row + x0);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (uint8_t)(u >> (8 * i));
    } else if constexpr (E == 8) {
        const uint2 u = *reinterpret_cast<const uint2 *>(row + x0);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (uint8_t)(u.x >> (8 * i));
#pragma unroll
        for (int i = 0; i < 4; ++i) v[4 + i] = (uint8_t)(u.y >> (8 * i));
    } else {
#pragma unroll
        for (int c = 0; c < E / 16; ++c) {
            const uint4 u = *reinterpret_cast<const uint4 *>(row + x0 + 16 * c);
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int i = 0; i < 16; ++i) v[16 * c + i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
        }
    }
}

// dst[0..E) = src[0..E) (16-byte accesses; src is a row this thread stored)
template <typename T, int E>
__device__ __forceinline__ void copy_row(T *dst, const T *src)
{
    constexpr int n = E * (int)sizeof(T) / 16;
#pragma unroll
    for (int c = 0; c < n; ++c) reinterpret_cast<uint4 *>(dst)[c] = reinterpret_cast<const uint4 *>(src)[c];
}

// E bins back into a byte row (the shared-memory copy of the band's bins)
template <int E>
__device__ __forceinline__ void put_bins(uint8_t *row, int x0, const uint8_t (&v)[E])
{
    if constexpr (E == 4) {
        uint32_t u = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) u |= (uint32_t)v[i] << (8 * i);
        *reinterpret_cast<uint32_t *>(row + x0) = u;
    } else {
#pragma unroll
        for (int c = 0; c < E / 8; ++c) {
            uint2 u = make_uint2(0u, 0u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                u.x |= (uint32_t)v[8 * c + i] << (8 * i);
                u.y |= (uint32_t)v[8 * c + 4 + i] << (8 * i);
            }
            reinterpret_cast<uint2 *>(row + x0)[c] = u;
        }
    }
}

// store E consecutive ring elements (16-byte aligned) with 16-byte vector stores
template <typename T, int E>
__device__ __forceinline__ void store_row(T *dst, const T (&v)[E])
{
    constexpr int per = 16 / sizeof(T);
#pragma unroll
    for (int c = 0; c < E / per; ++c) {
        if constexpr (sizeof(T) == 4) {
            reinterpret_cast<uint4 *>(dst)[c] =
                make_uint4((uint32_t)v[4 * c], (uint32_t)v[4 * c + 1], (uint32_t)v[4 * c + 2],
                           (uint32_t)v[4 * c + 3]);
        } else if constexpr (sizeof(T) == 16) {
            reinterpret_cast<ulonglong2 *>(dst)[c] = make_ulonglong2(v[c].lo, v[c].hi);
        } else {
            reinterpret_cast<ulonglong2 *>(dst)[c] =
                make_ulonglong2((unsigned long long)v[2 * c], (unsigned long long)v[2 * c + 1]);
        }
    }
}

template <typename T, int E>
__device__ __forceinline__ void store_state(T *dst, const T (&v)[E])
{
    constexpr int per = 16 / sizeof(T);
#pragma unroll
    for (int c = 0; c < E / per; ++c) {
        if constexpr (sizeof(T) == 4) {
            __stcg(reinterpret_cast<uint4 *>(dst) + c,
                   make_uint4((uint32_t)v[4 * c], (uint32_t)v[4 * c + 1], (uint32_t)v[4 * c + 2],
                              (uint32_t)v[4 * c + 3]));
        } else if constexpr (sizeof(T) == 16) {
            __stcg(reinterpret_cast<ulonglong2 *>(dst) + c, make_ulonglong2(v[c].lo, v[c].hi));
        } else {
            __stcg(reinterpret_cast<ulonglong2 *>(dst) + c,
                   make_ulonglong2((unsigned long long)v[2 * c], (unsigned long long)v[2 * c + 1]));
        }
    }
}

template <typename T, int E>
__device__ __forceinline__ void add_state(const T *src, T (&acc)[E])
{
    constexpr int per = 16 / sizeof(T);
#pragma unroll
    for (int c = 0; c < E / per; ++c) {
        if constexpr (sizeof(T) == 4) {
            const uint4 u = __ldcg(reinterpret_cast<const uint4 *>(src) + c);
            acc[4 * c] += u.x;
            acc[4 * c + 1] += u.y;
            acc[4 * c + 2] += u.z;
            acc[4 * c + 3] += u.w;
        } else if constexpr (sizeof(T) == 16) {
            const ulonglong2 u = __ldcg(reinterpret_cast<const ulonglong2 *>(src) + c);
            acc[c] += T(u.x, u.y);
        } else {
            const ulonglong2 u = __ldcg(reinterpret_cast<const ulonglong2 *>(src) + c);
            acc[2 * c] += u.x;
            acc[2 * c + 1] += u.y;
        }
    }
}

// One (chain, band) tile of one image region r; ticket = its ticket number.
template <typename T, int E, int NP, bool RUNS, bool SPARSE>
__device__ __forceinline__ void scan_tile(const ScanParams &p, const ScanRoi &r, const int ticket,
                                          const int band, const int chain)
{
    __shared__ int s_flag;
    __shared__ T s_warp[2][32];
    __shared__ unsigned long long s_rows;  // band rows (first 64) holding a pixel of bin b
    extern __shared__ __align__(16) uint8_t s_band_bins[];  // the band's bins when p.sb_rows > 0
    const int row_bytes = (int)blockDim.x * E;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int b = chain / p.n_q;
    const int qi = chain - b * p.n_q;
    const int q = p.q_val[qi];
    const int y_begin = band * p.band_rows;
    const int y_end = min(y_begin + p.band_rows, r.H);
    const int x0 = tid * E;
    const bool has_cols = x0 < r.W;               // any real column in this thread
    const bool in_pitch = x0 < r.ih_pitch;        // chunk lies inside a stored row
    const uint8_t bb = (uint8_t)b;
    const uint8_t *bins = r.bins + (int64_t)p.ch_of_bin[b] * p.ch_stride;  // the plane of b's feature channel
    if (ticket == p.stall_tile && band == 0) return;  // injected stall: publish nothing

    // ---- 1. band aggregate of [bin == b] * y^q per column, and which rows hold the bin.
    // When the band's bins are kept in shared memory they arrive there first,
    // all rows at once, by bulk copies (a row at a time, each a dependent global
    // load, exposed the memory latency once per row in short tiles).
    if (tid == 0) s_rows = 0ull;
    const bool bulk = p.sb_rows > 0 && ((reinterpret_cast<uintptr_t>(bins) | (uintptr_t)r.bins_pitch) & 15) == 0;
    if (bulk) {
        __shared__ __align__(8) uint64_t s_bar;
        const uint32_t seg = (uint32_t)((r.W + 15) & ~15);
        const uint8_t *band_src = bins + (int64_t)y_begin * r.bins_pitch;
        const int64_t pitch = r.bins_pitch;
        if (!rows_bulk(&s_bar, s_band_bins, row_bytes, y_end - y_begin, seg,
                       [&](int o) { return band_src + (int64_t)o * pitch; })) {
            if (tid == 0) {
                atomicOr(p.status, kStatusTimeout);
                st_release(r.flags + (int64_t)chain * r.n_bands + band, kFlagError);
            }
            return;  // uniform over the block
        }
    }
    T agg[E];
#pragma unroll
    for (int e = 0; e < E; ++e) agg[e] = 0;
    unsigned long long my_rows = 0ull;
    if (has_cols) {
        for (int y = y_begin; y < y_end; ++y) {
            uint8_t v[E];
            if (bulk) {
                load_bins<E>(s_band_bins + (y - y_begin) * row_bytes, x0, v);
            } else {
                load_bins<E>(bins + (int64_t)y * r.bins_pitch, x0, v);
                if (p.sb_rows > 0) put_bins<E>(s_band_bins + (y - y_begin) * row_bytes, x0, v);
            }
            bool hit[E];
            bool any = false;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                hit[e] = v[e] == bb && x0 + e < r.W;
                any |= hit[e];
            }
            if (!any) continue;  // y^q only for rows where this thread's columns hold the bin
            const T yq = ring_pow<T>((T)y, q);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (hit[e]) agg[e] += yq;
            if ((NP <= 3 || RUNS || SPARSE) && y - y_begin < 64) my_rows |= 1ull << (y - y_begin);
        }
    }
    __syncthreads();  // s_rows cleared
    if (my_rows) atomicOr(&s_rows, my_rows);

    const int64_t state_row = ((int64_t)chain * r.n_bands + band) * r.ih_pitch;
    int *my_flag = r.flags + (int64_t)chain * r.n_bands + band;
    if (in_pitch) store_state<T, E>((band == 0 ? (T *)r.incl : (T *)r.agg) + state_row + x0, agg);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        st_release(my_flag, band == 0 ? kFlagInclusive : kFlagAggregate);
        if (SPARSE && qi == 0) r.occ[(int64_t)b * r.n_bands + band] = s_rows;  // the rows this bin stores
    }

    // ---- 2. look back over the bands above for the column carry
    T carry[E];
#pragma unroll
    for (int e = 0; e < E; ++e) carry[e] = 0;
    bool failed = false;
    if (band > 0) {
        int j = band - 1;
        while (true) {
            if (tid == 0) {
                const int *fp = r.flags + (int64_t)chain * r.n_bands + j;
                int f = ld_acquire(fp);
                long long it = 0;
                while (f == kFlagEmpty) {
                    if (++it > p.spin_limit) {
                        f = kFlagError;
                        atomicOr(p.status, kStatusTimeout);
                        break;
                    }
                    __nanosleep(64);
                    f = ld_acquire(fp);
                }
                s_flag = f;
            }
            __syncthreads();
            const int f = s_flag;
            __syncthreads();
            if (f == kFlagError) {
                failed = true;
                break;
            }
            const T *src = (f == kFlagInclusive ? (const T *)r.incl : (const T *)r.agg) +
                           ((int64_t)chain * r.n_bands + j) * r.ih_pitch;
            if (in_pitch) add_state<T, E>(src + x0, carry);
            if (f == kFlagInclusive || j == 0) break;
            --j;
        }
        // ---- 3. publish the inclusive column sums of this band
        if (!failed && in_pitch) {
            T inc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) inc[e] = carry[e] + agg[e];
            store_state<T, E>((T *)r.incl + state_row + x0, inc);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(my_flag, failed ? kFlagError : kFlagInclusive);
        }
    }
    if (failed) return;  // uniform over the block (decided from s_flag)

    // ---- 4. sweep the band: column sums in registers; per row and term x^k y^q
    // (k < n_p), one block-wide scan: thread-serial over the E columns, warp
    // shuffles, then the warp totals through shared memory (double-buffered, one
    // barrier per scan). The values x^k cs(x) are built by repeated
    // multiplication by x (x < 2^13); the next row's bins are loaded while the
    // current row is scanned.
    const int n_p = p.p_count[qi];  // the chain's x-exponents are 0..n_p-1 (n_p <= NP)
    T cs[E];
#pragma unroll
    for (int e = 0; e < E; ++e) cs[e] = carry[e];
    int parity = 0;
    const unsigned long long rows = s_rows;  // read after the barrier of step 1's publication
    // the next row the sweep visits: with SPARSE only rows holding a pixel of bin
    // b (any other row changes no column sum and is not stored; bands are at most
    // 64 rows, all in the mask), otherwise every row
    auto next_row = [&](int y) -> int {
        if constexpr (SPARSE) {
            const int o = y - y_begin;
            const unsigned long long m = o < 64 ? rows >> o : 0ull;
            return m ? y + __ffsll((long long)m) - 1 : y_end;
        } else {
            return y;
        }
    };
    const int y_first = next_row(y_begin);
    uint8_t vnext[E];
    const bool cached = p.sb_rows > 0;  // each thread reads back the bins it stored in step 1
    if (!cached && has_cols && y_first < y_end) load_bins<E>(bins + (int64_t)y_first * r.bins_pitch, x0, vnext);
    // Rows without a pixel of bin b leave every column sum, hence every term's
    // row, as in the row above. With up to 3 terms per chain such a row is
    // copied from the row this thread stored last (still in L2) instead of
    // scanned. With the Gaussian's 5 terms of 8 bytes the copies' latency costs
    // more than the scans they save: with RUNS (the table kernel of many
    // regions, where it measured faster) each computed row is stored again into
    // the empty rows after it, from registers; otherwise every row is scanned. The band's first row is
    // always computed; rows past the first 64 count as holding b. With SPARSE
    // (bands of at most 64 rows) an empty row is neither scanned nor stored:
    // readers take the last stored row through the plan's row map.
    constexpr bool kSkip = NP <= 3 && !SPARSE;
    for (int y = y_first, yn; y < y_end; y = yn) {
        yn = next_row(y + 1);  // uniform over the block
        if (has_cols) {
            uint8_t v[E];
            if (cached) {
                load_bins<E>(s_band_bins + (y - y_begin) * row_bytes, x0, v);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = vnext[e];
                if (yn < y_end) load_bins<E>(bins + (int64_t)yn * r.bins_pitch, x0, vnext);
            }
            const T yq = ring_pow<T>((T)y, q);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (v[e] == bb && x0 + e < r.W) cs[e] += yq;
        }
        if constexpr (kSkip) {
            const bool holds = y - y_begin >= 64 || ((rows >> (y - y_begin)) & 1ull);
            if (y > y_begin && !holds) {
                if (in_pitch) {
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        if (k >= n_p) break;
                        T *row = (T *)r.ih + ((int64_t)p.term[qi][k] * p.B + b) * r.plane + (int64_t)y * r.ih_pitch;
                        copy_row<T, E>(row + x0, row - r.ih_pitch + x0);
                    }
                }
                continue;
            }
        }
        int run = 1;  // this row and the empty rows stored with it
        if constexpr (!kSkip && !SPARSE && RUNS) {
            auto holds = [&](int yy) { return yy - y_begin >= 64 || ((rows >> (yy - y_begin)) & 1ull); };
            if (y > y_begin && !holds(y)) continue;
            while (y + run < y_end && !holds(y + run)) ++run;
        }
        T cur[E];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (k >= n_p) break;
            T val[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                cur[e] = k == 0 ? cs[e] : mul_small<T>(cur[e], (uint32_t)(x0 + e));
                val[e] = e == 0 ? cur[0] : val[e - 1] + cur[e];
            }
            const T tot = val[E - 1];
            T inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T n = ring_shfl_up<T>(inc, o);
                if (lane >= o) inc += n;
            }
            if (lane == 31) s_warp[parity][warp] = inc;
            __syncthreads();
            T off = inc - tot;
            for (int w = 0; w < warp; ++w) off += s_warp[parity][w];
#pragma unroll
            for (int e = 0; e < E; ++e) val[e] += off;
            if (in_pitch) {
                T *row = (T *)r.ih + ((int64_t)p.term[qi][k] * p.B + b) * r.plane +
                         (int64_t)y * r.ih_pitch;
                if constexpr (!kSkip && !SPARSE && RUNS) {
                    for (int i = 0; i < run; ++i) store_row<T, E>(row + (int64_t)i * r.ih_pitch + x0, val);
                } else {
                    store_row<T, E>(row + x0, val);
                }
            }
            parity ^= 1;
        }
    }
}

template <typename T, int E, int NP, bool SPARSE>
__device__ __forceinline__ void plan_scan(const ScanParams &p);

template <typename T, int E, int NP, bool SPARSE>
__global__ void __launch_bounds__(kMaxScanThreads) ih_scan_kernel(const __grid_constant__ ScanParams p)
{
    plan_scan<T, E, NP, SPARSE>(p);
}

// The same for 256-thread blocks, compiled for 5 resident blocks per SM (at
// most 51 registers): the Gaussian plan's scan of images up to 1024 columns
template <typename T, int E, int NP, bool SPARSE>
__global__ void __launch_bounds__(256, 5) ih_scan_kernel_256x5(const __grid_constant__ ScanParams p)
{
    plan_scan<T, E, NP, SPARSE>(p);
}

template <typename T, int E, int NP, bool SPARSE>
__device__ __forceinline__ void plan_scan(const ScanParams &p)
{
    __shared__ int s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(p.ticket, 1);
    __syncthreads();
    const int ticket = s_ticket;
    const int n_chains = p.B * p.n_q;
    const int band = ticket / n_chains;
    ScanRoi r;
    r.bins = p.bins;
    r.bins_pitch = p.bins_pitch;
    r.ih = p.ih;
    r.ih_pitch = p.ih_pitch;
    r.plane = p.plane;
    r.agg = p.agg;
    r.incl = p.incl;
    r.flags = p.flags;
    r.H = p.H;
    r.W = p.W;
    r.n_bands = p.n_bands;
    r.ticket0 = 0;
    r.occ = p.occ;
    r.row_map = nullptr;
    scan_tile<T, E, NP, false, SPARSE>(p, r, ticket, band, ticket - band * n_chains);
}

// Several image regions in one launch: region i owns the tickets
// [table[i].ticket0, table[i + 1].ticket0), band-major, so every tile a tile
// may wait for (the same chain, an earlier band, the same region) holds a
// smaller ticket and has already started.
template <typename T, int E, int NP, bool SPARSE>
__global__ void __launch_bounds__(kMaxScanThreads)
    ih_scan_table_kernel(const __grid_constant__ ScanParams p, const ScanRoi *__restrict__ table, int n)
{
    __shared__ int s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(p.ticket, 1);
    __syncthreads();
    const int ticket = s_ticket;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].ticket0 <= ticket) lo = mid; else hi = mid - 1;
    }
    const ScanRoi r = table[lo];
    const int local = ticket - r.ticket0;
    const int n_chains = p.B * p.n_q;
    const int band = local / n_chains;
    scan_tile<T, E, NP, !SPARSE, SPARSE>(p, r, ticket, band, local - band * n_chains);
}

// the kernel's dynamic shared memory limit raised to `bytes` when the default
// 48 KB does not hold them beside the kernel's static shared memory
template <typename KernelFn>
cudaError_t allow_smem(KernelFn fn, size_t bytes)
{
    if (bytes == 0) return cudaSuccess;
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (bytes + fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int E, int NP>
cudaError_t launch_typed(const ScanParams &p_in, int threads, const ScanRoi *table, int n_roi, long long tiles,
                         cudaStream_t s)
{
    // the band's bins stay in shared memory between the aggregate pass and the
    // sweep when the band is at most 64 rows and the copy at most 96 KB
    ScanParams p = p_in;
    const size_t per_row = (size_t)threads * E;
    p.sb_rows = (p.band_rows <= 64 && (size_t)p.band_rows * per_row <= 96 * 1024) ? p.band_rows : 0;
    const size_t smem = (size_t)p.sb_rows * per_row;
    cudaError_t e;
    constexpr bool kTable = NP <= 5 && sizeof(T) <= 8;  // work sets use the narrow term sets only
    if constexpr (!kTable) {
        if (table) return cudaErrorInvalidValue;
    }
    if (kTable && table && p.occ) {
        if (p.band_rows > 64) return cudaErrorInvalidValue;  // the occupancy word covers 64 rows
        if constexpr (kTable) {
            e = allow_smem(ih_scan_table_kernel<T, E, NP, true>, smem);
            if (e != cudaSuccess) return e;
            ih_scan_table_kernel<T, E, NP, true><<<(unsigned)tiles, threads, smem, s>>>(p, table, n_roi);
        }
    } else if (kTable && table) {
        if constexpr (kTable) {
            e = allow_smem(ih_scan_table_kernel<T, E, NP, false>, smem);
            if (e != cudaSuccess) return e;
            ih_scan_table_kernel<T, E, NP, false><<<(unsigned)tiles, threads, smem, s>>>(p, table, n_roi);
        }
    } else if (p.occ) {
        if (p.band_rows > 64) return cudaErrorInvalidValue;  // the occupancy word covers 64 rows
        if constexpr (sizeof(T) == 8 && NP == 5 && E == 4) {
            if (threads == 256) {
                // the Gaussian plan's scan: 5 resident blocks need the full shared-memory carve-out
                e = allow_smem(ih_scan_kernel_256x5<T, E, NP, true>, smem);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(ih_scan_kernel_256x5<T, E, NP, true>,
                                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
                if (e != cudaSuccess) return e;
                ih_scan_kernel_256x5<T, E, NP, true>
                    <<<(unsigned)((long long)p.B * p.n_q * p.n_bands), threads, smem, s>>>(p);
                count_launches(1);
                return cudaGetLastError();
            }
        }
        e = allow_smem(ih_scan_kernel<T, E, NP, true>, smem);
        if (e != cudaSuccess) return e;
        ih_scan_kernel<T, E, NP, true><<<(unsigned)((long long)p.B * p.n_q * p.n_bands), threads, smem, s>>>(p);
    } else {
        e = allow_smem(ih_scan_kernel<T, E, NP, false>, smem);
        if (e != cudaSuccess) return e;
        ih_scan_kernel<T, E, NP, false><<<(unsigned)((long long)p.B * p.n_q * p.n_bands), threads, smem, s>>>(p);
    }
    count_launches(1);
    return cudaGetLastError();
}

// NP: a compile-time bound on the x-exponents per chain (1: plain; 3: up to
// the Euclidean terms; 5: the Gaussian), so the per-row term loop unrolls
template <typename T, int NP>
cudaError_t launch_np(const ScanParams &p, int E, int threads, const ScanRoi *table, int n_roi, long long tiles,
                      cudaStream_t s)
{
    switch (E) {
    case 4: return launch_typed<T, 4, NP>(p, threads, table, n_roi, tiles, s);
    case 8: return launch_typed<T, 8, NP>(p, threads, table, n_roi, tiles, s);
    case 16: return launch_typed<T, 16, NP>(p, threads, table, n_roi, tiles, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace swih
