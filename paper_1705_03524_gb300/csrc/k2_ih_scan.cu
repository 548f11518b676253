// K2 launchers: the weighted integral histograms of Eq. 2 (the scan kernel and
// its design are described in k2_ih_scan.cuh). This unit instantiates the
// 32- and 64-bit rings with up to 5 x-exponents per chain; wider term sets
// and the 128-bit ring are instantiated in k2_ih_scan_wide.cu.
#include "k2_ih_scan.cuh"

namespace swih {
namespace {

template <typename T>
cudaError_t launch_e(const ScanParams &p, int E, int threads, const ScanRoi *table, int n_roi, long long tiles,
                     cudaStream_t s)
{
    int np = 1;
    for (int i = 0; i < p.n_q; ++i) np = p.p_count[i] > np ? p.p_count[i] : np;
    if (np <= 1) return launch_np<T, 1>(p, E, threads, table, n_roi, tiles, s);
    if (np <= 3) return launch_np<T, 3>(p, E, threads, table, n_roi, tiles, s);
    if (np <= 5) return launch_np<T, 5>(p, E, threads, table, n_roi, tiles, s);
    if (table == nullptr && sizeof(T) == 8) return launch_ih_scan_wide(p, 8, E, threads, s);
    return cudaErrorInvalidValue;
}

// One warp per bin: the bands' last stored rows, a running maximum across the
// bands (warp prefix max, 32 bands at a time), then every row's last stored row.
__device__ __forceinline__ void row_map_body(const unsigned long long *__restrict__ occ, int *__restrict__ row_map,
                                             int H, int band_rows, int n_bands)
{
    const int lane = threadIdx.x;
    int carry = -1;  // last stored row of the bands before this group of 32
    for (int k0 = 0; k0 < n_bands; k0 += 32) {
        const int k = k0 + lane;
        const unsigned long long w = k < n_bands ? occ[k] : 0ull;
        int last = w ? k * band_rows + 63 - __clzll((long long)w) : -1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, last, d);
            if (lane >= d) last = max(last, o);
        }
        int before = __shfl_up_sync(0xffffffffu, last, 1);
        before = max(lane == 0 ? -1 : before, carry);
        if (k < n_bands) {
            const int y0 = k * band_rows, y1 = min(y0 + band_rows, H);
            int cur = before;
            for (int y = y0; y < y1; ++y) {
                if ((w >> (y - y0)) & 1ull) cur = y;
                row_map[y] = cur;
            }
        }
        carry = max(carry, __shfl_sync(0xffffffffu, last, 31));
    }
}

__global__ void __launch_bounds__(32) row_map_kernel(const unsigned long long *__restrict__ occ,
                                                     int *__restrict__ row_map, int H, int band_rows, int n_bands)
{
    const int b = blockIdx.x;
    row_map_body(occ + (int64_t)b * n_bands, row_map + (int64_t)b * H, H, band_rows, n_bands);
}

// block (region i, bin b) = blockIdx.x = i * B + b
__global__ void __launch_bounds__(32) row_map_table_kernel(const ScanRoi *__restrict__ table, int B, int band_rows)
{
    const int i = blockIdx.x / B, b = blockIdx.x - i * B;
    const ScanRoi &r = table[i];
    row_map_body(r.occ + (int64_t)b * r.n_bands, r.row_map + (int64_t)b * r.H, r.H, band_rows, r.n_bands);
}

}  // namespace

cudaError_t launch_row_map(const unsigned long long *occ, int *row_map, int B, int H, int band_rows, int n_bands,
                           cudaStream_t s)
{
    if (band_rows < 1 || band_rows > 64) return cudaErrorInvalidValue;
    row_map_kernel<<<(unsigned)B, 32, 0, s>>>(occ, row_map, H, band_rows, n_bands);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_row_map_table(const ScanRoi *d_table, int n_roi, int B, int band_rows, cudaStream_t s)
{
    if (band_rows < 1 || band_rows > 64) return cudaErrorInvalidValue;
    if ((long long)n_roi * B > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (n_roi <= 0) return cudaSuccess;
    row_map_table_kernel<<<(unsigned)(n_roi * B), 32, 0, s>>>(d_table, B, band_rows);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ih_scan(const ScanParams &p, int elem_bytes, int E, int threads, cudaStream_t s)
{
    if (threads < 32 || threads > kMaxScanThreads || threads % 32) return cudaErrorInvalidValue;
    if (elem_bytes == 4) return launch_e<uint32_t>(p, E, threads, nullptr, 0, 0, s);
    if (elem_bytes == 8) return launch_e<unsigned long long>(p, E, threads, nullptr, 0, 0, s);
    if (elem_bytes == 16) return launch_ih_scan_wide(p, 16, E, threads, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_ih_scan_table(const ScanParams &p, const ScanRoi *d_table, int n_roi, long long tiles,
                                 int elem_bytes, int E, int threads, cudaStream_t s)
{
    if (threads < 32 || threads > kMaxScanThreads || threads % 32) return cudaErrorInvalidValue;
    if (tiles <= 0) return cudaSuccess;
    if (elem_bytes == 4) return launch_e<uint32_t>(p, E, threads, d_table, n_roi, tiles, s);
    if (elem_bytes == 8) return launch_e<unsigned long long>(p, E, threads, d_table, n_roi, tiles, s);
    return cudaErrorInvalidValue;
}

}  // namespace swih
