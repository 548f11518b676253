// K1: quantisation Q of Sec. 2.1 (named after Eq. 2): pixel value -> bin.
//
//   b = floor(min(v, 2^bitdepth - 1) * B / 2^bitdepth)   (equal-width bins)
//
// (plus a constant bin0 for a feature channel whose bins follow other channels')
//
// One thread per 16 consecutive pixels of a row. With a 16-byte aligned image
// a u8 chunk is one 16-byte load and a u16 chunk two; the 16 bins leave as one
// 16-byte store. HBM-bound: (pixel bytes + 1) bytes per pixel.
#include "swih_internal.h"

namespace swih {
namespace {

__device__ __forceinline__ uint32_t bin_of(uint32_t v, uint32_t vmax, uint32_t B, int bitdepth)
{
    v = v > vmax ? vmax : v;
    return (v * B) >> bitdepth;
}

// bins of the 16-pixel chunk starting at column x0 of row y
template <int PB>
__device__ __forceinline__ void quantize_chunk(const uint8_t *image, int64_t pitch, int W, int y, int x0,
                                               bool vec, uint32_t vmax, uint32_t B, int bitdepth,
                                               uint8_t *bins, int64_t bins_pitch, uint32_t bin0 = 0)
{
    const uint8_t *row = image + (int64_t)y * pitch;
    uint32_t v[16];
    if (vec && x0 + 16 <= W) {
        if (PB == 1) {
            const uint4 u = *reinterpret_cast<const uint4 *>(row + x0);
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
        } else {
            const uint4 u0 = *reinterpret_cast<const uint4 *>(row + 2 * x0);
            const uint4 u1 = *reinterpret_cast<const uint4 *>(row + 2 * x0 + 16);
            const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = (w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int x = x0 + i;
            if (x < W) {
                v[i] = PB == 1 ? (uint32_t)row[x] : (uint32_t)reinterpret_cast<const uint16_t *>(row)[x];
            } else {
                v[i] = 0;
            }
        }
    }
    uint32_t o[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i >> 2] |= (bin0 + bin_of(v[i], vmax, B, bitdepth)) << (8 * (i & 3));
    *reinterpret_cast<uint4 *>(bins + (int64_t)y * bins_pitch + x0) = make_uint4(o[0], o[1], o[2], o[3]);
}

template <int PB>
__global__ void __launch_bounds__(256) quantize_kernel(QuantParams p)
{
    const int chunks_per_row = (p.W + 15) >> 4;
    const long long n_chunks = (long long)chunks_per_row * p.H;
    const uint32_t vmax = (1u << p.bitdepth) - 1u;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_chunks;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / chunks_per_row);
        const int x0 = (int)(c - (long long)y * chunks_per_row) << 4;
        quantize_chunk<PB>(p.image, p.pitch, p.W, y, x0, p.vec != 0, vmax, (uint32_t)p.B, p.bitdepth, p.bins,
                           p.bins_pitch, (uint32_t)p.bin0);
    }
}

// every chunk of several image regions; region i owns chunks
// [table[i].chunk0, table[i + 1].chunk0)
template <int PB>
__global__ void __launch_bounds__(256)
    quantize_table_kernel(const QuantRoi *__restrict__ table, int n, long long n_chunks, int B, int bitdepth)
{
    const uint32_t vmax = (1u << bitdepth) - 1u;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_chunks;
         c += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid].chunk0 <= c) lo = mid; else hi = mid - 1;
        }
        const QuantRoi &r = table[lo];
        const long long local = c - r.chunk0;
        const int chunks_per_row = (r.W + 15) >> 4;
        const int y = (int)(local / chunks_per_row);
        const int x0 = (int)(local - (long long)y * chunks_per_row) << 4;
        quantize_chunk<PB>(r.image, r.pitch, r.W, y, x0, r.vec != 0, vmax, (uint32_t)B, bitdepth, r.bins,
                           r.bins_pitch);
    }
}

}  // namespace

cudaError_t launch_quantize(const QuantParams &p, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long n_chunks = (long long)((p.W + 15) / 16) * p.H;
    long long blocks = (n_chunks + 255) / 256;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (p.pixel_bytes == 1)
        quantize_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(p);
    else
        quantize_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_quantize_table(const QuantRoi *d_table, int n, long long n_chunks, int B, int bitdepth,
                                  int pixel_bytes, cudaStream_t s)
{
    if (n_chunks <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n_chunks + 255) / 256;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (pixel_bytes == 1)
        quantize_table_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(d_table, n, n_chunks, B, bitdepth);
    else
        quantize_table_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(d_table, n, n_chunks, B, bitdepth);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace swih
