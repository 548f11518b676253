// K2 launchers for the wide term sets: Gaussian approximants of degree 3 and
// 4 (7 or 9 x-exponents per chain) in the 64-bit ring, and every Gaussian
// term set in the 128-bit ring (windows whose exact moments pass 2^64). Single
// plans only; the kernel is the one of k2_ih_scan.cuh.
#include "k2_ih_scan.cuh"

namespace swih {

namespace {

template <typename T>
cudaError_t launch_wide_t(const ScanParams &p, int E, int threads, cudaStream_t s)
{
    int np = 1;
    for (int i = 0; i < p.n_q; ++i) np = p.p_count[i] > np ? p.p_count[i] : np;
    if constexpr (sizeof(T) == 16) {
        // 128-bit elements: at most 8 columns per thread (widths up to 4096)
        if (E > 8) return cudaErrorInvalidValue;
        if (np <= 3) return launch_np<T, 3>(p, E, threads, nullptr, 0, 0, s);
        if (np <= 5) return launch_np<T, 5>(p, E, threads, nullptr, 0, 0, s);
    }
    if (np <= 7) return launch_np<T, 7>(p, E, threads, nullptr, 0, 0, s);
    if (np <= 9) return launch_np<T, 9>(p, E, threads, nullptr, 0, 0, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_ih_scan_wide(const ScanParams &p, int elem_bytes, int E, int threads, cudaStream_t s)
{
    if (threads < 32 || threads > kMaxScanThreads || threads % 32) return cudaErrorInvalidValue;
    if (elem_bytes == 8) return launch_wide_t<unsigned long long>(p, E, threads, s);
    if (elem_bytes == 16) return launch_wide_t<u128>(p, E, threads, s);
    return cudaErrorInvalidValue;
}

}  // namespace swih
