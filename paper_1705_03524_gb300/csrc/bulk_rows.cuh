// Rows of bytes from global into shared memory by TMA bulk copies: one thread
// issues a copy per row, completion is counted on an mbarrier, and every
// thread waits for at most about 2 s.
#pragma once

#include <cstdint>

namespace swih {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for phase 0 of the mbarrier for at most about 2 s; false when it gave up
__device__ __forceinline__ bool bar_wait0(uint64_t *bar)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 100000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar))
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}

// n_rows rows of seg bytes (seg a multiple of 16; every source row and dst
// 16-byte aligned) into shared memory at dst + o * row_bytes, row o read from
// src_row(o). Thread 0 issues the copies; every thread of the block calls this
// and waits (bounded). The result is the same in every thread of the block:
// false when any thread's wait gave up.
template <typename SrcRow>
__device__ __forceinline__ bool rows_bulk(uint64_t *bar, uint8_t *dst, int row_bytes, int n_rows, uint32_t seg,
                                          SrcRow src_row)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"((uint32_t)n_rows * seg)
                     : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int o = 0; o < n_rows; ++o)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(dst + (size_t)o * row_bytes)),
                "l"(src_row(o)), "r"(seg), "r"(smem_u32(bar))
                : "memory");
    }
    bool ok = bar_wait0(bar);
    if (!ok) ok = bar_wait0(bar);  // copies in flight still land in this block's shared memory: wait once more
    return !__syncthreads_or(!ok);
}

}  // namespace
}  // namespace swih
