// The ring of integers modulo 2^128 as two 64-bit limbs, for the integral
// histograms of Gaussian windows whose exact moments pass 2^64. Addition and
// subtraction carry through the PTX add.cc / sub.cc chains on the device;
// products keep the low 128 bits. Default construction leaves the value
// uninitialised (so the type may live in shared memory); construction from an
// unsigned integer zero-extends it.
#pragma once

#include <cstdint>

namespace swih {

struct alignas(16) u128 {
    unsigned long long lo, hi;
    u128() = default;
    __host__ __device__ constexpr u128(unsigned long long v) : lo(v), hi(0ull) {}
    __host__ __device__ constexpr u128(unsigned long long l, unsigned long long h) : lo(l), hi(h) {}
};

// the two's-complement image of a signed 64-bit value
__host__ __device__ inline u128 u128_from_i64(long long v)
{
    return u128((unsigned long long)v, v < 0 ? ~0ull : 0ull);
}

__host__ __device__ inline u128 operator+(u128 a, u128 b)
{
    u128 r;
#ifdef __CUDA_ARCH__
    asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
        : "=l"(r.lo), "=l"(r.hi)
        : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
#else
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
#endif
    return r;
}

__host__ __device__ inline u128 operator-(u128 a, u128 b)
{
    u128 r;
#ifdef __CUDA_ARCH__
    asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;"
        : "=l"(r.lo), "=l"(r.hi)
        : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
#else
    r.lo = a.lo - b.lo;
    r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
#endif
    return r;
}

__host__ __device__ inline unsigned long long mul_hi64(unsigned long long a, unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

// a * b mod 2^128
__host__ __device__ inline u128 operator*(u128 a, u128 b)
{
    return u128(a.lo * b.lo, mul_hi64(a.lo, b.lo) + a.lo * b.hi + a.hi * b.lo);
}

// a * f mod 2^128 for a 64-bit factor
__host__ __device__ inline u128 mul64(u128 a, unsigned long long f)
{
    return u128(a.lo * f, mul_hi64(a.lo, f) + a.hi * f);
}

__host__ __device__ inline u128 &operator+=(u128 &a, u128 b) { return a = a + b; }
__host__ __device__ inline u128 &operator-=(u128 &a, u128 b) { return a = a - b; }
__host__ __device__ inline u128 &operator*=(u128 &a, u128 b) { return a = a * b; }
__host__ __device__ inline bool operator==(u128 a, u128 b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ inline bool operator!=(u128 a, u128 b) { return !(a == b); }

// the value of a non-negative element (below 2^128) as a double, rounded
__host__ __device__ inline double u128_to_double(u128 a)
{
    return (double)a.hi * 18446744073709551616.0 + (double)a.lo;
}

}  // namespace swih
