// gd_device.cuh -- small device helpers shared by the kernel translation
// units of libgd (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gdi {
namespace dev {

constexpr int WARP = 32;

__device__ __forceinline__ int32_t ldg(const int32_t *p) { return __ldg(p); }

// Degree ordering: a precedes b iff (d_a, a) < (d_b, b).
__device__ __forceinline__ bool precedes(int32_t da, int32_t a, int32_t db, int32_t b) {
    return da < db || (da == db && a < b);
}

// first index i in [0,len) with a[i] >= key (len if none)
__device__ __forceinline__ int32_t lower_bound(const int32_t *a, int32_t len, int32_t key) {
    int32_t lo = 0;
    while (len > 0) {
        int32_t half = len >> 1;
        if (ldg(a + lo + half) < key) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo;
}

__device__ __forceinline__ int32_t find_in(const int32_t *a, int32_t len, int32_t key) {
    int32_t i = lower_bound(a, len, key);
    return (i < len && ldg(a + i) == key) ? i : -1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// inclusive prefix sum across the warp
__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// u128 accumulation into (lo, hi) words
__device__ __forceinline__ void add_u128(unsigned long long *lohi, unsigned long long x) {
    if (x == 0) return;
    unsigned long long old = atomicAdd(lohi, x);
    if (old + x < old) atomicAdd(lohi + 1, 1ull);
}

typedef unsigned __int128 u128;

// a full 128-bit addend into (lo, hi) words: the carry out of the low word
// joins the high addend (concurrent adders: the total is exact mod 2^128)
__device__ __forceinline__ void add_u128_wide(unsigned long long *lohi, u128 x) {
    const unsigned long long lo = (unsigned long long)x;
    unsigned long long hi = (unsigned long long)(x >> 64);
    if (lo) {
        const unsigned long long old = atomicAdd(lohi, lo);
        if (old + lo < old) hi += 1;
    }
    if (hi) atomicAdd(lohi + 1, hi);
}

__device__ __forceinline__ u128 warp_sum_u128(u128 x) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)x, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(x >> 64), o);
        x += ((u128)hi << 64) | lo;
    }
    return x;
}

__device__ __forceinline__ int global_warp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int num_warps() { return (gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

}  // namespace dev
}  // namespace gdi
