// Small device helpers used by several CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "mp_internal.cuh"

namespace mpg {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ long long lmod(long long x, long long m) {
    long long r = x % m;
    return r < 0 ? r + m : r;
}

// selection key: |rho|^2 bits in the high word, inverted flat index low
__device__ __forceinline__ unsigned long long make_key(float2 v, unsigned flat) {
    float s = fmaf(v.x, v.x, v.y * v.y);
    return ((unsigned long long)__float_as_uint(s) << 32) |
           (unsigned long long)(0xffffffffu - flat);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o; o >>= 1) k = umax64(k, __shfl_xor_sync(FULL, k, o));
    return k;
}

// warp-wide max Entry (key decides); every lane returns the winner.  The
// 64-bit key is reduced as two 32-bit redux steps (score word, then the
// inverted index among the lanes holding the top score), which is a much
// shorter dependent chain than a shuffle tree.
__device__ __forceinline__ Entry warp_max_entry(Entry e) {
    const unsigned hi = (unsigned)(e.key >> 32), lo = (unsigned)e.key;
    const unsigned mh = __reduce_max_sync(FULL, hi);
    const unsigned ml = __reduce_max_sync(FULL, hi == mh ? lo : 0u);
    const unsigned ball = __ballot_sync(FULL, hi == mh && lo == ml);
    const int src = __ffs(ball) - 1;
    Entry r;
    r.key = ((unsigned long long)mh << 32) | ml;
    r.val.x = __shfl_sync(FULL, e.val.x, src);
    r.val.y = __shfl_sync(FULL, e.val.y, src);
    return r;
}

}  // namespace mpg
