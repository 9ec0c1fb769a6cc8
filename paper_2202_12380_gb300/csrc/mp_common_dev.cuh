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

__device__ __forceinline__ float2 gamma_of(const DevDict& D, const float2* gam, int k) {
    if (k < D.gam_lo) return gam[D.gam_off + k];
    if (k >= D.Mr - D.gam_hi) return gam[D.gam_off + D.gam_lo + (k - (D.Mr - D.gam_hi))];
    return make_float2(0.f, 0.f);
}

// pedantic selection score (Sec. 5): energy removed by the real pair with
// the coefficient of eq. dualatprod, eq. projenfaster; c^2 at m in {0, M/2}.
// Non-negative, so its float bits order like the values.
__device__ __forceinline__ float pair_score(float2 v, int m, const DevDict& D, const float2* gam) {
    if (m == 0 || 2 * m == D.M) return v.x * v.x;
    const float2 g = gamma_of(D, gam, m);
    if (g.x == 0.f && g.y == 0.f) return 2.f * fmaf(v.x, v.x, v.y * v.y);
    const float inv = 1.f / (1.f - fmaf(g.x, g.x, g.y * g.y));
    const float cx = (v.x - fmaf(g.x, v.x, g.y * v.y)) * inv;
    const float cy = (v.y - fmaf(g.y, v.x, -g.x * v.y)) * inv;
    const float c2 = fmaf(cx, cx, cy * cy), d2 = fmaf(cx, cx, -cy * cy);
    return fmaxf(0.f, 2.f * (c2 + fmaf(g.x, d2, -2.f * g.y * cx * cy)));
}

// selection key: score bits in the high word (|rho|^2, or the pair energy
// drop when pedantic), inverted flat index in the low word
__device__ __forceinline__ unsigned long long make_key_sel(float2 v, unsigned flat, int m,
                                                           const DevDict& D, const float2* gam,
                                                           int pedantic) {
    const float s = pedantic ? pair_score(v, m, D, gam) : fmaf(v.x, v.x, v.y * v.y);
    return ((unsigned long long)__float_as_uint(s) << 32) |
           (unsigned long long)(0xffffffffu - flat);
}

// warp-wide max key; every lane returns it.  The 64-bit key is reduced as
// two 32-bit redux steps (score word, then the inverted index among the
// lanes holding the top score).
__device__ __forceinline__ Key warp_max_key(Key k) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mh = __reduce_max_sync(FULL, hi);
    const unsigned ml = __reduce_max_sync(FULL, hi == mh ? lo : 0u);
    return ((Key)mh << 32) | ml;
}

// two warp-wide max reductions run side by side (independent chains)
__device__ __forceinline__ void warp_max_key2(Key& a, Key& b) {
    const unsigned ha = (unsigned)(a >> 32), la = (unsigned)a;
    const unsigned hb = (unsigned)(b >> 32), lb = (unsigned)b;
    const unsigned mha = __reduce_max_sync(FULL, ha);
    const unsigned mhb = __reduce_max_sync(FULL, hb);
    const unsigned mla = __reduce_max_sync(FULL, ha == mha ? la : 0u);
    const unsigned mlb = __reduce_max_sync(FULL, hb == mhb ? lb : 0u);
    a = ((Key)mha << 32) | mla;
    b = ((Key)mhb << 32) | mlb;
}

}  // namespace mpg
