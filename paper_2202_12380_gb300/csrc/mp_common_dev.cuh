// Small device helpers used by several CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "mp_internal.cuh"

namespace mpg {

constexpr unsigned FULL = 0xffffffffu;

// Bounds check of one access (built with -DMP_CHECK_BOUNDS, a substitute for
// a memory sanitizer): true if 0 <= i < n; otherwise the first failing site's
// code is recorded in *err and the caller skips the access.  Without the
// macro it is always true and costs nothing.
__device__ __forceinline__ bool inb(long long i, long long n, int code, int* err) {
#ifdef MP_CHECK_BOUNDS
    if (i >= 0 && i < n) return true;
    atomicCAS(err, 0, code);
    return false;
#else
    (void)i;
    (void)n;
    (void)code;
    (void)err;
    return true;
#endif
}

__device__ __forceinline__ long long lmod(long long x, long long m) {
    long long r = x % m;
    return r < 0 ? r + m : r;
}

// Complex element types of the coefficient planes: float2 (default) or
// double2 (MP_COEF_FP64), with their real type and the plan's tables of
// the same precision.
template <typename C2> struct cx_t;
template <> struct cx_t<float2> {
    using R = float;
    static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
    static __device__ __forceinline__ const float2* gam(const DevPlan& P) { return P.gam; }
    static __device__ __forceinline__ const float2* tiles(const DevPlan& P) { return P.tiles; }
    static __device__ __forceinline__ const float2* cis(const DevPlan& P) { return P.cis; }
};
template <> struct cx_t<double2> {
    using R = double;
    static __device__ __forceinline__ double2 make(double x, double y) {
        return make_double2(x, y);
    }
    static __device__ __forceinline__ const double2* gam(const DevPlan& P) { return P.gam64; }
    static __device__ __forceinline__ const double2* tiles(const DevPlan& P) { return P.tiles64; }
    static __device__ __forceinline__ const double2* cis(const DevPlan& P) { return P.cis64; }
};
template <typename C2> struct plane_tables {
    static __device__ __forceinline__ const C2* gam(const DevPlan& P) { return cx_t<C2>::gam(P); }
};

template <typename C2>
__device__ __forceinline__ C2 gamma_of(const DevDict& D, const C2* gam, int k) {
    if (k < D.gam_lo) return gam[D.gam_off + k];
    if (k >= D.Mr - D.gam_hi) return gam[D.gam_off + D.gam_lo + (k - (D.Mr - D.gam_hi))];
    return cx_t<C2>::make(0, 0);
}

// pedantic selection score (Sec. 5): energy removed by the real pair with
// the coefficient of eq. dualatprod, eq. projenfaster; c^2 at m in {0, M/2}.
// Evaluated in the planes' precision and rounded to FP32 (rounding keeps the
// order); non-negative, so its float bits order like the values.
template <typename C2>
__device__ __forceinline__ float pair_score(C2 v, int m, const DevDict& D, const C2* gam) {
    using R = typename cx_t<C2>::R;
    if (m == 0 || 2 * m == D.M) return (float)(v.x * v.x);
    const C2 g = gamma_of(D, gam, m);
    if (g.x == R(0) && g.y == R(0)) return (float)(R(2) * fma(v.x, v.x, v.y * v.y));
    const R inv = R(1) / (R(1) - fma(g.x, g.x, g.y * g.y));
    const R cx = (v.x - fma(g.x, v.x, g.y * v.y)) * inv;
    const R cy = (v.y - fma(g.y, v.x, -g.x * v.y)) * inv;
    const R c2 = fma(cx, cx, cy * cy), d2 = fma(cx, cx, -cy * cy);
    const R e = R(2) * (c2 + fma(g.x, d2, R(-2) * g.y * cx * cy));
    return (float)(e > R(0) ? e : R(0));
}

// selection key: score bits in the high word (|rho|^2, or the pair energy
// drop when pedantic; FP32, rounded from the planes' precision), inverted
// flat index in the low word
template <typename C2>
__device__ __forceinline__ unsigned long long make_key_sel(C2 v, unsigned flat, int m,
                                                           const DevDict& D, const C2* gam,
                                                           int pedantic) {
    const float s = pedantic ? pair_score(v, m, D, gam) : (float)fma(v.x, v.x, v.y * v.y);
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
