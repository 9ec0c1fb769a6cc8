// Plan construction: cross-Gram kernels, alignment-class tiles, <d, conj d>
// tables and the DFT matrices of the analysis (Sec. 4.1, 4.2, 5).
//
// For dictionaries u (selected atom (k, j)) and v (updated coefficient
// (m, n)) the inner product of eq. GramKern, extended to cross-Gram matrices
// on the common grid a_min = min(a_u, a_v), M_max = max(M_u, M_v), is
//   <d^u_{k,j}, d^v_{m,n}> = e^{i 2 pi k tau / M_u} h_{u,v}(delta, tau),
//   tau = n a_v - j a_u,  delta = m M_max/M_v - k M_max/M_u  (mod M_max),
//   h_{u,v}(delta, tau) = sum_t g_u(t) g_v(t - tau) e^{-i 2 pi delta (t - tau) / M_max}.
// The modulation e^{i 2 pi k tau / M_u} is eq. hkj; it is applied per tile
// column at update time.  Subsampling by M_max/M_v and a_v/a_min (Alg. 3)
// makes only some (delta, tau) reachable from a given (k, j): they depend on
// cf = k mod rf and ct = j mod rt, rf = M_u/M_v if M_u > M_v else 1,
// rt = a_v/a_u if a_v > a_u else 1.  Each such alignment class is stored as
// its own dense tile over the bounding box of the entries with |h| > eps
// (entries at or below eps inside the box are stored as 0), so the update of
// dictionary v is a dense rectangle of its coefficient plane.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mp_internal.cuh"

#include <cudaTypedefs.h>

using namespace mpg;

namespace {

__device__ __forceinline__ long long dmod(long long x, long long m) {
    long long r = x % m;
    return r < 0 ? r + m : r;
}

// e^{-i 2 pi q / M}
__global__ void k_cis_table(double2* cs, int M) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    double s, c;
    sincospi(2.0 * (double)q / (double)M, &s, &c);
    cs[q] = make_double2(c, -s);
}

// e^{+i 2 pi q / M} rounded to FP32 for q < n (modulation of eq. hkj,
// looked up at update time)
__global__ void k_cis32(float2* cs, int n, int M) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s, c;
    sincospi(2.0 * (double)q / (double)M, &s, &c);
    cs[q] = make_float2((float)c, (float)s);
}

// the same table in FP64 (MP_COEF_FP64)
__global__ void k_cis64(double2* cs, int n, int M) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s, c;
    sincospi(2.0 * (double)q / (double)M, &s, &c);
    cs[q] = make_double2(c, s);
}

// h[it][delta] by direct sum over the window overlap (FP64)
__global__ void k_kernel_fp64(const double* __restrict__ gu, int wu, const double* __restrict__ gv,
                              int wv, int Mx, int an, int tmin, int ntau,
                              const double2* __restrict__ cs, double2* __restrict__ h) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ntau * Mx) return;
    int it = (int)(idx / Mx);
    int d = (int)(idx % Mx);
    int tau = tmin + it * an;
    int t0 = max(-wu / 2, tau - wv / 2);
    int t1 = min(wu / 2 - 1, tau + wv / 2 - 1);
    double re = 0.0, im = 0.0;
    long long q = dmod((long long)d * (t0 - tau), Mx);
    for (int t = t0; t <= t1; ++t) {
        double p = gu[t + wu / 2] * gv[t - tau + wv / 2];
        double2 c = cs[q];
        re = fma(p, c.x, re);
        im = fma(p, c.y, im);
        q += d;
        if (q >= Mx) q -= Mx;
    }
    h[idx] = make_double2(re, im);
}

struct ClassGeom {
    int cf, ct;
    int i0, i1;  // candidate row range (delta in (-Mx/2, Mx/2])
    int c0, c1;  // candidate column range (tau inside the kernel support)
};

__device__ __forceinline__ bool kern_at(const double2* h, int Mx, int an, int tmin, int ntau,
                                        long long delta, long long tau, double eps, double2* out) {
    long long off = tau - tmin;
    if (off < 0 || off % an) return false;
    long long it = off / an;
    if (it >= ntau) return false;
    double2 v = h[it * Mx + dmod(delta, Mx)];
    *out = v;
    return sqrt(v.x * v.x + v.y * v.y) > eps;
}

// bounding box of |h| > eps inside one alignment class
__global__ void k_class_bbox(const double2* __restrict__ h, int Mx, int an, int tmin, int ntau,
                             int rf, int av, int au, ClassGeom g, double eps, int* box) {
    int nr = g.i1 - g.i0 + 1, nc = g.c1 - g.c0 + 1;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nr * nc) return;
    int i = g.i0 + (int)(idx % nr);
    int c = g.c0 + (int)(idx / nr);
    long long delta = (long long)i * rf - g.cf;
    long long tau = (long long)c * av - (long long)g.ct * au;
    double2 v;
    if (kern_at(h, Mx, an, tmin, ntau, delta, tau, eps, &v)) {
        atomicMin(&box[0], i);
        atomicMax(&box[1], i);
        atomicMin(&box[2], c);
        atomicMax(&box[3], c);
        atomicAdd(&box[4], 1);
    }
}

__device__ __forceinline__ void put(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void put(double2* p, double2 v) { *p = v; }

// class tile entries, FP32 (T = float2) or FP64 (T = double2)
template <typename T>
__global__ void k_tile_fill(const double2* __restrict__ h, int Mx, int an, int tmin, int ntau,
                            int rf, int av, int au, int cf, int ct, int i_lo, int c_lo, int R,
                            int C, double eps, T* __restrict__ tile) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * C) return;
    int i = (int)(idx % R);
    int c = (int)(idx / R);
    long long delta = (long long)(i_lo + i) * rf - cf;
    long long tau = (long long)(c_lo + c) * av - (long long)ct * au;
    double2 v;
    double2 o = make_double2(0.0, 0.0);
    if (kern_at(h, Mx, an, tmin, ntau, delta, tau, eps, &v)) o = v;
    put(tile + (long long)c * R + i, o);
}

// <d_k, conj d_k> = G((M - k, j), (k, j)) = h_{u,u}(M - 2k, 0), zero when
// thresholded away and for k in {0, M/2} where the partner is missing.
__global__ void k_gamma(const double2* __restrict__ h, int M, int an, int tmin, int ntau,
                        double eps, double2* __restrict__ gam) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > M / 2) return;
    double2 o = make_double2(0.0, 0.0);
    double2 v;
    if (k != 0 && 2 * k != M && kern_at(h, M, an, tmin, ntau, (long long)M - 2 * k, 0, eps, &v))
        o = v;
    gam[k] = o;
}

// analysis matrix: A[2m][i] = g(i) cos(2 pi m t / M), A[2m+1][i] = -g(i) sin(..),
// t = i - w/2, m < M/2 + 1, i < w; all other entries zero.  Shape [Arows][Kp]
// with Arows a multiple of 128 and Kp = w rounded up to 16.
// (T = float for the FP32 analysis, double for MP_COEF_FP64)
template <typename T>
__global__ void k_dft_matrix(const double* __restrict__ g, int w, int Kp, int M, int Mr, int Arows,
                             T* __restrict__ A) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Arows * Kp) return;
    int r = (int)(idx / Kp);
    int i = (int)(idx % Kp);
    int m = r >> 1;
    double o = 0.0;
    if (m < Mr && i < w) {
        long long q = dmod((long long)m * (i - w / 2), M);
        double s, c;
        sincospi(2.0 * (double)q / (double)M, &s, &c);
        o = (r & 1) ? -g[i] * s : g[i] * c;
    }
    A[idx] = (T)o;
}

long long floordiv(long long x, long long d) {
    long long q = x / d;
    if ((x % d != 0) && ((x < 0) != (d < 0))) q -= 1;
    return q;
}
long long ceildiv(long long x, long long d) { return -floordiv(-x, d); }

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            mpg_set_error("%s failed: %s", #call, cudaGetErrorString(e_));            \
            rc = (e_ == cudaErrorMemoryAllocation) ? MP_ENOMEM : MP_ECUDA;            \
            goto fail;                                                                \
        }                                                                             \
    } while (0)

void plan_free(mp_plan* p) {
    if (!p) return;
    for (int w = 0; w < MAXW; ++w) {
        if (p->d_Ahi[w]) cudaFree(p->d_Ahi[w]);
        if (p->d_Alo[w]) cudaFree(p->d_Alo[w]);
    }
    for (int i = 0; i < MAXW * MAXW; ++i)
        if (p->d_kern[i]) cudaFree(p->d_kern[i]);
    for (int w = 0; w < MAXW; ++w) {
        if (p->d_A[w]) cudaFree(p->d_A[w]);
        if (p->d_A64[w]) cudaFree(p->d_A64[w]);
    }
    if (p->d_tiles64) cudaFree(p->d_tiles64);
    if (p->d_gam64) cudaFree(p->d_gam64);
    if (p->d_cis64) cudaFree(p->d_cis64);
    if (p->d_cls) cudaFree(p->d_cls);
    if (p->d_tiles) cudaFree(p->d_tiles);
    if (p->d_gam) cudaFree(p->d_gam);
    if (p->d_g32) cudaFree(p->d_g32);
    if (p->d_cis32) cudaFree(p->d_cis32);
    delete p;
}

}  // namespace

bool mpg::encode_bf16_map(void* map, const void* base, unsigned long long inner,
                          unsigned long long outer, unsigned long long row_bytes,
                          unsigned box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            mpg_set_error("cuTensorMapEncodeTiled is not available");
            return false;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        mpg_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return false;
    }
    return true;
}

extern "C" int mp_plan_create(mp_plan** out, int W, const double* const* windows,
                              const int* win_len, const int* a, const int* M, double kern_thr,
                              unsigned flags, void* cuda_stream) {
    mpg::NvtxRange nvtx_range("mp_plan_create");
    if (!out || W < 1 || W > MAXW || !windows || !win_len || !a || !M) {
        mpg_set_error("mp_plan_create: bad arguments (W must be 1..%d)", MAXW);
        return MP_EINVAL;
    }
    if (!(kern_thr >= 0.0) || !std::isfinite(kern_thr)) {
        mpg_set_error("mp_plan_create: kernel threshold must be finite and >= 0");
        return MP_EINVAL;
    }
    if (flags & ~(unsigned)(MP_ANALYSIS_BF16X3 | MP_PEDANTIC | MP_COEF_FP64)) {
        mpg_set_error("mp_plan_create: unknown flags %u", flags);
        return MP_EINVAL;
    }
    if ((flags & MP_ANALYSIS_BF16X3) && (flags & MP_COEF_FP64)) {
        mpg_set_error("mp_plan_create: MP_COEF_FP64 comes with its own FP64 analysis and cannot "
                      "be combined with MP_ANALYSIS_BF16X3");
        return MP_EINVAL;
    }
    const bool fp64 = (flags & MP_COEF_FP64) != 0;
    for (int w = 0; w < W; ++w) {
        if (!windows[w] || win_len[w] <= 0 || (win_len[w] & 1) || a[w] <= 0 || M[w] <= 0 ||
            (M[w] & 1) || win_len[w] > (1 << 20) || M[w] > (1 << 16)) {
            mpg_set_error("mp_plan_create: dictionary %d: need even w > 0, a > 0, even M > 0", w);
            return MP_EINVAL;
        }
        for (int i = 0; i < win_len[w]; ++i)
            if (!std::isfinite(windows[w][i])) {
                mpg_set_error("mp_plan_create: window %d holds a non-finite value", w);
                return MP_EINVAL;
            }
        if (M[w] % a[w]) {
            mpg_set_error("mp_plan_create: dictionary %d: M/a must be an integer", w);
            return MP_ENOTCOMPAT;
        }
    }
    for (int u = 0; u < W; ++u)
        for (int v = 0; v < W; ++v) {
            int amax = std::max(a[u], a[v]), amin = std::min(a[u], a[v]);
            int Mmax = std::max(M[u], M[v]), Mmin = std::min(M[u], M[v]);
            if (amax % amin || Mmax % Mmin) {
                mpg_set_error("mp_plan_create: dictionaries %d and %d are not compatible "
                              "(a must divide pairwise, M must divide pairwise)", u, v);
                return MP_ENOTCOMPAT;
            }
        }

    if (flags & MP_ANALYSIS_BF16X3)
        for (int w = 0; w < W; ++w)
            if (a[w] % 64 || (win_len[w] / 2) % a[w]) {
                mpg_set_error("mp_plan_create: the split-BF16 analysis needs every a to be a "
                              "multiple of 64 and every w/2 a multiple of a (dictionary %d)", w);
                return MP_EINVAL;
            }
    int rc = MP_OK;
    mp_plan* p = new mp_plan();
    memset(p->d_kern, 0, sizeof(p->d_kern));
    memset(p->d_A, 0, sizeof(p->d_A));
    memset(p->d_Ahi, 0, sizeof(p->d_Ahi));
    memset(p->d_Alo, 0, sizeof(p->d_Alo));
    memset(p->d_A64, 0, sizeof(p->d_A64));
    p->d_tiles64 = nullptr;
    p->d_gam64 = nullptr;
    p->d_cis64 = nullptr;
    p->d_cls = nullptr;
    p->d_tiles = nullptr;
    p->d_gam = nullptr;
    p->d_g32 = nullptr;
    p->d_cis32 = nullptr;
    p->W = W;
    p->eps = kern_thr;
    p->flags = flags;
    p->stream = (cudaStream_t)cuda_stream;
    memset(&p->dp, 0, sizeof(p->dp));
    p->dp.W = W;
    cudaStream_t st = p->stream;
    std::vector<double*> d_win(W, nullptr);
    std::vector<double2*> d_cis(W, nullptr);
    int* d_box = nullptr;
    {
        CK(cudaGetDevice(&p->device));
        CK(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
        int g_total = 0;
        for (int w = 0; w < W; ++w) {
            p->wlen[w] = win_len[w];
            p->a[w] = a[w];
            p->M[w] = M[w];
            DevDict& D = p->dp.d[w];
            D.wlen = win_len[w];
            D.a = a[w];
            D.M = M[w];
            D.Mr = M[w] / 2 + 1;
            D.nch = (D.Mr + CHUNK - 1) / CHUNK;
            D.Mrp = D.nch * CHUNK;
            D.msh = 0;
            while ((1 << D.msh) < D.Mr) ++D.msh;
            D.Mmask = (M[w] & (M[w] - 1)) == 0 ? M[w] - 1 : 0;
            D.g_off = g_total;
            g_total += win_len[w];
            CK(cudaMalloc(&d_win[w], sizeof(double) * win_len[w]));
            CK(cudaMemcpyAsync(d_win[w], windows[w], sizeof(double) * win_len[w],
                               cudaMemcpyHostToDevice, st));
        }
        // FP32 copy of the windows (synthesis)
        {
            std::vector<float> g32(g_total);
            for (int w = 0; w < W; ++w)
                for (int i = 0; i < win_len[w]; ++i)
                    g32[p->dp.d[w].g_off + i] = (float)windows[w][i];
            CK(cudaMalloc(&p->d_g32, sizeof(float) * g_total));
            CK(cudaMemcpyAsync(p->d_g32, g32.data(), sizeof(float) * g_total,
                               cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
        }
        // FP32 modulation tables, one per dictionary
        {
            int tot = 0;
            for (int w = 0; w < W; ++w) {
                DevDict& D = p->dp.d[w];
                D.cis_off = tot;
                D.cis_q = (M[w] % 4 == 0) ? M[w] / 4 : 0;
                D.cis_qsh = -1;
                for (int b = 0; b < 31; ++b)
                    if (D.cis_q == (1 << b)) D.cis_qsh = b;
                tot += D.cis_q ? D.cis_q : M[w];
            }
            p->dp.ncis = tot;
            CK(cudaMalloc(&p->d_cis32, sizeof(float2) * tot));
            if (fp64) CK(cudaMalloc(&p->d_cis64, sizeof(double2) * tot));
            for (int w = 0; w < W; ++w) {
                const int n = p->dp.d[w].cis_q ? p->dp.d[w].cis_q : M[w];
                k_cis32<<<(n + 255) / 256, 256, 0, st>>>(p->d_cis32 + p->dp.d[w].cis_off, n, M[w]);
                CK(cudaGetLastError());
                if (fp64) {
                    k_cis64<<<(n + 255) / 256, 256, 0, st>>>(p->d_cis64 + p->dp.d[w].cis_off, n,
                                                              M[w]);
                    CK(cudaGetLastError());
                }
            }
        }
        // cis tables per distinct M_max
        int Mmax_all = 0;
        for (int w = 0; w < W; ++w) Mmax_all = std::max(Mmax_all, M[w]);
        for (int w = 0; w < W; ++w) {
            CK(cudaMalloc(&d_cis[w], sizeof(double2) * M[w]));
            k_cis_table<<<(M[w] + 255) / 256, 256, 0, st>>>(d_cis[w], M[w]);
            CK(cudaGetLastError());
        }
        // kernels of all ordered pairs
        for (int u = 0; u < W; ++u)
            for (int v = 0; v < W; ++v) {
                int pi = u * W + v;
                int an = std::min(a[u], a[v]);
                int Mx = std::max(M[u], M[v]);
                int wu = win_len[u], wv = win_len[v];
                long long lo = -wu / 2 - wv / 2 + 1, hi = wu / 2 - 1 + wv / 2;
                int tmin = (int)(ceildiv(lo, an) * an);
                int tmax = (int)(floordiv(hi, an) * an);
                p->Mx[pi] = Mx;
                p->an[pi] = an;
                p->tmin[pi] = tmin;
                p->ntau[pi] = (tmax - tmin) / an + 1;
                long long n = (long long)p->ntau[pi] * Mx;
                CK(cudaMalloc(&p->d_kern[pi], sizeof(double2) * n));
                int wM = (M[u] >= M[v]) ? u : v;  // table of size M_max
                k_kernel_fp64<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
                    d_win[u], wu, d_win[v], wv, Mx, an, tmin, p->ntau[pi], d_cis[wM],
                    p->d_kern[pi]);
                CK(cudaGetLastError());
            }
        CK(cudaMalloc(&d_box, sizeof(int) * 5));
        // alignment classes: bounding boxes
        long long tiles_total = 0;
        for (int u = 0; u < W; ++u)
            for (int v = 0; v < W; ++v) {
                int pi = u * W + v;
                DevPair& PR = p->dp.p[pi];
                PR.rf = (M[u] > M[v]) ? M[u] / M[v] : 1;
                PR.rt = (a[v] > a[u]) ? a[v] / a[u] : 1;
                PR.cls_base = (int)p->cls.size();
                PR.rf_sh = -1;
                PR.rt_sh = -1;
                for (int b = 0; b < 31; ++b) {
                    if ((1 << b) == PR.rf) PR.rf_sh = b;
                    if ((1 << b) == PR.rt) PR.rt_sh = b;
                }
                PR.mratio = M[v] >= M[u] ? M[v] / M[u] : 0;
                PR.aratio = a[v] <= a[u] ? a[u] / a[v] : 0;
                int Mx = p->Mx[pi], an = p->an[pi], tmin = p->tmin[pi], ntau = p->ntau[pi];
                int tmax = tmin + (ntau - 1) * an;
                for (int cf = 0; cf < PR.rf; ++cf)
                    for (int ct = 0; ct < PR.rt; ++ct) {
                        ClassGeom g;
                        g.cf = cf;
                        g.ct = ct;
                        // delta = i rf - cf in (-Mx/2, Mx/2]
                        g.i0 = (int)ceildiv(-(long long)Mx / 2 + 1 + cf, PR.rf);
                        g.i1 = (int)floordiv((long long)Mx / 2 + cf, PR.rf);
                        // tau = c a_v - ct a_u in [tmin, tmax]
                        g.c0 = (int)ceildiv((long long)tmin + (long long)ct * a[u], a[v]);
                        g.c1 = (int)floordiv((long long)tmax + (long long)ct * a[u], a[v]);
                        int box_init[5] = {INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN, 0};
                        CK(cudaMemcpyAsync(d_box, box_init, sizeof(box_init),
                                           cudaMemcpyHostToDevice, st));
                        DevClass C;
                        C.off = 0;
                        C.R = C.C = 0;
                        C.i_lo = C.c_lo = 0;
                        int nnz = 0;
                        if (g.i1 >= g.i0 && g.c1 >= g.c0) {
                            long long n = (long long)(g.i1 - g.i0 + 1) * (g.c1 - g.c0 + 1);
                            k_class_bbox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                                p->d_kern[pi], Mx, an, tmin, ntau, PR.rf, a[v], a[u], g, kern_thr,
                                d_box);
                            CK(cudaGetLastError());
                            int box[5];
                            CK(cudaMemcpyAsync(box, d_box, sizeof(box), cudaMemcpyDeviceToHost,
                                               st));
                            CK(cudaStreamSynchronize(st));
                            nnz = box[4];
                            if (nnz > 0) {
                                C.i_lo = box[0];
                                C.R = box[1] - box[0] + 1;
                                C.c_lo = box[2];
                                C.C = box[3] - box[2] + 1;
                                C.off = tiles_total;
                                tiles_total += (long long)C.R * C.C;
                            }
                        }
                        p->cls.push_back(C);
                        p->cls_nnz.push_back(nnz);
                    }
            }
        p->tiles_len = tiles_total;
        p->dp.tiles_len = tiles_total;
        CK(cudaMalloc(&p->d_tiles, sizeof(float2) * std::max(tiles_total, 1LL)));
        if (fp64) CK(cudaMalloc(&p->d_tiles64, sizeof(double2) * std::max(tiles_total, 1LL)));
        for (int u = 0; u < W; ++u)
            for (int v = 0; v < W; ++v) {
                int pi = u * W + v;
                const DevPair& PR = p->dp.p[pi];
                for (int cf = 0; cf < PR.rf; ++cf)
                    for (int ct = 0; ct < PR.rt; ++ct) {
                        const DevClass& C = p->cls[PR.cls_base + cf * PR.rt + ct];
                        long long n = (long long)C.R * C.C;
                        if (n == 0) continue;
                        k_tile_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                            p->d_kern[pi], p->Mx[pi], p->an[pi], p->tmin[pi], p->ntau[pi], PR.rf,
                            a[v], a[u], cf, ct, C.i_lo, C.c_lo, C.R, C.C, kern_thr,
                            p->d_tiles + C.off);
                        CK(cudaGetLastError());
                        if (fp64) {
                            k_tile_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                                p->d_kern[pi], p->Mx[pi], p->an[pi], p->tmin[pi], p->ntau[pi],
                                PR.rf, a[v], a[u], cf, ct, C.i_lo, C.c_lo, C.R, C.C, kern_thr,
                                p->d_tiles64 + C.off);
                            CK(cudaGetLastError());
                        }
                    }
            }
        CK(cudaMalloc(&p->d_cls, sizeof(DevClass) * std::max<size_t>(p->cls.size(), 1)));
        CK(cudaMemcpyAsync(p->d_cls, p->cls.data(), sizeof(DevClass) * p->cls.size(),
                           cudaMemcpyHostToDevice, st));
        // <d, conj d>: full tables, then a compact copy holding only the
        // frequencies near 0 and M/2 where it can be nonzero
        std::vector<float2> gam_compact;
        std::vector<double2> gam_compact64;
        for (int u = 0; u < W; ++u) {
            int pi = u * W + u;
            int Mr = M[u] / 2 + 1;
            double2* d_g = nullptr;
            CK(cudaMalloc(&d_g, sizeof(double2) * Mr));
            k_gamma<<<(Mr + 255) / 256, 256, 0, st>>>(p->d_kern[pi], M[u], p->an[pi],
                                                       p->tmin[pi], p->ntau[pi], kern_thr, d_g);
            cudaError_t e1 = cudaGetLastError();
            std::vector<double2> hg64(Mr);
            std::vector<float2> hg(Mr);
            cudaError_t e2 = cudaMemcpyAsync(hg64.data(), d_g, sizeof(double2) * Mr,
                                             cudaMemcpyDeviceToHost, st);
            cudaError_t e3 = cudaStreamSynchronize(st);
            cudaFree(d_g);
            CK(e1);
            CK(e2);
            CK(e3);
            for (int k = 0; k < Mr; ++k)
                hg[k] = make_float2((float)hg64[k].x, (float)hg64[k].y);
            p->gam_full[u].resize(2 * Mr);
            for (int k = 0; k < Mr; ++k) {
                p->gam_full[u][2 * k] = hg[k].x;
                p->gam_full[u][2 * k + 1] = hg[k].y;
            }
            // lo part: k < gam_lo; hi part: k > M/2 - gam_hi; zero in between
            int half = Mr / 2;
            int lo = 0, hi = 0;
            for (int k = 0; k <= half; ++k)
                if (hg64[k].x != 0.0 || hg64[k].y != 0.0) lo = k + 1;
            for (int k = Mr - 1; k > half; --k)
                if (hg64[k].x != 0.0 || hg64[k].y != 0.0) hi = std::max(hi, Mr - k);
            DevDict& D = p->dp.d[u];
            D.gam_lo = lo;
            D.gam_hi = hi;
            D.gam_off = (int)gam_compact.size();
            for (int k = 0; k < lo; ++k) gam_compact.push_back(hg[k]);
            for (int k = Mr - hi; k < Mr; ++k) gam_compact.push_back(hg[k]);
            for (int k = 0; k < lo; ++k) gam_compact64.push_back(hg64[k]);
            for (int k = Mr - hi; k < Mr; ++k) gam_compact64.push_back(hg64[k]);
        }
        CK(cudaMalloc(&p->d_gam, sizeof(float2) * std::max<size_t>(gam_compact.size(), 1)));
        if (!gam_compact.empty())
            CK(cudaMemcpyAsync(p->d_gam, gam_compact.data(), sizeof(float2) * gam_compact.size(),
                               cudaMemcpyHostToDevice, st));
        if (fp64) {
            CK(cudaMalloc(&p->d_gam64,
                          sizeof(double2) * std::max<size_t>(gam_compact64.size(), 1)));
            if (!gam_compact64.empty())
                CK(cudaMemcpyAsync(p->d_gam64, gam_compact64.data(),
                                   sizeof(double2) * gam_compact64.size(), cudaMemcpyHostToDevice,
                                   st));
            // the host vector is read by the copy: wait for it before it goes
            CK(cudaStreamSynchronize(st));
        }
        // analysis matrices
        for (int w = 0; w < W; ++w) {
            const DevDict& D = p->dp.d[w];
            int rows = ((2 * D.Mrp + 127) / 128) * 128;
            int kp = ((D.wlen + 15) / 16) * 16;
            p->Arows[w] = rows;
            p->Akp[w] = kp;
            long long n = (long long)rows * kp;
            CK(cudaMalloc(&p->d_A[w], sizeof(float) * n));
            k_dft_matrix<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_win[w], D.wlen, kp, D.M,
                                                                       D.Mr, rows, p->d_A[w]);
            CK(cudaGetLastError());
            if (fp64) {
                CK(cudaMalloc(&p->d_A64[w], sizeof(double) * n));
                k_dft_matrix<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                    d_win[w], D.wlen, kp, D.M, D.Mr, rows, p->d_A64[w]);
                CK(cudaGetLastError());
            }
        }
        // split-BF16 operands and their tensor maps
        if (flags & MP_ANALYSIS_BF16X3)
            for (int w = 0; w < W; ++w) {
                const int kp = ((p->dp.d[w].wlen + 63) / 64) * 64;
                p->Kp64[w] = kp;
                const size_t bytes = (size_t)p->Arows[w] * kp * 2;
                CK(cudaMalloc(&p->d_Ahi[w], bytes));
                CK(cudaMalloc(&p->d_Alo[w], bytes));
                CK(launch_split_rows(p->d_A[w], p->Arows[w], p->dp.d[w].wlen, p->Akp[w], kp,
                                     p->d_Ahi[w], p->d_Alo[w], st));
                if (!encode_bf16_map(p->tmA[w][0], p->d_Ahi[w], kp, p->Arows[w], (size_t)kp * 2) ||
                    !encode_bf16_map(p->tmA[w][1], p->d_Alo[w], kp, p->Arows[w], (size_t)kp * 2)) {
                    rc = MP_ECUDA;
                    goto fail;
                }
            }
        CK(cudaStreamSynchronize(st));
        p->dp.cls = p->d_cls;
        p->dp.ncls = (int)p->cls.size();
        p->dp.ngam = (int)gam_compact.size();
        p->dp.tiles = p->d_tiles;
        p->dp.gam = p->d_gam;
        p->dp.g32 = p->d_g32;
        p->dp.cis = p->d_cis32;
        p->dp.fp64 = fp64 ? 1 : 0;
        p->dp.tiles64 = p->d_tiles64;
        p->dp.gam64 = p->d_gam64;
        p->dp.cis64 = p->d_cis64;
        p->dp.pedantic = (flags & MP_PEDANTIC) ? 1 : 0;
        p->dp.pow2 = 1;
        for (int w = 0; w < W; ++w)
            if ((M[w] & (M[w] - 1)) || (a[w] & (a[w] - 1))) p->dp.pow2 = 0;
    }
    for (int w = 0; w < W; ++w) {
        cudaFree(d_win[w]);
        cudaFree(d_cis[w]);
    }
    cudaFree(d_box);
    *out = p;
    return MP_OK;
fail:
    cudaStreamSynchronize(st);
    for (int w = 0; w < W; ++w) {
        if (d_win[w]) cudaFree(d_win[w]);
        if (d_cis[w]) cudaFree(d_cis[w]);
    }
    if (d_box) cudaFree(d_box);
    plan_free(p);
    return rc;
}

extern "C" void mp_plan_destroy(mp_plan* plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    plan_free(plan);
}

static int check_pair(const mp_plan* p, int u, int v) {
    if (!p || u < 0 || v < 0 || u >= p->W || v >= p->W) {
        mpg_set_error("bad plan or dictionary index");
        return MP_EINVAL;
    }
    return MP_OK;
}

extern "C" int mp_plan_kernel_dims(const mp_plan* p, int u, int v, int* Mx, int* an, int* tmin,
                                   int* ntau) {
    int rc = check_pair(p, u, v);
    if (rc) return rc;
    int pi = u * p->W + v;
    if (Mx) *Mx = p->Mx[pi];
    if (an) *an = p->an[pi];
    if (tmin) *tmin = p->tmin[pi];
    if (ntau) *ntau = p->ntau[pi];
    return MP_OK;
}

extern "C" int mp_plan_kernel_fp64(const mp_plan* p, int u, int v, double* h, int64_t cap) {
    int rc = check_pair(p, u, v);
    if (rc) return rc;
    int pi = u * p->W + v;
    long long n = (long long)p->ntau[pi] * p->Mx[pi];
    if (!h || cap < 2 * n) {
        mpg_set_error("mp_plan_kernel_fp64: buffer too small (%lld doubles needed)", 2 * n);
        return MP_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(h, p->d_kern[pi], sizeof(double2) * n, cudaMemcpyDeviceToHost,
                                    p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        mpg_set_error("mp_plan_kernel_fp64: %s", cudaGetErrorString(e));
        return MP_ECUDA;
    }
    return MP_OK;
}

static const DevClass* find_class(const mp_plan* p, int u, int v, int cf, int ct, int* idx) {
    const DevPair& PR = p->dp.p[u * p->W + v];
    if (cf < 0 || ct < 0 || cf >= PR.rf || ct >= PR.rt) return nullptr;
    *idx = PR.cls_base + cf * PR.rt + ct;
    return &p->cls[*idx];
}

extern "C" int mp_plan_tile_info(const mp_plan* p, int u, int v, int cf, int ct, int* info) {
    int rc = check_pair(p, u, v);
    if (rc) return rc;
    int idx;
    const DevClass* C = find_class(p, u, v, cf, ct, &idx);
    if (!C || !info) {
        mpg_set_error("mp_plan_tile_info: bad class index");
        return MP_EINVAL;
    }
    const DevPair& PR = p->dp.p[u * p->W + v];
    info[0] = PR.rf;
    info[1] = PR.rt;
    info[2] = C->R;
    info[3] = C->C;
    info[4] = C->i_lo;
    info[5] = C->c_lo;
    info[6] = p->cls_nnz[idx];
    return MP_OK;
}

extern "C" int mp_plan_tile(const mp_plan* p, int u, int v, int cf, int ct, float* out,
                            int64_t cap) {
    int rc = check_pair(p, u, v);
    if (rc) return rc;
    int idx;
    const DevClass* C = find_class(p, u, v, cf, ct, &idx);
    if (!C) {
        mpg_set_error("mp_plan_tile: bad class index");
        return MP_EINVAL;
    }
    long long n = (long long)C->R * C->C;
    if (n == 0) return MP_OK;
    if (!out || cap < 2 * n) {
        mpg_set_error("mp_plan_tile: buffer too small");
        return MP_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(out, p->d_tiles + C->off, sizeof(float2) * n,
                                    cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        mpg_set_error("mp_plan_tile: %s", cudaGetErrorString(e));
        return MP_ECUDA;
    }
    return MP_OK;
}

extern "C" int mp_plan_gamma(const mp_plan* p, int u, float* out, int64_t cap) {
    int rc = check_pair(p, u, u);
    if (rc) return rc;
    const std::vector<float>& g = p->gam_full[u];
    if (!out || cap < (int64_t)g.size()) {
        mpg_set_error("mp_plan_gamma: buffer too small");
        return MP_EINVAL;
    }
    memcpy(out, g.data(), sizeof(float) * g.size());
    return MP_OK;
}
