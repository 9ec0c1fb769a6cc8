// Analysis (Alg. 1 initialisation, Sec. 5): rho_0 = D_w^* x for every
// dictionary of every signal, E_0 = ||x||^2, and the max trees.
//
// The reduced DGT
//   rho(m, n) = sum_{i=0}^{w-1} x((n a + i - w/2) mod L) g(i) e^{-i 2 pi m (i - w/2) / M}
// is one real GEMM per dictionary: C = A B with A[2m + {0,1}][i] the
// windowed cosine / negated sine rows (built by the plan) and B[i][n] =
// x(n a + i - w/2) the frames, gathered on the fly from the signal (no
// framed copy is materialised).  The SIMT path below runs it with register
// blocking in FP32 (float2 planes) or, for MP_COEF_FP64 plans, in FP64
// (double2 planes); the epilogue writes complex rows of the frame-major
// coefficient plane directly.
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int BM = 128, BN = 64, BK = 16;

// locate the signal owning a global tile index
__device__ __forceinline__ int find_sig(const long long* prefix, int nsig, long long t) {
    int lo = 0, hi = nsig - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// eight consecutive matrix entries (k .. k + 7 of one row)
__device__ __forceinline__ void load8(const float* p, float o[8]) {
    const float4 a0 = *reinterpret_cast<const float4*>(p);
    const float4 a1 = *reinterpret_cast<const float4*>(p + 4);
    o[0] = a0.x; o[1] = a0.y; o[2] = a0.z; o[3] = a0.w;
    o[4] = a1.x; o[5] = a1.y; o[6] = a1.z; o[7] = a1.w;
}
__device__ __forceinline__ void load8(const double* p, double o[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double2 v = reinterpret_cast<const double2*>(p)[q];
        o[2 * q] = v.x;
        o[2 * q + 1] = v.y;
    }
}

// shared-memory reads of the inner product: 8 rows and 4 frames (vector loads)
__device__ __forceinline__ void lds84(const float* a, const float* b, float r8[8], float c4[4]) {
    const float4 x0 = *reinterpret_cast<const float4*>(a);
    const float4 x1 = *reinterpret_cast<const float4*>(a + 4);
    const float4 y0 = *reinterpret_cast<const float4*>(b);
    r8[0] = x0.x; r8[1] = x0.y; r8[2] = x0.z; r8[3] = x0.w;
    r8[4] = x1.x; r8[5] = x1.y; r8[6] = x1.z; r8[7] = x1.w;
    c4[0] = y0.x; c4[1] = y0.y; c4[2] = y0.z; c4[3] = y0.w;
}
__device__ __forceinline__ void lds84(const double* a, const double* b, double r8[8],
                                      double c4[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double2 x = reinterpret_cast<const double2*>(a)[q];
        r8[2 * q] = x.x;
        r8[2 * q + 1] = x.y;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const double2 y = reinterpret_cast<const double2*>(b)[q];
        c4[2 * q] = y.x;
        c4[2 * q + 1] = y.y;
    }
}

// four bins (re, im pairs) of one frame into the plane
__device__ __forceinline__ void store4(float2* dst, const float v[8], int left) {
    if (left >= 4) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        for (int b = 0; b < left; ++b) dst[b] = make_float2(v[2 * b], v[2 * b + 1]);
    }
}
__device__ __forceinline__ void store4(double2* dst, const double v[8], int left) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (b < left) dst[b] = make_double2(v[2 * b], v[2 * b + 1]);
}

template <typename T, typename C2>
__global__ void __launch_bounds__(256) k_analysis_gemm(const T* __restrict__ A, int Kp, int w,
                                                       int a, int Mrp, int nsig,
                                                       const long long* __restrict__ tprefix,
                                                       const DevSig* __restrict__ sigs, int dict,
                                                       int flagged) {
    __shared__ __align__(16) T As[BK][BM];
    __shared__ __align__(16) T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long gt = blockIdx.x;
    const int s = find_sig(tprefix, nsig, gt);
    const DevSig& S = sigs[s];
    if (flagged && !S.reanalyze) return;
    const long long N = S.N[dict];
    const long long L = S.L;
    const float* __restrict__ x = S.use_r ? S.r : S.x;
    const long long n0 = (gt - tprefix[s]) * BN;
    const int r0 = blockIdx.y * BM;

    T acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    // A tile loader: row r0 + (tid >> 1), 8 consecutive k from (tid & 1) * 8
    const int ar = tid >> 1, ak = (tid & 1) * 8;
    const T* Arow = A + (long long)(r0 + ar) * Kp;
    // B tile loader: k = tid & 15, frames (tid >> 4) + 16 q
    const int bk = tid & 15, bn = tid >> 4;

    for (int k0 = 0; k0 < Kp; k0 += BK) {
        T a8[8];
        load8(Arow + k0 + ak, a8);
        T bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long n = n0 + bn + 16 * q;
            int i = k0 + bk;
            T v = T(0);
            if (n < N && i < w) v = (T)__ldg(x + lmod(n * a + i - w / 2, L));
            bv[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) As[ak + q][ar] = a8[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) Bs[bk][bn + 16 * q] = bv[q];
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ar8[8], bc4[4];
            lds84(&As[kk][ty * 8], &Bs[kk][tx * 4], ar8, bc4);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(ar8[i], bc4[j], acc[i][j]);
        }
    }
    // epilogue: rows ty*8 .. +7 are bins (r0 + ty*8)/2 .. +3 (re, im pairs)
    const int m0 = (r0 + ty * 8) >> 1;
    C2* plane = reinterpret_cast<C2*>(S.plane[dict]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        long long n = n0 + tx * 4 + j;
        if (n >= N) continue;
        const T v[8] = {acc[0][j], acc[1][j], acc[2][j], acc[3][j],
                        acc[4][j], acc[5][j], acc[6][j], acc[7][j]};
        store4(plane + n * Mrp + m0, v, Mrp - m0);
    }
}

// FP64 squared norms of whole signals, spread over the GPU: each signal is
// cut into ENERGY_PARTS equal segments, one block per segment writes its
// partial sum, and one warp per signal adds the partials; every step has a
// fixed order, so the result does not depend on scheduling.  (The FP64 pipe
// of this part is narrow: one block per signal took 0.58 ms for 2^20
// samples.)
//   RESID = false: E_0 = ||x||^2 at the start of a decomposition;
//   RESID = true:  reset pass (Alg. 2) of the flagged signals, r = x - y and
//                  E = E_out = ||r||^2.

// sum over the block (256 threads), fixed order; valid in thread 0
__device__ __forceinline__ double block_sum256(double acc) {
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double v = 0.0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < 8; ++i) v += red[i];
    return v;
}

template <bool RESID>
__global__ void __launch_bounds__(256) k_sqnorm_part(DevSig* sigs, double* __restrict__ part) {
    DevSig& S = sigs[blockIdx.y];
    if (RESID && !S.reanalyze) return;
    const long long per = (S.L + ENERGY_PARTS - 1) / ENERGY_PARTS;
    const long long l0 = (long long)blockIdx.x * per;
    const long long l1 = l0 + per < S.L ? l0 + per : S.L;
    double acc = 0.0;
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
        double v;
        if (RESID) {
            const float d = S.x[l] - S.y[l];
            S.r[l] = d;
            v = (double)d;
        } else {
            v = (double)S.x[l];
        }
        acc = fma(v, v, acc);
    }
    acc = block_sum256(acc);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * ENERGY_PARTS + blockIdx.x] = acc;
}

template <bool RESID>
__global__ void k_sqnorm_final(DevSig* sigs, int nsig, const double* __restrict__ part) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= nsig) return;
    DevSig& S = sigs[s];
    if (RESID && !S.reanalyze) return;
    static_assert(ENERGY_PARTS == 64, "two partials per lane");
    double v = part[(size_t)s * ENERGY_PARTS + lane] + part[(size_t)s * ENERGY_PARTS + 32 + lane];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (lane) return;
    if (RESID) {
        S.E = v;
        S.E_out = v;
        S.k_out = S.k;
        S.reset_pending = 0;
        S.use_r = 1;
    } else {
        S.E0 = v;
        S.E = v;
        S.k = 0;
        S.stop = 0;
        S.timed_out = 0;
        S.k_out = 0;
        S.E_out = v;
        S.reset_pending = 0;
        S.reanalyze = 0;
        S.use_r = 0;
    }
}

// copy of up to GATHER_MAX signals (device to device) in one launch: block
// row y copies signal y, 16-byte accesses when both ends are 16-byte aligned
__global__ void __launch_bounds__(256) k_gather_signals(GatherArgs g) {
    const int b = blockIdx.y;
    const float* __restrict__ src = g.src[b];
    float* __restrict__ dst = g.dst[b];
    const long long n = g.len[b];
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (((reinterpret_cast<size_t>(src) | reinterpret_cast<size_t>(dst)) & 15) == 0) {
        const long long n4 = n >> 2;
        for (long long i = i0; i < n4; i += step)
            reinterpret_cast<float4*>(dst)[i] = __ldg(reinterpret_cast<const float4*>(src) + i);
        done = n4 << 2;
    }
    for (long long i = done + i0; i < n; i += step) dst[i] = src[i];
}

// level 0 (per 32-bin chunk) and level 1 (per frame) of dictionary `dict`,
// one warp per frame (C2: float2 or double2 planes)
template <typename C2>
__global__ void k_tree_build(DevPlan P, const DevSig* __restrict__ sigs, int nsig,
                             const long long* __restrict__ fprefix, long long total, int dict,
                             int flagged) {
    long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= total) return;
    const int lane = threadIdx.x & 31;
    const int s = find_sig(fprefix, nsig, gw);
    const DevSig& S = sigs[s];
    if (flagged && !S.reanalyze) return;
    const long long n = gw - fprefix[s];
    const DevDict& D = P.d[dict];
    const C2* row = reinterpret_cast<const C2*>(S.plane[dict]) + n * D.Mrp;
    const C2* gam = plane_tables<C2>::gam(P);
    Key* l0 = S.l0[dict] + n * D.nch;
    const unsigned fb = S.fbase[dict] + ((unsigned)n << D.msh);
    Key best = 0ull;
    // four chunks' loads in flight per warp (one at a time left the planes'
    // read at about a third of the HBM bandwidth)
    constexpr int U = 4;
    for (int ch0 = 0; ch0 < D.nch; ch0 += U) {
        C2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (ch0 + u < D.nch) v[u] = row[(ch0 + u) * CHUNK + lane];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (ch0 + u >= D.nch) break;
            const int m = (ch0 + u) * CHUNK + lane;
            const Key k = (m < D.Mr) ? make_key_sel(v[u], fb + m, m, D, gam, P.pedantic) : 0ull;
            const Key r = warp_max_key(k);
            if (lane == 0) l0[ch0 + u] = r;
            best = r > best ? r : best;
        }
    }
    if (lane == 0) S.l1[dict][n] = best;
}

}  // namespace

cudaError_t launch_analysis_sgemm(const float* A, int Arows, int Kp, int w_len, int a, int Mrp,
                                  int nsig, const long long* d_tile_prefix, const DevSig* d_sigs,
                                  int dict, long long total_frame_tiles, cudaStream_t st,
                                  int flagged) {
    if (total_frame_tiles <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_frame_tiles, (unsigned)(Arows / BM));
    k_analysis_gemm<float, float2><<<grid, 256, 0, st>>>(A, Kp, w_len, a, Mrp, nsig,
                                                         d_tile_prefix, d_sigs, dict, flagged);
    return cudaGetLastError();
}

cudaError_t launch_analysis_dgemm(const double* A, int Arows, int Kp, int w_len, int a, int Mrp,
                                  int nsig, const long long* d_tile_prefix, const DevSig* d_sigs,
                                  int dict, long long total_frame_tiles, cudaStream_t st,
                                  int flagged) {
    if (total_frame_tiles <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_frame_tiles, (unsigned)(Arows / BM));
    k_analysis_gemm<double, double2><<<grid, 256, 0, st>>>(A, Kp, w_len, a, Mrp, nsig,
                                                           d_tile_prefix, d_sigs, dict, flagged);
    return cudaGetLastError();
}

cudaError_t launch_gather_signals(const GatherArgs& g, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > GATHER_MAX) return cudaErrorInvalidValue;
    k_gather_signals<<<dim3(64, (unsigned)n), 256, 0, st>>>(g);
    return cudaGetLastError();
}

template <bool RESID>
static cudaError_t launch_sqnorm(DevSig* d_sigs, int nsig, double* d_part, cudaStream_t st) {
    if (nsig <= 0) return cudaSuccess;
    k_sqnorm_part<RESID><<<dim3(ENERGY_PARTS, (unsigned)nsig), 256, 0, st>>>(d_sigs, d_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sqnorm_final<RESID><<<(unsigned)((nsig + 7) / 8), 256, 0, st>>>(d_sigs, nsig, d_part);
    return cudaGetLastError();
}

cudaError_t launch_reset_residual(DevSig* d_sigs, int nsig, double* d_part, cudaStream_t st) {
    return launch_sqnorm<true>(d_sigs, nsig, d_part, st);
}

cudaError_t launch_energy(DevSig* d_sigs, int nsig, double* d_part, cudaStream_t st) {
    return launch_sqnorm<false>(d_sigs, nsig, d_part, st);
}

cudaError_t launch_tree_build(const DevPlan& P, const DevSig* d_sigs, int nsig,
                              const long long* d_frame_prefix, long long total_frames, int dict,
                              cudaStream_t st, int flagged) {
    if (total_frames <= 0) return cudaSuccess;
    const int wpb = 8;
    const unsigned grid = (unsigned)((total_frames + wpb - 1) / wpb);
    if (P.fp64)
        k_tree_build<double2><<<grid, wpb * 32, 0, st>>>(P, d_sigs, nsig, d_frame_prefix,
                                                         total_frames, dict, flagged);
    else
        k_tree_build<float2><<<grid, wpb * 32, 0, st>>>(P, d_sigs, nsig, d_frame_prefix,
                                                        total_frames, dict, flagged);
    return cudaGetLastError();
}


}  // namespace mpg
