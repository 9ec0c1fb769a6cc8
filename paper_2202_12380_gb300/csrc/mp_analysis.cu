// Analysis (Alg. 1 initialisation, Sec. 5): rho_0 = D_w^* x for every
// dictionary of every signal, E_0 = ||x||^2, and the max trees.
//
// The reduced DGT
//   rho(m, n) = sum_{i=0}^{w-1} x((n a + i - w/2) mod L) g(i) e^{-i 2 pi m (i - w/2) / M}
// is one real GEMM per dictionary: C = A B with A[2m + {0,1}][i] the
// windowed cosine / negated sine rows (built by the plan) and B[i][n] =
// x(n a + i - w/2) the frames, gathered on the fly from the signal (no
// framed copy is materialised).  The FP32 path below runs it on the SIMT
// cores with register blocking; the epilogue writes complex rows of the
// frame-major coefficient plane directly.
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

__global__ void __launch_bounds__(256) k_analysis_sgemm(const float* __restrict__ A, int Kp, int w,
                                                        int a, int Mrp, int nsig,
                                                        const long long* __restrict__ tprefix,
                                                        const DevSig* __restrict__ sigs, int dict,
                                                        int flagged) {
    __shared__ __align__(16) float As[BK][BM];
    __shared__ __align__(16) float Bs[BK][BN];
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

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    // A tile loader: row r0 + (tid >> 1), 8 consecutive k from (tid & 1) * 8
    const int ar = tid >> 1, ak = (tid & 1) * 8;
    const float* Arow = A + (long long)(r0 + ar) * Kp;
    // B tile loader: k = tid & 15, frames (tid >> 4) + 16 q
    const int bk = tid & 15, bn = tid >> 4;

    for (int k0 = 0; k0 < Kp; k0 += BK) {
        float4 a0 = *reinterpret_cast<const float4*>(Arow + k0 + ak);
        float4 a1 = *reinterpret_cast<const float4*>(Arow + k0 + ak + 4);
        float bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long n = n0 + bn + 16 * q;
            int i = k0 + bk;
            float v = 0.f;
            if (n < N && i < w) v = __ldg(x + lmod(n * a + i - w / 2, L));
            bv[q] = v;
        }
        __syncthreads();
        As[ak + 0][ar] = a0.x;
        As[ak + 1][ar] = a0.y;
        As[ak + 2][ar] = a0.z;
        As[ak + 3][ar] = a0.w;
        As[ak + 4][ar] = a1.x;
        As[ak + 5][ar] = a1.y;
        As[ak + 6][ar] = a1.z;
        As[ak + 7][ar] = a1.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) Bs[bk][bn + 16 * q] = bv[q];
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 x0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
            float4 x1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
            float4 y0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            float ar8[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            float bc4[4] = {y0.x, y0.y, y0.z, y0.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar8[i], bc4[j], acc[i][j]);
        }
    }
    // epilogue: rows ty*8 .. +7 are bins (r0 + ty*8)/2 .. +3 (re, im pairs)
    const int m0 = (r0 + ty * 8) >> 1;
    float2* plane = S.plane[dict];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        long long n = n0 + tx * 4 + j;
        if (n >= N) continue;
        float2* dst = plane + n * Mrp + m0;
        if (m0 + 3 < Mrp) {
            float4 v0 = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
            float4 v1 = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
            reinterpret_cast<float4*>(dst)[0] = v0;
            reinterpret_cast<float4*>(dst)[1] = v1;
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (m0 + b < Mrp) dst[b] = make_float2(acc[2 * b][j], acc[2 * b + 1][j]);
        }
    }
}

// E_0 = ||x||^2 in FP64, one block per signal, fixed reduction order
__global__ void __launch_bounds__(1024) k_energy(DevSig* sigs) {
    DevSig& S = sigs[blockIdx.x];
    const float* x = S.x;
    double acc = 0.0;
    for (long long l = threadIdx.x; l < S.L; l += blockDim.x) {
        double v = (double)x[l];
        acc = fma(v, v, acc);
    }
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (threadIdx.x == 0) {
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
}

// level 0 (per 32-bin chunk) and level 1 (per frame) of dictionary `dict`,
// one warp per frame
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
    const float2* row = S.plane[dict] + n * D.Mrp;
    Key* l0 = S.l0[dict] + n * D.nch;
    const unsigned fb = S.fbase[dict] + ((unsigned)n << D.msh);
    Key best = 0ull;
    for (int ch = 0; ch < D.nch; ++ch) {
        const int m = ch * CHUNK + lane;
        const float2 v = row[m];
        const Key k = (m < D.Mr) ? make_key_sel(v, fb + m, m, D, P.gam, P.pedantic) : 0ull;
        const Key r = warp_max_key(k);
        if (lane == 0) l0[ch] = r;
        best = r > best ? r : best;
    }
    if (lane == 0) S.l1[dict][n] = best;
}

// reset pass, one block per signal: r = x - y and E = E_out = ||r||^2
// (FP64, fixed order) for the flagged signals
__global__ void __launch_bounds__(1024) k_reset_residual(DevSig* sigs) {
    DevSig& S = sigs[blockIdx.x];
    if (!S.reanalyze) return;
    double acc = 0.0;
    for (long long l = threadIdx.x; l < S.L; l += blockDim.x) {
        const float d = S.x[l] - S.y[l];
        S.r[l] = d;
        acc = fma((double)d, (double)d, acc);
    }
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (threadIdx.x == 0) {
            S.E = v;
            S.E_out = v;
            S.k_out = S.k;
            S.reset_pending = 0;
            S.use_r = 1;
        }
    }
}

}  // namespace

cudaError_t launch_analysis_sgemm(const float* A, int Arows, int Kp, int w_len, int a, int Mrp,
                                  int nsig, const long long* d_tile_prefix, const DevSig* d_sigs,
                                  int dict, long long total_frame_tiles, cudaStream_t st,
                                  int flagged) {
    if (total_frame_tiles <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_frame_tiles, (unsigned)(Arows / BM));
    k_analysis_sgemm<<<grid, 256, 0, st>>>(A, Kp, w_len, a, Mrp, nsig, d_tile_prefix, d_sigs, dict,
                                           flagged);
    return cudaGetLastError();
}

cudaError_t launch_reset_residual(DevSig* d_sigs, int nsig, cudaStream_t st) {
    k_reset_residual<<<nsig, 1024, 0, st>>>(d_sigs);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DevSig* d_sigs, int nsig, double*, int, cudaStream_t st) {
    k_energy<<<nsig, 1024, 0, st>>>(const_cast<DevSig*>(d_sigs));
    return cudaGetLastError();
}

cudaError_t launch_tree_build(const DevPlan& P, const DevSig* d_sigs, int nsig,
                              const long long* d_frame_prefix, long long total_frames, int dict,
                              cudaStream_t st, int flagged) {
    if (total_frames <= 0) return cudaSuccess;
    const int wpb = 8;
    k_tree_build<<<(unsigned)((total_frames + wpb - 1) / wpb), wpb * 32, 0, st>>>(
        P, d_sigs, nsig, d_frame_prefix, total_frames, dict, flagged);
    return cudaGetLastError();
}


}  // namespace mpg
