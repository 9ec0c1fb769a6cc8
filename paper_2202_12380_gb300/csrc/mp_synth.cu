// Synthesis of the selected atoms (eq. idgtreal) and the true residual
// energy ||x - y||^2 (FP64).
//
// Each atom (w, m, n, c) adds 2 Re(c d_{m,n}) (or Re(c d) at m in {0, M/2},
// where the conjugate partner is missing) to y, with
// d_{m,n}(n a + t) = g(t) e^{i 2 pi m t / M}, t = -w/2 .. w/2-1.  One block
// per atom (grid-stride), FP32 accumulation with atomics into y.
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

__global__ void k_synth(DevPlan P, const DevSig* __restrict__ sig, float* __restrict__ y) {
    const long long natoms = sig->k;
    const long long L = sig->L;
    for (long long at = blockIdx.x; at < natoms; at += gridDim.x) {
        const mp_atom A = sig->atoms[at];
        const DevDict& D = P.d[A.dict];
        const float* g = P.g32 + D.g_off;
        const float fac = (A.m == 0 || 2 * A.m == D.M) ? 1.f : 2.f;
        for (int i = threadIdx.x; i < D.wlen; i += blockDim.x) {
            const long long t = i - D.wlen / 2;
            const long long q = lmod((long long)A.m * t, D.M);
            float s, c;
            sincospif(2.0f * (float)q / (float)D.M, &s, &c);
            const float v = fac * g[i] * (A.re * c - A.im * s);
            atomicAdd(y + lmod(A.n * D.a + t, L), v);
        }
    }
}

__global__ void __launch_bounds__(1024) k_resid_energy(const DevSig* __restrict__ sig,
                                                       const float* __restrict__ y,
                                                       double* __restrict__ out) {
    const float* x = sig->x;
    const long long L = sig->L;
    double acc = 0.0;
    for (long long l = threadIdx.x; l < L; l += blockDim.x) {
        double d = (double)x[l] - (double)y[l];
        acc = fma(d, d, acc);
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
        if (threadIdx.x == 0) out[0] = v;
    }
}

}  // namespace

cudaError_t launch_synth(const DevPlan& P, const DevSig* d_sig, long long, float* y, long long L,
                         cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(float) * L, st);
    if (e != cudaSuccess) return e;
    k_synth<<<152 * 8, 256, 0, st>>>(P, d_sig, y);
    return cudaGetLastError();
}

cudaError_t launch_resid_energy(const DevSig* d_sig, const float* y, long long, double* d_out, int,
                                cudaStream_t st) {
    k_resid_energy<<<1, 1024, 0, st>>>(d_sig, y, d_out);
    return cudaGetLastError();
}

}  // namespace mpg
