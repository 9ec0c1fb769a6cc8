// Launch logic of the persistent matching-pursuit loop (kernel in
// mp_loop_kernel.cuh): launch shapes, occupancy queries and the launch.
#include <cuda_runtime.h>

#include "mp_internal.cuh"

namespace mpg {

using LoopKernel_t = void (*)(DevPlan, DevSig*, const int*, long long, double, long long, int,
                              int, long long, double);
LoopKernel_t loop_kernel_f32(int threads, bool pow2);
LoopKernel_t loop_kernel_f64(int threads, bool pow2);

namespace {

using LoopKernel = LoopKernel_t;

// top-level keys a single CTA may hold: 512-thread CTAs run one per SM,
// 256-thread CTAs two and 128-thread CTAs three, so the shared memory of the
// top level shrinks with the CTA
int loop_topcap(int threads) { return threads >= 512 ? TOPCAP : threads == 256 ? TOPCAP / 2 : TOPCAP / 4; }

// top-level keys of a signal run by a single CTA: every frame, or groups of
// 2^gs frames with the smallest gs that fits the cap (the kernel makes the
// same choice)
int single_top(const DevSig& S, int W, int cap) {
    long long t = 0;
    for (int gs = 0;; ++gs) {
        t = 0;
        for (int w = 0; w < W; ++w) t += (S.N[w] + (1ll << gs) - 1) >> gs;
        if (t <= cap || gs >= 30) break;
    }
    return (int)t;
}

// the loop instantiation for a CTA size (0 if unsupported)
LoopKernel loop_kernel(int threads, bool pow2, bool fp64) {
    return fp64 ? loop_kernel_f64(threads, pow2) : loop_kernel_f32(threads, pow2);
}

cudaLaunchConfig_t loop_config(int nsig, int threads, int cs, size_t smem, cudaStream_t st,
                               cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nsig * cs));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t prepare(LoopKernel kf, int cs, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) e = cudaFuncSetAttribute(kf, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

int max_clusters(LoopKernel kf, int threads, int cs, size_t smem) {
    if (!kf || prepare(kf, cs, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = loop_config(1, threads, cs, smem, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kf, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

// dynamic shared memory of the loop: top level, class descriptors, <d, conj d>
// and modulation tables, dirty-group bits and list, touched-chunk lists
size_t mp_loop_smem_bytes(const DevPlan& P, int T, int, int) {
    size_t chl = 0;
    for (int w = 0; w < P.W; ++w) chl += (size_t)((P.d[w].nch + 7) & ~7);
    const size_t c2 = P.fp64 ? sizeof(double2) : sizeof(float2);
    size_t b = (size_t)((T + 1) & ~1) * sizeof(Key) + (size_t)P.ncls * sizeof(DevClass) + 16 +
               (size_t)(P.ngam + P.ncis) * c2 + 4 * (size_t)((T + 31) >> 5) +
               2 * (size_t)((T + 7) & ~7) + 2 * chl;
    return (b + 15) & ~(size_t)15;
}

int mp_loop_max_clusters(int threads, int cs, size_t smem, bool fp64) {
    // the power-of-two and generic instantiations have the same resources;
    // the generic one stands in
    return max_clusters(loop_kernel(threads, false, fp64), threads, cs, smem);
}

int mp_loop_threads(int nsig, int num_sms) {
    // 512-thread CTAs while every signal has SMs to itself, 256-thread CTAs
    // (two per SM) when there are more signals than SMs
    return nsig <= num_sms ? 512 : 256;
}

// largest dynamic shared memory of one CTA on this part
constexpr size_t SMEM_MAX = 227 * 1024;

// one CTA per signal whose top level holds at most `cap` keys (frames
// grouped by the smallest 2^gs that fits); cap a power of two in
// 64 .. loop_topcap(threads)
bool mp_loop_shape_single_cap(const DevPlan& P, const DevSig* hs, int B, int threads, int cap,
                              LoopShape* out) {
    if (threads != 128 && threads != 256 && threads != 512) return false;
    if (cap < 64 || (cap & (cap - 1)) || cap > loop_topcap(threads)) return false;
    int tmax = 1;
    for (int b = 0; b < B; ++b) {
        const int t = single_top(hs[b], P.W, cap);
        tmax = t > tmax ? t : tmax;
    }
    const size_t sm = mp_loop_smem_bytes(P, tmax, threads, 1);
    if (sm > SMEM_MAX || mp_loop_max_clusters(threads, 1, sm, P.fp64 != 0) < 1) return false;
    out->threads = threads;
    out->cs = 1;
    out->topcap = cap;
    out->smem = sm;
    return true;
}

// feasibility of a requested launch shape (threads per CTA, cluster size).
// A single CTA per signal groups its frames so that the top level fits: the
// cap starts at loop_topcap(threads) and halves while the shared memory
// does not fit.  A cluster CTA holds its own frames ungrouped.
bool mp_loop_shape_ok(const DevPlan& P, const DevSig* hs, int B, int threads, int c,
                      LoopShape* out) {
    if (threads != 128 && threads != 256 && threads != 512) return false;
    if (c != 1 && c != 2 && c != 4 && c != 8 && c != 16) return false;
    if (c == 1) {
        for (int cap = loop_topcap(threads); cap >= 64; cap >>= 1)
            if (mp_loop_shape_single_cap(P, hs, B, threads, cap, out)) return true;
        return false;
    }
    int lt = 0;
    for (int b = 0; b < B; ++b) {
        int t = 0;
        for (int w = 0; w < P.W; ++w) {
            if (hs[b].N[w] % c) return false;
            t += (int)(hs[b].N[w] / c);
        }
        lt = t > lt ? t : lt;
    }
    if (lt > TOPCAP_CLUSTER) return false;
    const size_t sm = mp_loop_smem_bytes(P, lt, threads, c);
    if (sm > SMEM_MAX || mp_loop_max_clusters(threads, c, sm, P.fp64 != 0) < 1) return false;
    out->threads = threads;
    out->cs = c;
    out->topcap = TOPCAP_CLUSTER;
    out->smem = sm;
    return true;
}

// launch shape for B signals.  Clusters give a signal several SMs while there
// are SMs to spare; they need every N_w divisible by the cluster size and the
// per-CTA top level to fit on chip.  Otherwise one CTA per signal.
void mp_loop_shape(const DevPlan& P, const DevSig* hs, int B, int num_sms, LoopShape* out) {
    const int nt = mp_loop_threads(B, num_sms);
    int c = B <= 8 ? 16 : B <= 16 ? 8 : B * 4 <= num_sms ? 4 : B * 2 <= num_sms ? 2 : 1;
    *out = LoopShape();
    // a cluster CTA runs only a few frame jobs per iteration: with up to
    // three dictionaries one warp per scheduler (and a spare warp) is fastest;
    // with more dictionaries the jobs and descriptors need more warps
    // (measured on GB300: 3 dictionaries 128 threads, 5 dictionaries 512)
    const int nt_cluster = P.W <= 3 ? 128 : 512;
    for (; c > 1; c >>= 1) {
        if (mp_loop_shape_ok(P, hs, B, nt_cluster, c, out)) return;
        if (nt_cluster != 128 && mp_loop_shape_ok(P, hs, B, 128, c, out)) return;
    }
    if (mp_loop_shape_ok(P, hs, B, nt, 1, out)) return;
    for (int t : {512, 256, 128})
        if (mp_loop_shape_ok(P, hs, B, t, 1, out)) return;
    *out = LoopShape();
}

cudaError_t launch_mp_loop(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig,
                           long long kmax, double thr_scale, long long budget_ns,
                           const LoopShape& sh, cudaStream_t st, long long reset_it,
                           double reset_scale) {
    if (nsig <= 0) return cudaSuccess;
    LoopKernel kf = loop_kernel(sh.threads, P.pow2 != 0, P.fp64 != 0);
    if (!kf || sh.topcap < 1) return cudaErrorInvalidValue;
    cudaError_t e = prepare(kf, sh.cs, sh.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = loop_config(nsig, sh.threads, sh.cs, sh.smem, st, attr);
    e = cudaLaunchKernelEx(&cfg, kf, P, d_sigs, d_order, kmax, thr_scale, budget_ns, sh.cs,
                           sh.topcap, reset_it, reset_scale);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mpg
