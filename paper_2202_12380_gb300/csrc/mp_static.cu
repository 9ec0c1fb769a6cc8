// mp_decompose_static: analysis + matching pursuit of one signal without any
// device allocation.
//
// Who needs it: callers that must not call cudaMalloc while decomposing --
// real-time audio threads that may not block on the allocator (cudaMalloc
// can synchronise the device and take unbounded time), and hosts that run
// under a fixed device-memory budget or have handed the device's memory to
// their own pool allocator.  They create the plan once at set-up (that call
// does allocate) and then decompose with this entry point, which takes its
// coefficient planes, max trees and bookkeeping from one file-scope device
// array instead of allocating a state.  It runs the FP32 analysis only, so
// plans made with MP_ANALYSIS_BF16X3 are rejected.
//
// The array g_static_scratch (MP_STATIC_SCRATCH_BYTES) is part of the
// library image: every GPU that loads the library holds it until the process
// exits.  In host code its name is only a host-side stand-in, so the device
// address is obtained once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.  Every call on a device shares
// the array and finds the previous call's contents there; all regions are
// rewritten from scratch by each call (descriptor, signal copy, energy
// partial sums, planes including padding bins, all tree levels), so nothing
// is carried over.
// Calls that overlap on the GPU (other streams, other host threads) race on
// the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "mp_internal.cuh"

using namespace mpg;

namespace {

constexpr size_t MP_STATIC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[MP_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};

// small per-call tables written by a kernel (passed by value, no copy from
// host memory)
struct StaticTables {
    DevSig sig;
    long long tile_prefix[MAXW][2];
    long long frame_prefix[MAXW][2];
};

struct StaticLayout {
    size_t o_sig, o_order, o_tp, o_fp, o_epart, o_errs, total;
    size_t o_plane[MAXW], o_l0[MAXW], o_l1[MAXW], o_x;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_static_init(StaticTables t, unsigned char* base, StaticLayout lay, int W) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *reinterpret_cast<DevSig*>(base + lay.o_sig) = t.sig;
    *reinterpret_cast<int*>(base + lay.o_order) = 0;
    long long* tp = reinterpret_cast<long long*>(base + lay.o_tp);
    long long* fp = reinterpret_cast<long long*>(base + lay.o_fp);
    for (int w = 0; w < W; ++w) {
        tp[2 * w] = t.tile_prefix[w][0];
        tp[2 * w + 1] = t.tile_prefix[w][1];
        fp[2 * w] = t.frame_prefix[w][0];
        fp[2 * w + 1] = t.frame_prefix[w][1];
    }
}

// device address of the scratch array for the current device; the first
// call on a device resolves it (do that before any stream capture)
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        mpg_set_error("mp_decompose_static: cudaGetDevice: %s", cudaGetErrorString(e));
        return MP_ECUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        mpg_set_error("mp_decompose_static: device index %d out of range", dev);
        return MP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            mpg_set_error("mp_decompose_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return MP_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return MP_OK;
}

}  // namespace

extern "C" int mp_decompose_static(const mp_plan* p, const float* x_dev, int64_t L, int64_t K_max,
                                   double target_snr_db, mp_atom* atoms_dev, double* errors_dev,
                                   int64_t* n_atoms, int* stop_reason, double* final_snr_db) {
    mpg::NvtxRange nvtx_range("mp_decompose_static");
    if (!p || !x_dev || !atoms_dev || L <= 0 || K_max < 1 || std::isnan(target_snr_db)) {
        mpg_set_error("mp_decompose_static: bad argument (need plan, signal, atom buffer, "
                      "L > 0, K_max >= 1)");
        return MP_EINVAL;
    }
    if (p->flags & MP_COEF_FP64) {
        mpg_set_error("mp_decompose_static: the plan asks for FP64 coefficient planes; this entry "
                      "point holds FP32 planes only (use mp_analyze / mp_run)");
        return MP_ENOTCOMPAT;
    }
    if (p->flags & MP_ANALYSIS_BF16X3) {
        mpg_set_error("mp_decompose_static: the plan asks for the split-BF16 analysis; this entry "
                      "point runs the FP32 analysis only (make the plan without "
                      "MP_ANALYSIS_BF16X3, or use mp_analyze / mp_run)");
        return MP_ENOTCOMPAT;
    }
    {
        int cur = -1;
        cudaError_t ge = cudaGetDevice(&cur);
        if (ge != cudaSuccess) {
            mpg_set_error("mp_decompose_static: cudaGetDevice: %s", cudaGetErrorString(ge));
            return MP_ECUDA;
        }
        if (cur != p->device) {
            mpg_set_error("mp_decompose_static: the current device is %d but the plan lives on "
                          "device %d; make the plan's device current first", cur, p->device);
            return MP_EINVAL;
        }
    }
    const int W = p->W;
    int wmax = 0;
    for (int w = 0; w < W; ++w) {
        wmax = wmax > p->wlen[w] ? wmax : p->wlen[w];
        if (L % p->a[w] || L % p->M[w]) {
            mpg_set_error("mp_decompose_static: L=%lld is not a multiple of a=%d and M=%d",
                          (long long)L, p->a[w], p->M[w]);
            return MP_EINVAL;
        }
    }
    if (L < 2LL * wmax) {
        mpg_set_error("mp_decompose_static: L=%lld is below 2 max(w) = %d", (long long)L, 2 * wmax);
        return MP_EINVAL;
    }
    // layout inside the scratch array (same structure as an mp_state of one signal)
    StaticTables t;
    memset(&t, 0, sizeof(t));
    StaticLayout lay;
    memset(&lay, 0, sizeof(lay));
    DevSig& S = t.sig;
    S.L = L;
    size_t off = 0;
    lay.o_sig = off;
    off = al(off + sizeof(DevSig));
    lay.o_order = off;
    off = al(off + sizeof(int));
    lay.o_tp = off;
    off = al(off + sizeof(long long) * 2 * MAXW);
    lay.o_fp = off;
    off = al(off + sizeof(long long) * 2 * MAXW);
    lay.o_epart = off;
    off = al(off + sizeof(double) * ENERGY_PARTS);
    unsigned long long P = 0;
    for (int w = 0; w < W; ++w) {
        const DevDict& D = p->dp.d[w];
        S.N[w] = L / D.a;
        S.Nmask[w] = (S.N[w] & (S.N[w] - 1)) == 0 ? (int)(S.N[w] - 1) : 0;
        S.fbase[w] = (unsigned)P;
        P += (unsigned long long)S.N[w] << D.msh;
        lay.o_plane[w] = off;
        off = al(off + sizeof(float2) * S.N[w] * D.Mrp);
        lay.o_l0[w] = off;
        off = al(off + sizeof(Key) * S.N[w] * D.nch);
        lay.o_l1[w] = off;
        off = al(off + sizeof(Key) * S.N[w]);
        t.tile_prefix[w][1] = (S.N[w] + 63) / 64;
        t.frame_prefix[w][1] = S.N[w];
    }
    if (P >= 0xffffffffull) {
        mpg_set_error("mp_decompose_static: too many coefficients");
        return MP_EINVAL;
    }
    S.fbase[W] = (unsigned)P;
    lay.o_x = off;
    off = al(off + sizeof(float) * L);
    lay.o_errs = off;
    if (!errors_dev) off = al(off + sizeof(double) * K_max);
    lay.total = off;
    if (lay.total > MP_STATIC_SCRATCH_BYTES) {
        mpg_set_error("mp_decompose_static: this signal needs %zu bytes of scratch, the static "
                      "array holds %zu (use mp_analyze / mp_run)", lay.total,
                      MP_STATIC_SCRATCH_BYTES);
        return MP_EINVAL;
    }
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    for (int w = 0; w < W; ++w) {
        S.plane[w] = reinterpret_cast<float2*>(base + lay.o_plane[w]);
        S.l0[w] = reinterpret_cast<Key*>(base + lay.o_l0[w]);
        S.l1[w] = reinterpret_cast<Key*>(base + lay.o_l1[w]);
    }
    S.x = reinterpret_cast<const float*>(base + lay.o_x);
    S.atoms = atoms_dev;
    S.errs = errors_dev ? errors_dev : reinterpret_cast<double*>(base + lay.o_errs);
    S.cap = K_max;

    cudaStream_t st = p->stream;
    DevSig* d_sig = reinterpret_cast<DevSig*>(base + lay.o_sig);
    const int* d_order = reinterpret_cast<const int*>(base + lay.o_order);
    const long long* d_tp = reinterpret_cast<const long long*>(base + lay.o_tp);
    const long long* d_fp = reinterpret_cast<const long long*>(base + lay.o_fp);
    cudaError_t e;
#define CKS(call)                                                                        \
    do {                                                                                 \
        e = (call);                                                                      \
        if (e != cudaSuccess) {                                                          \
            mpg_set_error("mp_decompose_static: %s: %s", #call, cudaGetErrorString(e));  \
            return MP_ECUDA;                                                             \
        }                                                                                \
    } while (0)
    k_static_init<<<1, 32, 0, st>>>(t, base, lay, W);
    CKS(cudaGetLastError());
    CKS(cudaMemcpyAsync(base + lay.o_x, x_dev, sizeof(float) * L, cudaMemcpyDeviceToDevice, st));
    CKS(launch_energy(d_sig, 1, reinterpret_cast<double*>(base + lay.o_epart), st));
    for (int w = 0; w < W; ++w) {
        const DevDict& D = p->dp.d[w];
        CKS(launch_analysis_sgemm(p->d_A[w], p->Arows[w], p->Akp[w], D.wlen, D.a, D.Mrp, 1,
                                  d_tp + 2 * w, d_sig, w, t.tile_prefix[w][1], st));
        CKS(launch_tree_build(p->dp, d_sig, 1, d_fp + 2 * w, t.frame_prefix[w][1], w, st));
    }
    const double thr_scale = std::pow(10.0, -target_snr_db / 10.0);
    LoopShape shape;
    mp_loop_shape(p->dp, &S, 1, p->num_sms, &shape);
    if (shape.threads == 0) {
        mpg_set_error("mp_decompose_static: no MP launch shape fits in shared memory");
        return MP_ENOTCOMPAT;
    }
    CKS(launch_mp_loop(p->dp, d_sig, d_order, 1, K_max, thr_scale, 0, shape, st));
    if (n_atoms || stop_reason || final_snr_db) {
        DevSig out;
        CKS(cudaMemcpyAsync(&out, d_sig, sizeof(DevSig), cudaMemcpyDeviceToHost, st));
        CKS(cudaStreamSynchronize(st));
        if (out.bounds) {
            mpg_set_error("mp_decompose_static: bounds check: MP-loop access site %d was out of "
                          "range (the access was skipped)", out.bounds);
            return MP_ECUDA;
        }
        if (n_atoms) *n_atoms = out.k;
        if (stop_reason) *stop_reason = out.stop;
        if (final_snr_db) *final_snr_db = 10.0 * std::log10(out.E0 / out.E);
    }
#undef CKS
    return MP_OK;
}
