// C ABI: state management, analysis, the MP launch, atom read-back and
// synthesis.  Host code only orchestrates; every arithmetic step of the
// method runs in the kernels of mp_plan.cu, mp_analysis.cu, mp_loop.cu and
// mp_synth.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "mp_internal.cuh"

using namespace mpg;

static thread_local char g_err[512] = "";

extern "C" void mpg_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char* mp_last_error(void) { return g_err; }

struct mp_state {
    const mp_plan* plan;
    int B;
    std::vector<long long> L;
    std::vector<DevSig> hs;  // host copy of the static descriptor fields
    DevSig* d_sigs;
    int* d_order;
    void* pool;              // planes, trees, signal copies
    long long* d_tile_prefix[MAXW];
    long long total_tiles[MAXW];
    long long* d_frame_prefix[MAXW];
    long long total_frames[MAXW];
    LoopShape shape;         // MP launch shape (see mp_loop_shape)
    long long cap;           // atom capacity per signal
    mp_atom* d_atoms;
    double* d_errs;
    double* d_scalar;
    double* d_epart;         // [B][ENERGY_PARTS]: partial sums of the FP64 signal energies
    double time_limit_s;
    long long reset_it;      // resets (Alg. 2): selections per reset, 0 = off
    double reset_db;         // resets once 10 log10(E/E_out) < reset_db (< 0), 0 = off
    // split-BF16 analysis: padded BF16 signal segments and per-dictionary views
    void* d_xhi;
    void* d_xlo;
    long long* d_seg;        // [2][B]: segment offsets, lengths (elements)
    int seg_pad;
    int* d_brow;             // [W][B]: first view row of each signal's frame 0
    long long* d_tc_prefix[MAXW];
    long long total_tc_tiles[MAXW];
    int tc_frames[MAXW];     // frames per tensor-core analysis tile (128 or 256)
    int* d_err;
    alignas(64) unsigned char tmB[MAXW][2][128];
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    mpg_set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
}

#define CKR(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

void state_free(mp_state* s) {
    if (!s) return;
    if (s->d_sigs) cudaFree(s->d_sigs);
    if (s->d_order) cudaFree(s->d_order);
    if (s->pool) cudaFree(s->pool);
    for (int w = 0; w < MAXW; ++w) {
        if (s->d_tile_prefix[w]) cudaFree(s->d_tile_prefix[w]);
        if (s->d_frame_prefix[w]) cudaFree(s->d_frame_prefix[w]);
    }
    if (s->d_atoms) cudaFree(s->d_atoms);
    if (s->d_errs) cudaFree(s->d_errs);
    if (s->d_scalar) cudaFree(s->d_scalar);
    if (s->d_epart) cudaFree(s->d_epart);
    if (s->d_xhi) cudaFree(s->d_xhi);
    if (s->d_xlo) cudaFree(s->d_xlo);
    if (s->d_seg) cudaFree(s->d_seg);
    if (s->d_brow) cudaFree(s->d_brow);
    for (int w = 0; w < MAXW; ++w)
        if (s->d_tc_prefix[w]) cudaFree(s->d_tc_prefix[w]);
    if (s->d_err) cudaFree(s->d_err);
    delete s;
}

int validate_lengths(const mp_plan* p, int B, const int64_t* L) {
    if (B < 1 || !L) {
        mpg_set_error("mp_analyze: need B >= 1 and a length array");
        return MP_EINVAL;
    }
    int wmax = 0;
    for (int w = 0; w < p->W; ++w) wmax = std::max(wmax, p->wlen[w]);
    for (int b = 0; b < B; ++b) {
        if (L[b] <= 0) {
            mpg_set_error("mp_analyze: signal %d has length %lld", b, (long long)L[b]);
            return MP_EINVAL;
        }
        for (int w = 0; w < p->W; ++w)
            if (L[b] % p->a[w] || L[b] % p->M[w]) {
                mpg_set_error("mp_analyze: length %lld of signal %d is not a multiple of a=%d "
                              "and M=%d", (long long)L[b], b, p->a[w], p->M[w]);
                return MP_EINVAL;
            }
        if (L[b] < 2LL * wmax) {
            mpg_set_error("mp_analyze: length %lld of signal %d is below 2 max(w) = %d",
                          (long long)L[b], b, 2 * wmax);
            return MP_EINVAL;
        }
        unsigned long long P = 0;
        for (int w = 0; w < p->W; ++w)
            P += (unsigned long long)(L[b] / p->a[w]) << p->dp.d[w].msh;
        if (P >= 0xffffffffull) {
            mpg_set_error("mp_analyze: signal %d needs a flat index range of %llu (limit 2^32-1)",
                          b, P);
            return MP_EINVAL;
        }
    }
    return MP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int state_create(const mp_plan* p, int B, const int64_t* L, mp_state** out) {
    mp_state* s = new mp_state();
    s->d_xhi = s->d_xlo = nullptr;
    s->d_seg = nullptr;
    s->d_brow = nullptr;
    s->d_err = nullptr;
    memset(s->d_tc_prefix, 0, sizeof(s->d_tc_prefix));
    memset(s->tc_frames, 0, sizeof(s->tc_frames));
    memset(s->d_tile_prefix, 0, sizeof(s->d_tile_prefix));
    memset(s->d_frame_prefix, 0, sizeof(s->d_frame_prefix));
    s->plan = p;
    s->B = B;
    s->L.assign(L, L + B);
    s->hs.resize(B);
    s->d_sigs = nullptr;
    s->d_order = nullptr;
    s->pool = nullptr;
    s->d_atoms = nullptr;
    s->d_errs = nullptr;
    s->d_scalar = nullptr;
    s->d_epart = nullptr;
    s->cap = 0;
    s->time_limit_s = 0.0;
    s->reset_it = 0;
    s->reset_db = 0.0;
    const int W = p->W;
    const size_t esz = (p->flags & MP_COEF_FP64) ? sizeof(double2) : sizeof(float2);
    // layout of every signal inside one pool
    size_t off = 0;
    std::vector<size_t> o_plane(B * W), o_l0(B * W), o_l1(B * W), o_x(B), o_r(B), o_y(B);
    for (int b = 0; b < B; ++b) {
        DevSig& S = s->hs[b];
        memset(&S, 0, sizeof(S));
        S.L = L[b];
        long long F = 0;
        unsigned fb = 0;
        for (int w = 0; w < W; ++w) {
            const DevDict& D = p->dp.d[w];
            S.N[w] = L[b] / D.a;
            S.Nmask[w] = (S.N[w] & (S.N[w] - 1)) == 0 ? (int)(S.N[w] - 1) : 0;
            S.fbase[w] = fb;
            fb += (unsigned)(S.N[w] << D.msh);
            F += S.N[w];
            o_plane[b * W + w] = off;
            off = align256(off + esz * S.N[w] * D.Mrp);
            o_l0[b * W + w] = off;
            off = align256(off + sizeof(Key) * S.N[w] * D.nch);
            o_l1[b * W + w] = off;
            off = align256(off + sizeof(Key) * S.N[w]);
        }
        S.fbase[W] = fb;
        o_x[b] = off;
        off = align256(off + sizeof(float) * L[b]);
        o_r[b] = off;
        off = align256(off + sizeof(float) * L[b]);
        o_y[b] = off;
        off = align256(off + sizeof(float) * L[b]);
    }
    cudaError_t e = cudaMalloc(&s->pool, std::max<size_t>(off, 256));
    if (e != cudaSuccess) {
        state_free(s);
        return cuda_fail(e, "mp_analyze: allocating coefficient planes");
    }
    char* base = (char*)s->pool;
    for (int b = 0; b < B; ++b) {
        DevSig& S = s->hs[b];
        for (int w = 0; w < W; ++w) {
            S.plane[w] = (float2*)(base + o_plane[b * W + w]);
            S.l0[w] = (Key*)(base + o_l0[b * W + w]);
            S.l1[w] = (Key*)(base + o_l1[b * W + w]);
        }
        S.x = (const float*)(base + o_x[b]);
        S.r = (float*)(base + o_r[b]);
        S.y = (float*)(base + o_y[b]);
    }
    // zero the pool once so padding bins are zero
    cudaStream_t st = p->stream;
    e = cudaMemsetAsync(s->pool, 0, std::max<size_t>(off, 256), st);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_sigs, sizeof(DevSig) * B);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_sigs, s->hs.data(), sizeof(DevSig) * B, cudaMemcpyHostToDevice, st);
    // CTA order: longest signal first
    std::vector<int> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return L[x] > L[y]; });
    if (e == cudaSuccess) e = cudaMalloc(&s->d_order, sizeof(int) * B);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_order, order.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st);
    // per-dictionary work tables for the analysis and the tree build
    for (int w = 0; w < W && e == cudaSuccess; ++w) {
        std::vector<long long> tp(B + 1, 0), fp(B + 1, 0);
        for (int b = 0; b < B; ++b) {
            tp[b + 1] = tp[b] + (s->hs[b].N[w] + 63) / 64;
            fp[b + 1] = fp[b] + s->hs[b].N[w];
        }
        s->total_tiles[w] = tp[B];
        s->total_frames[w] = fp[B];
        e = cudaMalloc(&s->d_tile_prefix[w], sizeof(long long) * (B + 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_frame_prefix[w], sizeof(long long) * (B + 1));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_tile_prefix[w], tp.data(), sizeof(long long) * (B + 1),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_frame_prefix[w], fp.data(), sizeof(long long) * (B + 1),
                                cudaMemcpyHostToDevice, st);
        // host vectors must outlive the async copies
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->d_scalar, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_epart, sizeof(double) * ENERGY_PARTS * B);
    if (e == cudaSuccess && (p->flags & MP_ANALYSIS_BF16X3)) {
        // padded BF16 segments: seg[j] = x(j - pad), offsets multiples of a_max
        int amax = 0, wmax = 0, kmax64 = 0;
        for (int w = 0; w < W; ++w) {
            amax = std::max(amax, p->a[w]);
            wmax = std::max(wmax, p->wlen[w]);
            kmax64 = std::max(kmax64, p->Kp64[w]);
        }
        const long long pad = ((wmax / 2 + amax - 1) / amax) * (long long)amax;
        s->seg_pad = (int)pad;
        std::vector<long long> seg(2 * B);
        long long tot = 0;
        for (int b = 0; b < B; ++b) {
            const long long len = ((pad + L[b] + kmax64 + amax + amax - 1) / amax) * amax;
            seg[b] = tot;
            seg[B + b] = len;
            tot += len;
        }
        std::vector<int> brow((size_t)W * B);
        for (int w = 0; w < W; ++w)
            for (int b = 0; b < B; ++b)
                brow[(size_t)w * B + b] = (int)((seg[b] + pad - p->wlen[w] / 2) / p->a[w]);
        e = cudaMalloc(&s->d_xhi, 2 * tot);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_xlo, 2 * tot);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_seg, sizeof(long long) * 2 * B);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_brow, sizeof(int) * W * B);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(int), st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_seg, seg.data(), sizeof(long long) * 2 * B,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_brow, brow.data(), sizeof(int) * W * B, cudaMemcpyHostToDevice,
                                st);
        for (int w = 0; w < W && e == cudaSuccess; ++w) {
            long long t256 = 0, f128 = 0;
            for (int b = 0; b < B; ++b) {
                t256 += (s->hs[b].N[w] + 255) / 256;
                f128 += (s->hs[b].N[w] + 127) / 128 * 128;
            }
            const int bn = analysis_tc_frames(p->Arows[w] / 128, t256, f128, t256 * 256, p->num_sms);
            s->tc_frames[w] = bn;
            std::vector<long long> tp(B + 1, 0);
            for (int b = 0; b < B; ++b) tp[b + 1] = tp[b] + (s->hs[b].N[w] + bn - 1) / bn;
            s->total_tc_tiles[w] = tp[B];
            e = cudaMalloc(&s->d_tc_prefix[w], sizeof(long long) * (B + 1));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->d_tc_prefix[w], tp.data(), sizeof(long long) * (B + 1),
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            const unsigned long long aw = (unsigned long long)p->a[w];
            if (e == cudaSuccess &&
                (!encode_bf16_map(s->tmB[w][0], s->d_xhi, aw, tot / aw, aw * 2, (unsigned)bn) ||
                 !encode_bf16_map(s->tmB[w][1], s->d_xlo, aw, tot / aw, aw * 2, (unsigned)bn))) {
                state_free(s);
                return MP_ECUDA;
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        state_free(s);
        return cuda_fail(e, "mp_analyze: state set-up");
    }
    mp_loop_shape(p->dp, s->hs.data(), B, p->num_sms, &s->shape);
    if (s->shape.threads == 0) {
        state_free(s);
        mpg_set_error("mp_analyze: no MP launch shape fits these signals and dictionaries in "
                      "shared memory");
        return MP_ENOTCOMPAT;
    }
    *out = s;
    return MP_OK;
}

int analysis_pass(mp_state* s, int flagged);

int analyze_impl(const mp_plan* p, mp_state** state, int B, const float* const* x,
                 const int64_t* L, cudaMemcpyKind kind) {
    if (!p || !state || !x) {
        mpg_set_error("mp_analyze: null argument");
        return MP_EINVAL;
    }
    int rc = validate_lengths(p, B, L);
    if (rc) return rc;
    for (int b = 0; b < B; ++b)
        if (!x[b]) {
            mpg_set_error("mp_analyze: signal pointer %d is null", b);
            return MP_EINVAL;
        }
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    if (kind == cudaMemcpyDeviceToDevice &&
        cudaStreamIsCapturing(p->stream, &capst) == cudaSuccess &&
        capst == cudaStreamCaptureStatusNone) {
        // the signals are read by a kernel: each must be memory this device
        // can address (its own device memory, managed or page-locked host
        // memory).  Checked outside stream capture only, where no query
        // can disturb a capture.
        for (int b = 0; b < B; ++b) {
            cudaPointerAttributes pa;
            if (cudaPointerGetAttributes(&pa, x[b]) != cudaSuccess) {
                cudaGetLastError();
                mpg_set_error("mp_analyze: signal pointer %d is not a CUDA address", b);
                return MP_EINVAL;
            }
            if (pa.type == cudaMemoryTypeUnregistered) {
                mpg_set_error("mp_analyze: signal %d is in pageable host memory (use "
                              "mp_analyze_host)", b);
                return MP_EINVAL;
            }
            if (pa.type == cudaMemoryTypeDevice && pa.device != p->device) {
                mpg_set_error("mp_analyze: signal %d is on device %d, the plan's is %d", b,
                              pa.device, p->device);
                return MP_EINVAL;
            }
        }
    }
    mp_state* s = *state;
    if (s) {
        bool same = s->plan == p && s->B == B;
        for (int b = 0; same && b < B; ++b) same = s->L[b] == L[b];
        if (!same) {
            mpg_set_error("mp_analyze: state was made for another plan or other lengths");
            return MP_EINVAL;
        }
    } else {
        rc = state_create(p, B, L, &s);
        if (rc) return rc;
    }
    cudaStream_t st = p->stream;
    if (kind == cudaMemcpyDeviceToDevice) {
        // one launch per GATHER_MAX signals instead of one copy per signal
        GatherArgs g;
        for (int b0 = 0; b0 < B; b0 += GATHER_MAX) {
            const int n = std::min(GATHER_MAX, B - b0);
            for (int i = 0; i < n; ++i) {
                g.src[i] = x[b0 + i];
                g.dst[i] = const_cast<float*>(s->hs[b0 + i].x);
                g.len[i] = L[b0 + i];
            }
            CKR(launch_gather_signals(g, n, st));
        }
    } else {
        for (int b = 0; b < B; ++b)
            CKR(cudaMemcpyAsync((void*)s->hs[b].x, x[b], sizeof(float) * L[b], kind, st));
    }
    CKR(launch_energy(s->d_sigs, B, s->d_epart, st));
    rc = analysis_pass(s, 0);
    if (rc) return rc;
    if (kind == cudaMemcpyHostToDevice) CKR(cudaStreamSynchronize(st));
    *state = s;
    return MP_OK;
}

// coefficient planes and max trees of every signal (flagged = 0) or of the
// signals flagged for a reset pass (flagged = 1)
int analysis_pass(mp_state* s, int flagged) {
    const mp_plan* p = s->plan;
    const int B = s->B;
    cudaStream_t st = p->stream;
    const bool tc = (p->flags & MP_ANALYSIS_BF16X3) != 0;
    if (tc)
        CKR(launch_split_segments(s->d_sigs, B, s->d_seg, s->d_seg + B, s->seg_pad, s->d_xhi,
                                  s->d_xlo, st, flagged));
    for (int w = 0; w < p->W; ++w) {
        const DevDict& D = p->dp.d[w];
        if (tc) {
            alignas(64) unsigned char maps[4][128];
            memcpy(maps[0], p->tmA[w][0], 128);
            memcpy(maps[1], p->tmA[w][1], 128);
            memcpy(maps[2], s->tmB[w][0], 128);
            memcpy(maps[3], s->tmB[w][1], 128);
            CKR(launch_analysis_tc(maps, s->tc_frames[w], p->Arows[w], p->Kp64[w], D.a, D.Mrp, B,
                                   s->d_tc_prefix[w], s->d_brow + (size_t)w * B, s->d_sigs, w,
                                   s->total_tc_tiles[w], s->d_err, st, flagged));
        } else if (p->flags & MP_COEF_FP64) {
            CKR(launch_analysis_dgemm(p->d_A64[w], p->Arows[w], p->Akp[w], D.wlen, D.a, D.Mrp, B,
                                      s->d_tile_prefix[w], s->d_sigs, w, s->total_tiles[w], st,
                                      flagged));
        } else {
            CKR(launch_analysis_sgemm(p->d_A[w], p->Arows[w], p->Akp[w], D.wlen, D.a, D.Mrp, B,
                                      s->d_tile_prefix[w], s->d_sigs, w, s->total_tiles[w], st,
                                      flagged));
        }
        CKR(launch_tree_build(p->dp, s->d_sigs, B, s->d_frame_prefix[w], s->total_frames[w], w, st,
                              flagged));
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CKR(cudaStreamIsCapturing(st, &cap));
    if (tc && cap == cudaStreamCaptureStatusNone) {
        // the tensor-core kernel bounds its waits; report an expired wait
        int err = 0;
        CKR(cudaMemcpyAsync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        if (err) {
            mpg_set_error("mp_analyze: a tensor-core analysis wait timed out");
            return MP_ETIMEOUT;
        }
    }
    return MP_OK;
}

int ensure_capacity(mp_state* s, long long kmax) {
    if (kmax <= s->cap) return MP_OK;
    const int B = s->B;
    cudaStream_t st = s->plan->stream;
    long long ncap = std::max(kmax, s->cap * 2);
    mp_atom* na = nullptr;
    double* ne = nullptr;
    CKR(cudaMalloc(&na, sizeof(mp_atom) * ncap * B));
    cudaError_t e = cudaMalloc(&ne, sizeof(double) * ncap * B);
    if (e != cudaSuccess) {
        cudaFree(na);
        return cuda_fail(e, "mp_run: atom buffer");
    }
    if (s->cap > 0) {
        CKR(cudaMemcpy2DAsync(na, sizeof(mp_atom) * ncap, s->d_atoms, sizeof(mp_atom) * s->cap,
                              sizeof(mp_atom) * s->cap, B, cudaMemcpyDeviceToDevice, st));
        CKR(cudaMemcpy2DAsync(ne, sizeof(double) * ncap, s->d_errs, sizeof(double) * s->cap,
                              sizeof(double) * s->cap, B, cudaMemcpyDeviceToDevice, st));
    }
    CKR(cudaStreamSynchronize(st));
    if (s->d_atoms) cudaFree(s->d_atoms);
    if (s->d_errs) cudaFree(s->d_errs);
    s->d_atoms = na;
    s->d_errs = ne;
    s->cap = ncap;
    for (int b = 0; b < B; ++b) {
        s->hs[b].atoms = na + (long long)b * ncap;
        s->hs[b].errs = ne + (long long)b * ncap;
        s->hs[b].cap = ncap;
        // patch only the pointer fields; the dynamic fields live on the device
        char* dst = (char*)(s->d_sigs + b);
        CKR(cudaMemcpyAsync(dst + offsetof(DevSig, atoms), &s->hs[b].atoms,
                            offsetof(DevSig, x) - offsetof(DevSig, atoms), cudaMemcpyHostToDevice,
                            st));
    }
    CKR(cudaStreamSynchronize(st));
    return MP_OK;
}

int read_status(mp_state* s, int64_t* n_atoms, int* stop, double* snr, bool* timed_out,
                std::vector<int>* resets = nullptr) {
    std::vector<DevSig> dv(s->B);
    CKR(cudaMemcpyAsync(dv.data(), s->d_sigs, sizeof(DevSig) * s->B, cudaMemcpyDeviceToHost,
                        s->plan->stream));
    CKR(cudaStreamSynchronize(s->plan->stream));
    if (resets) {
        resets->clear();
        for (int b = 0; b < s->B; ++b)
            if (dv[b].reset_pending) resets->push_back(b);
    }
    for (int b = 0; b < s->B; ++b)
        if (dv[b].bounds) {
            // only a library built with MP_CHECK_BOUNDS records this
            mpg_set_error("bounds check: signal %d, MP-loop access site %d was out of range "
                          "(the access was skipped)", b, dv[b].bounds);
            return MP_ECUDA;
        }
    bool to = false;
    for (int b = 0; b < s->B; ++b) {
        if (n_atoms) n_atoms[b] = dv[b].k;
        if (stop) stop[b] = dv[b].stop;
        if (snr) snr[b] = 10.0 * std::log10(dv[b].E0 / dv[b].E);
        to = to || dv[b].timed_out;
    }
    if (timed_out) *timed_out = to;
    return MP_OK;
}

}  // namespace

extern "C" int mp_analyze(const mp_plan* plan, mp_state** state, int B, const float* const* x_dev,
                          const int64_t* L) {
    mpg::NvtxRange nvtx_range("mp_analyze");
    return analyze_impl(plan, state, B, x_dev, L, cudaMemcpyDeviceToDevice);
}

extern "C" int mp_analyze_host(const mp_plan* plan, mp_state** state, int B,
                               const float* const* x_host, const int64_t* L) {
    mpg::NvtxRange nvtx_range("mp_analyze_host");
    return analyze_impl(plan, state, B, x_host, L, cudaMemcpyHostToDevice);
}

extern "C" int mp_state_coefficients(const mp_state* s, int sig, int w, float* host, int64_t cap) {
    if (!s || sig < 0 || sig >= s->B || w < 0 || w >= s->plan->W || !host) {
        mpg_set_error("mp_state_coefficients: bad argument");
        return MP_EINVAL;
    }
    const DevDict& D = s->plan->dp.d[w];
    const long long N = s->hs[sig].N[w];
    if (cap < 2 * N * D.Mr) {
        mpg_set_error("mp_state_coefficients: buffer too small");
        return MP_EINVAL;
    }
    if (s->plan->flags & MP_COEF_FP64) {
        // FP64 planes: copied as they are, rounded to float on the host
        std::vector<double> tmp((size_t)2 * N * D.Mr);
        CKR(cudaMemcpy2DAsync(tmp.data(), sizeof(double2) * D.Mr, s->hs[sig].plane[w],
                              sizeof(double2) * D.Mrp, sizeof(double2) * D.Mr, N,
                              cudaMemcpyDeviceToHost, s->plan->stream));
        CKR(cudaStreamSynchronize(s->plan->stream));
        for (size_t i = 0; i < tmp.size(); ++i) host[i] = (float)tmp[i];
        return MP_OK;
    }
    CKR(cudaMemcpy2DAsync(host, sizeof(float2) * D.Mr, s->hs[sig].plane[w], sizeof(float2) * D.Mrp,
                          sizeof(float2) * D.Mr, N, cudaMemcpyDeviceToHost, s->plan->stream));
    CKR(cudaStreamSynchronize(s->plan->stream));
    return MP_OK;
}

extern "C" int mp_state_set_time_limit(mp_state* s, double seconds) {
    if (!s || !std::isfinite(seconds)) {
        mpg_set_error("mp_state_set_time_limit: bad argument");
        return MP_EINVAL;
    }
    s->time_limit_s = seconds;
    return MP_OK;
}

extern "C" int mp_run_async(mp_state* s, int64_t K_max, double target_snr_db) {
    mpg::NvtxRange nvtx_range("mp_run_async");
    if (!s || K_max < 0 || std::isnan(target_snr_db)) {
        mpg_set_error("mp_run: bad argument");
        return MP_EINVAL;
    }
    int rc = ensure_capacity(s, std::max<long long>(K_max, 1));
    if (rc) return rc;
    const double thr_scale = std::pow(10.0, -target_snr_db / 10.0);
    const long long budget =
        s->time_limit_s > 0 ? (long long)std::min(s->time_limit_s * 1e9, 9e18) : 0LL;
    const double reset_scale = s->reset_db < 0.0 ? std::pow(10.0, s->reset_db / 10.0) : 0.0;
    CKR(launch_mp_loop(s->plan->dp, s->d_sigs, s->d_order, s->B, K_max, thr_scale, budget,
                       s->shape, s->plan->stream, s->reset_it, reset_scale));
    return MP_OK;
}

// Alg. 2 reset pass for the listed signals: synthesise all atoms so far,
// r = x - y, E = E_out = ||r||^2, re-analyse r
static int reset_pass(mp_state* s, const std::vector<int>& sigs) {
    cudaStream_t st = s->plan->stream;
    const int one = 1;
    for (int b : sigs) {
        CKR(launch_synth(s->plan->dp, s->d_sigs + b, 0, s->hs[b].y, s->L[b], st));
        CKR(cudaMemcpyAsync((char*)(s->d_sigs + b) + offsetof(DevSig, reanalyze), &one, sizeof(int),
                            cudaMemcpyHostToDevice, st));
    }
    CKR(launch_reset_residual(s->d_sigs, s->B, s->d_epart, st));
    int rc = analysis_pass(s, 1);
    if (rc) return rc;
    const int zero = 0;
    for (int b : sigs)
        CKR(cudaMemcpyAsync((char*)(s->d_sigs + b) + offsetof(DevSig, reanalyze), &zero,
                            sizeof(int), cudaMemcpyHostToDevice, st));
    CKR(cudaStreamSynchronize(st));
    return MP_OK;
}

extern "C" int mp_get_status(mp_state* s, int64_t* n_atoms, int* stop, double* snr) {
    if (!s) {
        mpg_set_error("mp_get_status: null state");
        return MP_EINVAL;
    }
    bool to = false;
    int rc = read_status(s, n_atoms, stop, snr, &to);
    if (rc) return rc;
    if (to) {
        mpg_set_error("mp_run: time limit reached before every signal stopped");
        return MP_ETIMEOUT;
    }
    return MP_OK;
}

extern "C" int mp_run(mp_state* s, int64_t K_max, double target_snr_db, int64_t* n_atoms,
                      int* stop_reason, double* final_snr_db) {
    mpg::NvtxRange nvtx_range("mp_run");
    for (;;) {
        int rc = mp_run_async(s, K_max, target_snr_db);
        if (rc) return rc;
        if (s->reset_it <= 0 && s->reset_db >= 0.0) break;
        std::vector<int> pend;
        bool to = false;
        rc = read_status(s, nullptr, nullptr, nullptr, &to, &pend);
        if (rc) return rc;
        if (pend.empty() || to) break;
        rc = reset_pass(s, pend);
        if (rc) return rc;
    }
    return mp_get_status(s, n_atoms, stop_reason, final_snr_db);
}

extern "C" int mp_state_set_launch(mp_state* s, int threads, int cluster) {
    if (!s) {
        mpg_set_error("mp_state_set_launch: null state");
        return MP_EINVAL;
    }
    if (threads == 0 && cluster == 0) {
        LoopShape sh;
        mp_loop_shape(s->plan->dp, s->hs.data(), s->B, s->plan->num_sms, &sh);
        if (sh.threads) s->shape = sh;
        return MP_OK;
    }
    LoopShape sh;
    if (!mp_loop_shape_ok(s->plan->dp, s->hs.data(), s->B, threads, cluster, &sh)) {
        mpg_set_error("mp_state_set_launch: %d threads x cluster %d is not feasible for this "
                      "state", threads, cluster);
        return MP_EINVAL;
    }
    s->shape = sh;
    return MP_OK;
}

extern "C" int mp_state_get_launch(const mp_state* s, int* threads, int* cluster) {
    if (!s) {
        mpg_set_error("mp_state_get_launch: null state");
        return MP_EINVAL;
    }
    if (threads) *threads = s->shape.threads;
    if (cluster) *cluster = s->shape.cs;
    return MP_OK;
}

extern "C" int mp_state_set_top_keys(mp_state* s, int max_keys) {
    if (!s) {
        mpg_set_error("mp_state_set_top_keys: null state");
        return MP_EINVAL;
    }
    if (s->shape.cs != 1) {
        mpg_set_error("mp_state_set_top_keys: the launch runs clusters of %d CTAs; the cap "
                      "applies to one CTA per signal", s->shape.cs);
        return MP_EINVAL;
    }
    LoopShape sh;
    const bool ok =
        max_keys == 0
            ? mp_loop_shape_ok(s->plan->dp, s->hs.data(), s->B, s->shape.threads, 1, &sh)
            : mp_loop_shape_single_cap(s->plan->dp, s->hs.data(), s->B, s->shape.threads,
                                       max_keys, &sh);
    if (!ok) {
        mpg_set_error("mp_state_set_top_keys: %d is not a power of two from 64 to the cap of "
                      "%d-thread CTAs, or the top level does not fit in shared memory",
                      max_keys, s->shape.threads);
        return MP_EINVAL;
    }
    s->shape = sh;
    return MP_OK;
}

extern "C" int mp_state_get_top_keys(const mp_state* s, int* max_keys) {
    if (!s || !max_keys) {
        mpg_set_error("mp_state_get_top_keys: null argument");
        return MP_EINVAL;
    }
    *max_keys = s->shape.cs == 1 ? s->shape.topcap : 0;
    return MP_OK;
}

extern "C" int mp_state_set_work_hint(mp_state* s, const double* work) {
    if (!s) {
        mpg_set_error("mp_state_set_work_hint: null state");
        return MP_EINVAL;
    }
    const int B = s->B;
    if (work)
        for (int b = 0; b < B; ++b)
            if (!(work[b] >= 0.0) || !std::isfinite(work[b])) {
                mpg_set_error("mp_state_set_work_hint: work[%d] must be finite and >= 0", b);
                return MP_EINVAL;
            }
    // launch order: most work first (then the longer signal, then the lower
    // index); without hints the longer signal first
    std::vector<int> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (work && work[x] != work[y]) return work[x] > work[y];
        return s->L[x] > s->L[y];
    });
    CKR(cudaMemcpyAsync(s->d_order, order.data(), sizeof(int) * B, cudaMemcpyHostToDevice,
                        s->plan->stream));
    CKR(cudaStreamSynchronize(s->plan->stream));
    return MP_OK;
}

extern "C" int mp_state_set_resets(mp_state* s, int64_t reset_every, double reset_err_db) {
    if (!s || reset_every < 0 || !(reset_err_db <= 0.0)) {
        mpg_set_error("mp_state_set_resets: need reset_every >= 0 and reset_err_db <= 0");
        return MP_EINVAL;
    }
    s->reset_it = reset_every;
    s->reset_db = reset_err_db;
    return MP_OK;
}

extern "C" int mp_get_atoms(const mp_state* s, int sig, mp_atom* out, int64_t cap, int64_t* n) {
    if (!s || sig < 0 || sig >= s->B) {
        mpg_set_error("mp_get_atoms: bad argument");
        return MP_EINVAL;
    }
    long long k = 0;
    CKR(cudaMemcpyAsync(&k, (const char*)(s->d_sigs + sig) + offsetof(DevSig, k), sizeof(k),
                        cudaMemcpyDeviceToHost, s->plan->stream));
    CKR(cudaStreamSynchronize(s->plan->stream));
    if (n) *n = k;
    long long c = std::min<long long>(k, cap);
    if (c > 0 && out) {
        CKR(cudaMemcpyAsync(out, s->hs[sig].atoms, sizeof(mp_atom) * c, cudaMemcpyDeviceToHost,
                            s->plan->stream));
        CKR(cudaStreamSynchronize(s->plan->stream));
    }
    return MP_OK;
}

extern "C" int mp_get_errors(const mp_state* s, int sig, double* E, int64_t cap, int64_t* n) {
    if (!s || sig < 0 || sig >= s->B) {
        mpg_set_error("mp_get_errors: bad argument");
        return MP_EINVAL;
    }
    long long k = 0;
    CKR(cudaMemcpyAsync(&k, (const char*)(s->d_sigs + sig) + offsetof(DevSig, k), sizeof(k),
                        cudaMemcpyDeviceToHost, s->plan->stream));
    CKR(cudaStreamSynchronize(s->plan->stream));
    if (n) *n = k;
    long long c = std::min<long long>(k, cap);
    if (c > 0 && E) {
        CKR(cudaMemcpyAsync(E, s->hs[sig].errs, sizeof(double) * c, cudaMemcpyDeviceToHost,
                            s->plan->stream));
        CKR(cudaStreamSynchronize(s->plan->stream));
    }
    return MP_OK;
}

extern "C" int mp_synthesize(const mp_state* s, int sig, float* y, double* true_snr_db) {
    mpg::NvtxRange nvtx_range("mp_synthesize");
    if (!s || sig < 0 || sig >= s->B || !y) {
        mpg_set_error("mp_synthesize: bad argument");
        return MP_EINVAL;
    }
    cudaStream_t st = s->plan->stream;
    if (s->cap == 0) {
        // no MP run yet: the approximation is zero
        CKR(cudaMemsetAsync(y, 0, sizeof(float) * s->L[sig], st));
    } else {
        CKR(launch_synth(s->plan->dp, s->d_sigs + sig, 0, y, s->L[sig], st));
    }
    if (true_snr_db) {
        CKR(launch_resid_energy(s->d_sigs + sig, y, s->L[sig], s->d_scalar, 1, st));
        double r = 0.0, e0 = 0.0;
        CKR(cudaMemcpyAsync(&r, s->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
        CKR(cudaMemcpyAsync(&e0, (const char*)(s->d_sigs + sig) + offsetof(DevSig, E0),
                            sizeof(double), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        *true_snr_db = 10.0 * std::log10(e0 / r);
    }
    return MP_OK;
}

extern "C" void mp_state_destroy(mp_state* s) {
    if (!s) return;
    cudaStreamSynchronize(s->plan->stream);
    state_free(s);
}
