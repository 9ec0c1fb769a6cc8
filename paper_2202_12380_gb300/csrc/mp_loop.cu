// Persistent matching-pursuit loop (Alg. 1 with the residual update of
// Alg. 3): one CTA per signal, iterating selection -> real-pair adjustment
// -> energy bookkeeping -> coefficient-domain update of every dictionary ->
// max-tree repair, entirely on the device.
//
// Selection (Sec. 5.1).  The top level of the max tree (one Entry per frame,
// or per group of 2^gshift frames) and a level of "super" entries (one per
// 32 top entries) live in shared memory; warp 0 reduces the supers.  Level 0
// (per frame and 32-bin chunk) and level 1 (per frame) live in global memory
// next to the coefficient planes.
//
// Update (eqs. fastkernupdate, hkj, Alg. 3).  For the selected (u, k, j) and
// each dictionary v, the atom and (for 0 < k < M_u/2) its conjugate partner
// (M_u - k, conj(c)) each hit one dense class tile of h_{u,v}; the tile's
// rows wrap mod M_v and only rows 0..M_v/2 are stored, its columns wrap mod
// N_v.  The work is cut into warp jobs of (frame, 32-bin chunk): each lane
// owns one bin, applies both terms, and the warp recomputes the chunk's
// level-0 entry on the spot.  Frames touched are then re-reduced from level
// 0, groups from level 1, supers from the top level.
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int NWARPS = LOOP_THREADS / 32;

struct Term {
    int active;
    int Arow;   // first tile row, as a bin of dictionary v, in [0, M_v)
    int R;
    int Acol;   // first tile column, as a frame of dictionary v, in [0, N_v)
    int C;
    int kk;     // frequency index (in dictionary u) of this atom
    int tau0;   // tau of tile column 0
    float2 coef;
    const float2* tile;
};

struct VJob {
    Term t[2];
    long long nstart;  // first frame of the column hull (wrapped)
    int ncols;
    int nr;            // chunk ranges [cr0, cr1)
    int cr0[4], cr1[4];
    int nchunks;
    int njobs, jbase;  // update jobs and their prefix
    int fbase;         // prefix of frame jobs
};

struct Shared {
    VJob vj[MAXW];
    Entry win;
    int u, kk;
    long long j;
    int stop;
    int total_jobs, total_frames;
    int S;  // number of supers
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// rows of a term inside the stored range [0, Mr): up to two intervals
__device__ void term_rows(const Term& t, int Mv, int Mr, int* lo, int* hi, int* n) {
    *n = 0;
    int e1 = min(t.Arow + t.R, Mv);
    int a0 = t.Arow, a1 = min(e1, Mr);
    if (a1 > a0) { lo[*n] = a0; hi[*n] = a1; ++*n; }
    if (t.Arow + t.R > Mv) {
        int b1 = min(t.Arow + t.R - Mv, Mr);
        if (b1 > 0) { lo[*n] = 0; hi[*n] = b1; ++*n; }
    }
}

// describe the update of dictionary v for selected (u, k, j) with coefficient c
__device__ void make_vjob(const DevPlan& P, const DevSig& S, int u, int k, long long j, float2 c,
                          bool edge, int v, VJob& J) {
    const DevDict& Du = P.d[u];
    const DevDict& Dv = P.d[v];
    const DevPair& PR = P.p[u * P.W + v];
    const int Mu = Du.M, Mv = Dv.M, au = Du.a, av = Dv.a;
    const long long Nv = S.N[v];
    const int ct = (int)(j % PR.rt);
    const long long base_n = (av <= au) ? j * (au / av) : (j - ct) / PR.rt;
    int rlo[4], rhi[4], nrng = 0;
    long long cmin = 0, cmax = 0;
    bool any = false;
    for (int ti = 0; ti < 2; ++ti) {
        Term& T = J.t[ti];
        T.active = 0;
        if (ti == 1 && edge) continue;
        const int kk = ti == 0 ? k : Mu - k;
        const int cf = kk % PR.rf;
        const long long base_m = (Mv >= Mu) ? (long long)kk * (Mv / Mu) : (kk - cf) / PR.rf;
        const DevClass& C = P.cls[PR.cls_base + cf * PR.rt + ct];
        if (C.R == 0) continue;
        T.Arow = (int)lmod(base_m + C.i_lo, Mv);
        T.R = C.R;
        T.C = C.C;
        T.kk = kk;
        T.tau0 = C.c_lo * av - ct * au;
        T.coef = ti == 0 ? c : make_float2(c.x, -c.y);
        T.tile = P.tiles + C.off;
        int lo[2], hi[2], nn;
        term_rows(T, Mv, Dv.Mr, lo, hi, &nn);
        if (nn == 0) continue;
        T.active = 1;
        for (int q = 0; q < nn; ++q) {
            rlo[nrng] = lo[q] / CHUNK;
            rhi[nrng] = (hi[q] - 1) / CHUNK + 1;
            ++nrng;
        }
        long long a0 = base_n + C.c_lo;
        T.Acol = (int)lmod(a0, Nv);
        if (!any) { cmin = a0; cmax = a0 + C.C; any = true; }
        else { cmin = min(cmin, a0); cmax = max(cmax, a0 + (long long)C.C); }
    }
    J.nr = 0;
    J.nchunks = 0;
    J.ncols = 0;
    J.nstart = 0;
    if (!any) return;
    // merge chunk ranges (at most 4) into disjoint sorted ranges
    for (int a = 1; a < nrng; ++a)
        for (int b = a; b > 0 && rlo[b] < rlo[b - 1]; --b) {
            int t0 = rlo[b]; rlo[b] = rlo[b - 1]; rlo[b - 1] = t0;
            int t1 = rhi[b]; rhi[b] = rhi[b - 1]; rhi[b - 1] = t1;
        }
    for (int a = 0; a < nrng; ++a) {
        if (J.nr > 0 && rlo[a] <= J.cr1[J.nr - 1]) {
            J.cr1[J.nr - 1] = max(J.cr1[J.nr - 1], rhi[a]);
        } else {
            J.cr0[J.nr] = rlo[a];
            J.cr1[J.nr] = rhi[a];
            ++J.nr;
        }
    }
    for (int a = 0; a < J.nr; ++a) J.nchunks += J.cr1[a] - J.cr0[a];
    long long ncols = cmax - cmin;
    if (ncols >= Nv) { J.nstart = 0; J.ncols = (int)Nv; }
    else { J.nstart = lmod(cmin, Nv); J.ncols = (int)ncols; }
}

__device__ __forceinline__ float2 gamma_of(const DevPlan& P, int u, int k) {
    const DevDict& D = P.d[u];
    if (k < D.gam_lo) return P.gam[D.gam_off + k];
    if (k >= D.Mr - D.gam_hi) return P.gam[D.gam_off + D.gam_lo + (k - (D.Mr - D.gam_hi))];
    return make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(LOOP_THREADS, 1)
    k_mp_loop(DevPlan P, DevSig* __restrict__ sigs, const int* __restrict__ order,
              long long kmax, double thr_scale, long long budget_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;
    __shared__ DevSig S;
    DevSig& Sg = sigs[order[blockIdx.x]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int* src = reinterpret_cast<const int*>(&Sg);
        int* dst = reinterpret_cast<int*>(&S);
        for (int i = tid; i < (int)(sizeof(DevSig) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int W = P.W;
    const int T = S.T;
    const int NS = (T + 31) >> 5;
    Entry* top = reinterpret_cast<Entry*>(smem_raw);
    Entry* sup = top + T;
    unsigned char* tdirty = reinterpret_cast<unsigned char*>(sup + NS);
    unsigned char* sdirty = tdirty + T;

    // load the top level and build the supers
    for (int w = 0; w < W; ++w) {
        const int tb = S.tbase[w], te = S.tbase[w + 1];
        const Entry* src = S.gshift == 0 ? S.l1[w] : S.grp + tb;
        for (int i = tid; i < te - tb; i += blockDim.x) top[tb + i] = src[i];
    }
    for (int i = tid; i < T; i += blockDim.x) tdirty[i] = 0;
    for (int i = tid; i < NS; i += blockDim.x) sdirty[i] = 0;
    __syncthreads();
    for (int s = warp; s < NS; s += NWARPS) {
        Entry e;
        int i = s * 32 + lane;
        if (i < T) e = top[i]; else { e.key = 0; e.val = make_float2(0.f, 0.f); }
        Entry r = warp_max_entry(e);
        if (lane == 0) sup[s] = r;
    }
    if (tid == 0) sh.S = NS;
    __syncthreads();

    long long k = S.k;
    double E = S.E;
    const double E0 = S.E0;
    const double thr = E0 * thr_scale;
    const unsigned long long t_start = gtimer();

    for (;;) {
        // ---- selection, adjustment, bookkeeping (warp 0) ----------------
        if (warp == 0) {
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            for (int i = lane; i < NS; i += 32) {
                Entry e = sup[i];
                if (e.key > b.key) b = e;
            }
            Entry best = warp_max_entry(b);
            int stop = 0;
            if (!isfinite(E0)) stop = MP_STOP_INVALID;
            else if (E <= 0.0) stop = MP_STOP_NEGENERGY;
            else if (E <= thr) stop = MP_STOP_SNR;
            else if (k >= kmax) stop = MP_STOP_KMAX;
            else if (budget_ns > 0 && (long long)(gtimer() - t_start) > budget_ns) stop = -1;
            else if ((unsigned)(best.key >> 32) == 0u) stop = MP_STOP_ZEROMAX;
            int u = 0, kk = 0;
            long long j = 0;
            float2 c = make_float2(0.f, 0.f);
            bool edge = false;
            if (stop == 0) {
                const unsigned flat = 0xffffffffu - (unsigned)(best.key & 0xffffffffull);
                while (u + 1 < W && S.fbase[u + 1] <= flat) ++u;
                const int Mr = P.d[u].Mr;
                const unsigned rel = flat - S.fbase[u];
                j = rel / (unsigned)Mr;
                kk = (int)(rel - (unsigned)j * (unsigned)Mr);
                const int Mu = P.d[u].M;
                edge = (kk == 0) || (2 * kk == Mu);
                // eqs. dualatprod / projenfaster in FP64
                double rx = best.val.x, ry = best.val.y, cx, cy, Ed;
                if (edge) {
                    cx = rx;
                    cy = 0.0;
                    Ed = rx * rx;
                } else {
                    float2 g = gamma_of(P, u, kk);
                    double gx = g.x, gy = g.y;
                    double den = 1.0 - (gx * gx + gy * gy);
                    // rho - conj(gamma) conj(rho)
                    double nx = rx - (gx * rx + gy * ry);
                    double ny = ry - (gy * rx - gx * ry);
                    cx = nx / den;
                    cy = ny / den;
                    Ed = 2.0 * (cx * cx + cy * cy + gx * (cx * cx - cy * cy) - 2.0 * gy * cx * cy);
                }
                E -= Ed;
                c = make_float2((float)cx, (float)cy);
                if (lane == 0) {
                    mp_atom at;
                    at.dict = u;
                    at.m = kk;
                    at.n = j;
                    at.re = c.x;
                    at.im = c.y;
                    S.atoms[k] = at;
                    S.errs[k] = E;
                }
            }
            if (lane < W && stop == 0) make_vjob(P, S, u, kk, j, c, edge, lane, sh.vj[lane]);
            __syncwarp();
            if (lane == 0) {
                sh.stop = stop;
                sh.u = u;
                sh.kk = kk;
                sh.j = j;
                int jb = 0, fb = 0;
                if (stop == 0)
                    for (int v = 0; v < W; ++v) {
                        VJob& J = sh.vj[v];
                        J.njobs = J.ncols * J.nchunks;
                        J.jbase = jb;
                        J.fbase = fb;
                        jb += J.njobs;
                        fb += J.nchunks > 0 ? J.ncols : 0;
                    }
                sh.total_jobs = jb;
                sh.total_frames = fb;
            }
        }
        __syncthreads();
        if (sh.stop) break;
        ++k;

        // ---- coefficient-domain update + level 0 -------------------------
        const int tj = sh.total_jobs;
        for (int g = warp; g < tj; g += NWARPS) {
            int v = 0;
            while (v + 1 < W && sh.vj[v + 1].jbase <= g) ++v;
            const VJob& J = sh.vj[v];
            const DevDict& Dv = P.d[v];
            const long long Nv = S.N[v];
            const int local = g - J.jbase;
            const int col = local / J.nchunks;
            int ci = local - col * J.nchunks;
            int r = 0;
            while (ci >= J.cr1[r] - J.cr0[r]) { ci -= J.cr1[r] - J.cr0[r]; ++r; }
            const int chunk = J.cr0[r] + ci;
            const long long n = lmod(J.nstart + col, Nv);
            const int m = chunk * CHUNK + lane;
            float2* p = S.plane[v] + n * Dv.Mrp + m;
            float2 val = *p;
            bool mod = false;
            if (m < Dv.Mr) {
#pragma unroll
                for (int ti = 0; ti < 2; ++ti) {
                    const Term& T = J.t[ti];
                    if (!T.active) continue;
                    long long cc = n - T.Acol;
                    if (cc < 0) cc += Nv;
                    if (cc >= T.C) continue;
                    int i = m - T.Arow;
                    if (i < 0) i += Dv.M;
                    if (i >= T.R) continue;
                    const float2 h = __ldg(T.tile + cc * T.R + i);
                    // modulation of eq. hkj for this column: e^{i 2 pi kk tau / M_u}
                    const int Mu = P.d[sh.u].M;
                    const long long tau = T.tau0 + cc * Dv.a;
                    const long long q = lmod((long long)T.kk * tau, Mu);
                    float sn, cs;
                    sincospif(2.0f * (float)q / (float)Mu, &sn, &cs);
                    const float2 ph = make_float2(cs, sn);
                    const float2 d = cmul(T.coef, cmul(ph, h));
                    val.x -= d.x;
                    val.y -= d.y;
                    mod = true;
                }
            }
            if (mod) *p = val;
            Entry e;
            e.val = val;
            e.key = (m < Dv.Mr) ? make_key(val, S.fbase[v] + (unsigned)(n * Dv.Mr) + m) : 0ull;
            Entry rr = warp_max_entry(e);
            if (lane == 0) S.l0[v][n * Dv.nch + chunk] = rr;
        }
        __syncthreads();

        // ---- level 1 of touched frames -----------------------------------
        const int tf = sh.total_frames;
        for (int g = warp; g < tf; g += NWARPS) {
            // last dictionary whose prefix is <= g (it always has frames)
            int v = 0;
            while (v + 1 < W && sh.vj[v + 1].fbase <= g) ++v;
            const VJob& J = sh.vj[v];
            const DevDict& Dv = P.d[v];
            const long long n = lmod(J.nstart + (g - J.fbase), S.N[v]);
            const Entry* l0 = S.l0[v] + n * Dv.nch;
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            for (int c = lane; c < Dv.nch; c += 32) {
                Entry e = l0[c];
                if (e.key > b.key) b = e;
            }
            Entry r = warp_max_entry(b);
            if (lane == 0) {
                S.l1[v][n] = r;
                if (S.gshift == 0) {
                    const int ti = S.tbase[v] + (int)n;
                    top[ti] = r;
                    sdirty[ti >> 5] = 1;
                } else {
                    tdirty[S.tbase[v] + (int)(n >> S.gshift)] = 1;
                }
            }
        }
        __syncthreads();

        // ---- level 2 (groups) of touched frames --------------------------
        if (S.gshift > 0) {
            for (int base = warp * 32; base < T; base += NWARPS * 32) {
                const int i = base + lane;
                unsigned ball = __ballot_sync(FULL, i < T && tdirty[i]);
                while (ball) {
                    const int b = __ffs(ball) - 1;
                    ball &= ball - 1;
                    const int gi = base + b;
                    int w = 0;
                    while (w + 1 < W && S.tbase[w + 1] <= gi) ++w;
                    const long long f0 = (long long)(gi - S.tbase[w]) << S.gshift;
                    const long long f1 = min(f0 + (1ll << S.gshift), S.N[w]);
                    Entry bb;
                    bb.key = 0;
                    bb.val = make_float2(0.f, 0.f);
                    for (long long f = f0 + lane; f < f1; f += 32) {
                        Entry e = S.l1[w][f];
                        if (e.key > bb.key) bb = e;
                    }
                    Entry r = warp_max_entry(bb);
                    if (lane == 0) {
                        S.grp[gi] = r;
                        top[gi] = r;
                        tdirty[gi] = 0;
                        sdirty[gi >> 5] = 1;
                    }
                }
            }
            __syncthreads();
        }

        // ---- supers --------------------------------------------------------
        for (int base = warp * 32; base < NS; base += NWARPS * 32) {
            const int i = base + lane;
            unsigned ball = __ballot_sync(FULL, i < NS && sdirty[i]);
            while (ball) {
                const int b = __ffs(ball) - 1;
                ball &= ball - 1;
                const int s = base + b;
                const int ti = s * 32 + lane;
                Entry e;
                if (ti < T) e = top[ti]; else { e.key = 0; e.val = make_float2(0.f, 0.f); }
                Entry r = warp_max_entry(e);
                if (lane == 0) {
                    sup[s] = r;
                    sdirty[s] = 0;
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        Sg.k = k;
        Sg.E = E;
        if (sh.stop > 0) {
            Sg.stop = sh.stop;
            Sg.timed_out = 0;
        } else {
            Sg.stop = 0;
            Sg.timed_out = 1;
        }
    }
}

}  // namespace

size_t mp_loop_smem_bytes(int T, int) {
    const int NS = (T + 31) / 32;
    size_t b = (size_t)(T + NS) * sizeof(Entry) + (size_t)T + (size_t)NS;
    return (b + 15) & ~(size_t)15;
}

cudaError_t launch_mp_loop(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig,
                           long long kmax, double thr_scale, long long budget_ns, size_t smem,
                           cudaStream_t st) {
    if (nsig <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mp_loop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_mp_loop<<<nsig, LOOP_THREADS, smem, st>>>(P, d_sigs, d_order, kmax, thr_scale, budget_ns);
    return cudaGetLastError();
}

}  // namespace mpg
