// Persistent matching-pursuit loop (Alg. 1 with the residual update of
// Alg. 3): one CTA per signal, iterating selection -> real-pair adjustment
// -> energy bookkeeping -> coefficient-domain update of every dictionary ->
// max-tree repair, entirely on the device.
//
// Max tree (Sec. 5.1).  Level 0 (per frame and 32-bin chunk) and level 1
// (per frame) live in global memory next to the coefficient planes; the top
// level (one Entry per frame, or per group of 2^gshift frames) lives in
// shared memory and is scanned by the whole CTA every iteration (a few
// shared loads per thread), so there is no further level to maintain.
//
// One iteration, for every warp of the CTA:
//   1. scan the top level, warp-reduce, publish the warp's best; barrier;
//   2. reduce the per-warp bests (every warp redundantly), apply the stop
//      tests, adjust the selected coefficient to the real-pair coefficient
//      (eqs. dualatprod / projenfaster), accumulate E in FP64 and describe
//      the update of every dictionary: lane 2v + t builds term t (0: the
//      atom, 1: its conjugate partner) of dictionary v;
//   3. run frame jobs: for each touched frame of each dictionary, load the
//      frame's level-0 entries together with the touched 32-bin chunks of the
//      plane and the matching class-tile entries (one round of independent
//      loads), subtract both terms (eq. fastkernupdate with the modulation of
//      eq. hkj), recompute the touched chunks' level-0 entries, the frame's
//      level-1 entry and its top-level slot; barrier.
// Every warp computes the same selection; thread 0 alone writes the atom list
// and keeps the FP64 energy E, whose stop tests it publishes for the next
// iteration before the closing barrier.
//
// Clusters.  A signal may be given a thread-block cluster of CS CTAs (on CS
// SMs) instead of one CTA: frame n of every dictionary belongs to CTA
// n mod CS, which holds its top-level entry and runs its frame jobs.  In step
// 1 each warp pushes its best candidate into every CTA's shared memory
// (distributed shared memory) and the cluster barrier replaces the CTA
// barrier; every CTA then takes the same selection.  The time limit is
// decided by CTA 0 and pushed the same way, so all CTAs leave the loop in the
// same iteration.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int MAXL0 = 4;   // level-0 entries held per lane (larger frames loop)
constexpr int CB = 4;      // touched chunks processed per batch of loads

// one term (the atom or its conjugate partner) of the update of dictionary v
struct Term {
    int active;
    int Arow;   // first tile row, as a bin of dictionary v, in [0, M_v)
    int R;
    int Acol;   // first tile column, as a frame of dictionary v, in [0, N_v)
    int C;
    int kk;     // frequency index (in dictionary u) of this atom
    int tau0;   // tau of tile column 0
    int a0;     // unwrapped first column (for the column hull)
    long long tile;  // float2 offset of the class tile
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int imod(int x, int m) {
    int r = x % m;
    return r < 0 ? r + m : r;
}

__device__ __forceinline__ Term shfl_term(const Term& t, int src) {
    Term r;
    r.active = __shfl_sync(FULL, t.active, src);
    r.Arow = __shfl_sync(FULL, t.Arow, src);
    r.R = __shfl_sync(FULL, t.R, src);
    r.Acol = __shfl_sync(FULL, t.Acol, src);
    r.C = __shfl_sync(FULL, t.C, src);
    r.kk = __shfl_sync(FULL, t.kk, src);
    r.tau0 = __shfl_sync(FULL, t.tau0, src);
    r.a0 = __shfl_sync(FULL, t.a0, src);
    r.tile = __shfl_sync(FULL, t.tile, src);
    return r;
}

// term t of dictionary v for the selected (u, k, j)
__device__ __forceinline__ Term make_term(const DevDict* sd, const DevPair* sp,
                                          const DevClass* scls, int W, const DevSig& S, int u,
                                          int k, int j, bool edge, int v, int t) {
    Term T;
    T.active = 0;
    T.Arow = T.R = T.Acol = T.C = T.kk = T.tau0 = T.a0 = 0;
    T.tile = 0;
    if (t == 1 && edge) return T;
    const DevDict& Du = sd[u];
    const DevDict& Dv = sd[v];
    const DevPair& PR = sp[u * W + v];
    const int Mu = Du.M, Mv = Dv.M, au = Du.a, av = Dv.a;
    const int kk = t == 0 ? k : Mu - k;
    const int ct = PR.rt_sh >= 0 ? (j & (PR.rt - 1)) : j % PR.rt;
    const int cf = PR.rf_sh >= 0 ? (kk & (PR.rf - 1)) : kk % PR.rf;
    const DevClass& C = scls[PR.cls_base + cf * PR.rt + ct];
    if (C.R == 0) return T;
    const int base_m = PR.mratio ? kk * PR.mratio
                                 : (PR.rf_sh >= 0 ? (kk - cf) >> PR.rf_sh : (kk - cf) / PR.rf);
    const int base_n = PR.aratio ? j * PR.aratio
                                 : (PR.rt_sh >= 0 ? (j - ct) >> PR.rt_sh : (j - ct) / PR.rt);
    T.Arow = Dv.Mmask ? ((base_m + C.i_lo) & Dv.Mmask) : imod(base_m + C.i_lo, Mv);
    T.R = C.R;
    // any stored row (0 .. M_v/2) inside [Arow, Arow + R) mod M_v ?
    const bool rows = (T.Arow < Dv.Mr) || (T.Arow + T.R > Mv);
    if (!rows) return T;
    T.active = 1;
    T.C = C.C;
    T.kk = kk;
    T.tau0 = C.c_lo * av - ct * au;
    T.a0 = base_n + C.c_lo;
    T.Acol = S.Nmask[v] ? (T.a0 & S.Nmask[v]) : imod(T.a0, (int)S.N[v]);
    T.tile = C.off;
    return T;
}

// chunk ranges [lo, hi) of a term's stored rows: up to two
__device__ __forceinline__ int term_chunks(const Term& t, int Mv, int Mr, int* lo, int* hi) {
    if (!t.active) return 0;
    int n = 0;
    const int e1 = min(min(t.Arow + t.R, Mv), Mr);
    if (e1 > t.Arow) { lo[n] = t.Arow / CHUNK; hi[n] = (e1 - 1) / CHUNK + 1; ++n; }
    if (t.Arow + t.R > Mv) {
        const int b1 = min(t.Arow + t.R - Mv, Mr);
        if (b1 > 0) { lo[n] = 0; hi[n] = (b1 - 1) / CHUNK + 1; ++n; }
    }
    return n;
}

__device__ __forceinline__ bool term_hit(const Term& T, int m, int n, int Mv, int Nv, int* off) {
    if (!T.active) return false;
    int cc = n - T.Acol;
    if (cc < 0) cc += Nv;
    if (cc >= T.C) return false;
    int i = m - T.Arow;
    if (i < 0) i += Mv;
    if (i >= T.R) return false;
    *off = cc * T.R + i;
    return true;
}

__device__ __forceinline__ float2 term_phase(const Term& T, int n, int Nv, int av, int Mu,
                                             int Mumask) {
    int cc = n - T.Acol;
    if (cc < 0) cc += Nv;
    const int tau = T.tau0 + cc * av;
    unsigned q;
    if (Mumask) {
        q = ((unsigned)T.kk * ((unsigned)tau & (unsigned)Mumask)) & (unsigned)Mumask;
    } else {
        const unsigned tm = (unsigned)imod(tau, Mu);
        q = ((unsigned)T.kk * tm) % (unsigned)Mu;
    }
    float sn, cs;
    sincospif(2.0f * (float)q / (float)Mu, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ float2 gamma_of(const DevDict& D, const float2* sgam, int k) {
    if (k < D.gam_lo) return sgam[D.gam_off + k];
    if (k >= D.Mr - D.gam_hi) return sgam[D.gam_off + D.gam_lo + (k - (D.Mr - D.gam_hi))];
    return make_float2(0.f, 0.f);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_mp_loop(DevPlan P, DevSig* __restrict__ sigs, const int* __restrict__ order,
              long long kmax, double thr_scale, long long budget_ns, int CS) {
    namespace cg = cooperative_groups;
    constexpr int NWARPS = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevSig S;
    __shared__ DevDict sd[MAXW];
    __shared__ DevPair sp[MAXW * MAXW];
    __shared__ int sstop[2];  // stop decision per iteration parity
    __shared__ int cflag[2];  // time-limit decision of CTA 0, per parity
    __shared__ int ltb[MAXW + 1];  // local top-level base per dictionary
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = CS > 1 ? (int)cluster.block_rank() : 0;
    DevSig& Sg = sigs[order[blockIdx.x / CS]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int* src = reinterpret_cast<const int*>(&Sg);
        int* dst = reinterpret_cast<int*>(&S);
        for (int i = tid; i < (int)(sizeof(DevSig) / sizeof(int)); i += NT) dst[i] = src[i];
    }
    const int W = P.W;
    for (int i = tid; i < W; i += NT) sd[i] = P.d[i];
    for (int i = tid; i < W * W; i += NT) sp[i] = P.p[i];
    __syncthreads();
    // top level of this CTA: all frames (CS == 1, with frame groups when
    // 2^gshift > 1) or the frames n = rank (mod CS) (CS > 1, gshift == 0)
    if (tid == 0) {
        int b = 0;
        for (int w = 0; w < W; ++w) {
            ltb[w] = b;
            b += CS > 1 ? (int)(S.N[w] / CS) : S.tbase[w + 1] - S.tbase[w];
        }
        ltb[W] = b;
        cflag[0] = cflag[1] = 0;
    }
    __syncthreads();
    const int T = ltb[W];
    const int NC = CS * NWARPS;  // candidates exchanged per iteration
    Entry* cand = reinterpret_cast<Entry*>(smem_raw);           // [2][NC]
    Entry* top = cand + 2 * NC;
    DevClass* scls = reinterpret_cast<DevClass*>(top + T);
    float2* sgam = reinterpret_cast<float2*>(scls + P.ncls);
    unsigned char* tdirty = reinterpret_cast<unsigned char*>(sgam + P.ngam);

    for (int i = tid; i < P.ncls; i += NT) scls[i] = P.cls[i];
    for (int i = tid; i < P.ngam; i += NT) sgam[i] = P.gam[i];
    for (int w = 0; w < W; ++w) {
        const int tb = ltb[w], te = ltb[w + 1];
        if (CS > 1) {
            for (int i = tid; i < te - tb; i += NT) top[tb + i] = S.l1[w][(long long)i * CS + rank];
        } else {
            const Entry* src = S.gshift == 0 ? S.l1[w] : S.grp + S.tbase[w];
            for (int i = tid; i < te - tb; i += NT) top[tb + i] = src[i];
        }
    }
    for (int i = tid; i < T; i += NT) tdirty[i] = 0;
    if (CS > 1) cluster.sync(); else __syncthreads();

    long long k = S.k;
    // FP64 work stays in thread 0 (the FP64 pipe is narrow on this part):
    // E, and the stop tests that read it, are evaluated there one iteration
    // ahead and published in sstop
    double E = S.E;
    const double E0 = S.E0;
    const double thr = E0 * thr_scale;
    const unsigned long long t_start = gtimer();
    const float2* __restrict__ tiles = P.tiles;
    int stop = 0;
    if (tid == NT - 32) {
        int s0 = 0;
        if (!isfinite(E0)) s0 = MP_STOP_INVALID;
        else if (E <= 0.0) s0 = MP_STOP_NEGENERGY;
        else if (E <= thr) s0 = MP_STOP_SNR;
        else if (k >= kmax) s0 = MP_STOP_KMAX;
        sstop[k & 1] = s0;
    }
    __syncthreads();

    for (;;) {
        // ---- 1. scan of the top level ------------------------------------
        {
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            for (int i = tid; i < T; i += NT) {
                const Entry e = top[i];
                if (e.key > b.key) b = e;
            }
            const Entry r = warp_max_entry(b);
            Entry* slot = cand + (k & 1) * NC + rank * NWARPS + warp;
            // the time limit is read once per iteration by one thread (of CTA
            // 0) so that every warp of every CTA takes the same decision
            if (CS > 1) {
                if (lane < CS) {
                    Entry* rs = static_cast<Entry*>(__cluster_map_shared_rank(slot, lane));
                    *rs = r;
                }
            } else if (lane == 0) {
                *slot = r;
            }
            if (budget_ns > 0 && rank == 0 && warp == 0) {
                int tflag = 0;
                if (lane == 0) tflag = (long long)(gtimer() - t_start) > budget_ns ? 1 : 0;
                tflag = __shfl_sync(FULL, tflag, 0);
                if (lane < CS) {
                    int* rf = CS > 1 ? static_cast<int*>(__cluster_map_shared_rank(&cflag[k & 1], lane))
                                     : &cflag[k & 1];
                    *rf = tflag;
                }
            }
        }
        if (CS > 1) cluster.sync(); else __syncthreads();

        // ---- 2. selection, adjustment, update description (every warp) --
        Entry best;
        {
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            const Entry* cb = cand + (k & 1) * NC;
            for (int i = lane; i < NC; i += 32) {
                const Entry e = cb[i];
                if (e.key > b.key) b = e;
            }
            best = warp_max_entry(b);
        }
        stop = sstop[k & 1];
        if (stop == 0 && cflag[k & 1]) stop = -1;
        if (stop == 0 && (unsigned)(best.key >> 32) == 0u) stop = MP_STOP_ZEROMAX;
        if (stop) break;

        const unsigned flat = 0xffffffffu - (unsigned)(best.key & 0xffffffffull);
        int u = 0;
        while (u + 1 < W && S.fbase[u + 1] <= flat) ++u;
        const unsigned rel = flat - S.fbase[u];
        const int j = (int)(rel >> sd[u].msh);
        const int kk = (int)(rel & ((1u << sd[u].msh) - 1u));
        const int Mu = sd[u].M;
        const int Mumask = sd[u].Mmask;
        const bool edge = (kk == 0) || (2 * kk == Mu);
        // eqs. dualatprod / projenfaster: coefficient and energy drop in FP32
        // (gamma is zero away from m = 0 and m = M/2), E accumulated in FP64
        const float rx = best.val.x, ry = best.val.y;
        float cx, cy, Edf;
        if (edge) {
            cx = rx;
            cy = 0.f;
            Edf = rx * rx;
        } else {
            const float2 g = gamma_of(sd[u], sgam, kk);
            if (g.x == 0.f && g.y == 0.f) {
                cx = rx;
                cy = ry;
                Edf = 2.f * fmaf(cx, cx, cy * cy);
            } else {
                const float inv = 1.f / (1.f - fmaf(g.x, g.x, g.y * g.y));
                cx = (rx - fmaf(g.x, rx, g.y * ry)) * inv;   // rho - conj(gamma) conj(rho)
                cy = (ry - fmaf(g.y, rx, -g.x * ry)) * inv;
                const float c2 = fmaf(cx, cx, cy * cy), d2 = fmaf(cx, cx, -cy * cy);
                Edf = 2.f * (c2 + fmaf(g.x, d2, -2.f * g.y * cx * cy));
            }
        }
        // bookkeeping (FP64 energy, atom list, next stop decision) in lane 0 of
        // the last warp, which the frame jobs reach last
        const bool keeper = (tid == NT - 32);
        if (keeper) {
            E -= (double)Edf;
        }
        if (keeper && rank == 0) {
            mp_atom at;
            at.dict = u;
            at.m = kk;
            at.n = j;
            at.re = cx;
            at.im = cy;
            S.atoms[k] = at;
            S.errs[k] = E;
        }
        if (keeper) {
            int s1 = 0;  // stop tests before the next selection
            if (E <= 0.0) s1 = MP_STOP_NEGENERGY;
            else if (E <= thr) s1 = MP_STOP_SNR;
            else if (k + 1 >= kmax) s1 = MP_STOP_KMAX;
            sstop[(k + 1) & 1] = s1;
        }
        ++k;
        const float2 c_main = make_float2(cx, cy), c_conj = make_float2(cx, -cy);
        // lane 2v + t describes term t of dictionary v
        Term mine;
        {
            const int v = lane >> 1, t = lane & 1;
            if (v < W) {
                mine = make_term(sd, sp, scls, W, S, u, kk, j, edge, v, t);
            } else {
                mine.active = 0;
                mine.Arow = mine.R = mine.Acol = mine.C = mine.kk = mine.tau0 = mine.a0 = 0;
                mine.tile = 0;
            }
        }
        // frame counts per dictionary: column hull of its active terms
        int nframes = 0, nstart = 0;  // meaningful in lanes 2v
        {
            const int oa = __shfl_xor_sync(FULL, mine.active, 1);
            const int oa0 = __shfl_xor_sync(FULL, mine.a0, 1);
            const int oc = __shfl_xor_sync(FULL, mine.C, 1);
            if ((lane & 1) == 0 && (lane >> 1) < W) {
                int lo = 0, hi = 0;
                bool any = false;
                if (mine.active) { lo = mine.a0; hi = mine.a0 + mine.C; any = true; }
                if (oa) {
                    if (any) { lo = min(lo, oa0); hi = max(hi, oa0 + oc); }
                    else { lo = oa0; hi = oa0 + oc; any = true; }
                }
                if (any) {
                    const int Nv = (int)S.N[lane >> 1];
                    const int nc = hi - lo;
                    if (nc >= Nv) { nstart = 0; nframes = Nv; }
                    else { nstart = imod(lo, Nv); nframes = nc; }
                    // frames of the hull owned by this CTA: i = i0, i0 + CS, ...
                    const int i0 = imod(rank - nstart, CS);
                    nstart += i0;  // first owned frame (may reach N_v: wrapped below)
                    nframes = nframes > i0 ? (nframes - i0 + CS - 1) / CS : 0;
                }
            }
        }
        // inclusive prefix of frame counts over v (held in lanes 0, 2, 4, ...)
        int pre = nframes;
#pragma unroll
        for (int o = 2; o < 2 * MAXW; o <<= 1) {
            const int x = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += x;
        }
        const int total = __shfl_sync(FULL, pre, 2 * W - 2);

        // ---- 3. frame jobs -------------------------------------------------
        for (int g = warp; g < total; g += NWARPS) {
            // dictionary: number of inclusive prefixes <= g
            int v = 0;
            for (int q = 0; q < W; ++q) {
                const int pq = __shfl_sync(FULL, pre, 2 * q);
                v += (pq <= g) ? 1 : 0;
            }
            const int pv = __shfl_sync(FULL, pre, 2 * v);
            const int fv = __shfl_sync(FULL, nframes, 2 * v);
            const int sv = __shfl_sync(FULL, nstart, 2 * v);
            const Term t0 = shfl_term(mine, 2 * v);
            const Term t1 = shfl_term(mine, 2 * v + 1);
            const DevDict& Dv = sd[v];
            const int Nv = (int)S.N[v];
            int n = sv + (g - (pv - fv)) * CS;
            if (n >= Nv) n -= Nv;
            // level-0 entries of the whole frame (untouched chunks keep theirs)
            const Entry* l0row = S.l0[v] + (long long)n * Dv.nch;
            Entry l0v[MAXL0];
#pragma unroll
            for (int q = 0; q < MAXL0; ++q) {
                const int c = lane + 32 * q;
                if (c < Dv.nch) l0v[q] = l0row[c];
            }
            // chunk list: the atom's ranges, then the partner's outside them
            int lo[4], hi[4];
            const int nr0 = term_chunks(t0, Dv.M, Dv.Mr, lo, hi);
            const int nr1 = term_chunks(t1, Dv.M, Dv.Mr, lo + nr0, hi + nr0);
            const int nr = nr0 + nr1;
            float2* prow = S.plane[v] + (long long)n * Dv.Mrp;
            const float2 w0 =
                t0.active ? cmul(c_main, term_phase(t0, n, Nv, Dv.a, Mu, Mumask)) : make_float2(0.f, 0.f);
            const float2 w1 =
                t1.active ? cmul(c_conj, term_phase(t1, n, Nv, Dv.a, Mu, Mumask)) : make_float2(0.f, 0.f);
            Entry fmax;
            fmax.key = 0;
            fmax.val = make_float2(0.f, 0.f);
            // walk the chunks of ranges 0..nr-1, skipping partner chunks that
            // the atom's ranges already cover
            int r = 0, c = nr > 0 ? lo[0] : 0;
            while (r < nr) {
                int chunk[CB];
                int cnt = 0;
                while (cnt < CB && r < nr) {
                    bool dup = false;
                    if (r >= nr0)
                        for (int q = 0; q < nr0; ++q) dup |= (c >= lo[q] && c < hi[q]);
                    if (!dup) chunk[cnt++] = c;
                    if (++c >= hi[r]) {
                        ++r;
                        if (r < nr) c = lo[r];
                    }
                }
                float2 val[CB], h0[CB], h1[CB];
                bool hit0[CB], hit1[CB];
#pragma unroll
                for (int q = 0; q < CB; ++q) {
                    hit0[q] = hit1[q] = false;
                    if (q < cnt) {
                        const int m = chunk[q] * CHUNK + lane;
                        val[q] = prow[m];
                        int off;
                        if (m < Dv.Mr) {
                            if (term_hit(t0, m, n, Dv.M, Nv, &off)) {
                                hit0[q] = true;
                                h0[q] = __ldg(tiles + t0.tile + off);
                            }
                            if (term_hit(t1, m, n, Dv.M, Nv, &off)) {
                                hit1[q] = true;
                                h1[q] = __ldg(tiles + t1.tile + off);
                            }
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < CB; ++q) {
                    if (q >= cnt) continue;
                    const int m = chunk[q] * CHUNK + lane;
                    float2 x2 = val[q];
                    if (hit0[q]) {
                        const float2 d = cmul(w0, h0[q]);
                        x2.x -= d.x;
                        x2.y -= d.y;
                    }
                    if (hit1[q]) {
                        const float2 d = cmul(w1, h1[q]);
                        x2.x -= d.x;
                        x2.y -= d.y;
                    }
                    if (hit0[q] || hit1[q]) prow[m] = x2;
                    Entry e;
                    e.val = x2;
                    e.key = (m < Dv.Mr) ? make_key(x2, S.fbase[v] + ((unsigned)n << Dv.msh) + m) : 0ull;
                    const Entry rr = warp_max_entry(e);
                    if (lane == 0) S.l0[v][(long long)n * Dv.nch + chunk[q]] = rr;
                    if (rr.key > fmax.key) fmax = rr;
                }
            }
            // frame maximum: untouched chunks from level 0, touched ones recomputed
            Entry b = fmax;
#pragma unroll
            for (int q = 0; q < MAXL0; ++q) {
                const int cq = lane + 32 * q;
                bool touched = false;
                for (int z = 0; z < nr; ++z) touched |= (cq >= lo[z] && cq < hi[z]);
                if (cq < Dv.nch && !touched && l0v[q].key > b.key) b = l0v[q];
            }
            for (int cq = lane + 32 * MAXL0; cq < Dv.nch; cq += 32) {
                bool touched = false;
                for (int z = 0; z < nr; ++z) touched |= (cq >= lo[z] && cq < hi[z]);
                if (touched) continue;
                const Entry e = l0row[cq];
                if (e.key > b.key) b = e;
            }
            const Entry fr = warp_max_entry(b);
            if (lane == 0) {
                S.l1[v][n] = fr;
                if (CS > 1) top[ltb[v] + n / CS] = fr;
                else if (S.gshift == 0) top[ltb[v] + n] = fr;
                else tdirty[ltb[v] + (n >> S.gshift)] = 1;
            }
        }
        __syncthreads();

        // ---- level 2 (groups) of touched frames --------------------------
        if (CS == 1 && S.gshift > 0) {
            for (int base = warp * 32; base < T; base += NWARPS * 32) {
                const int i = base + lane;
                unsigned ball = __ballot_sync(FULL, i < T && tdirty[i]);
                while (ball) {
                    const int bb = __ffs(ball) - 1;
                    ball &= ball - 1;
                    const int gi = base + bb;
                    int w = 0;
                    while (w + 1 < W && S.tbase[w + 1] <= gi) ++w;
                    const int f0 = (gi - S.tbase[w]) << S.gshift;
                    const int f1 = min(f0 + (1 << S.gshift), (int)S.N[w]);
                    Entry m2;
                    m2.key = 0;
                    m2.val = make_float2(0.f, 0.f);
                    for (int f = f0 + lane; f < f1; f += 32) {
                        const Entry e = S.l1[w][f];
                        if (e.key > m2.key) m2 = e;
                    }
                    const Entry gr = warp_max_entry(m2);
                    if (lane == 0) {
                        S.grp[gi] = gr;
                        top[gi] = gr;
                        tdirty[gi] = 0;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (CS > 1) cluster.sync();  // no CTA leaves while others may address it
    if (tid == NT - 32 && rank == 0) {
        Sg.k = k;
        Sg.E = E;
        if (stop > 0) {
            Sg.stop = stop;
            Sg.timed_out = 0;
        } else {
            Sg.stop = 0;
            Sg.timed_out = 1;
        }
    }
}

template <int NT>
cudaError_t launch_nt(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig, long long kmax,
                      double thr_scale, long long budget_ns, size_t smem, int cs, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_mp_loop<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(k_mp_loop<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nsig * cs));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_mp_loop<NT>, P, d_sigs, d_order, kmax, thr_scale, budget_ns, cs);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int NT>
int max_clusters(int cs, size_t smem) {
    if (cs > 8 &&
        cudaFuncSetAttribute(k_mp_loop<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
        return 0;
    if (cudaFuncSetAttribute(k_mp_loop<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_mp_loop<NT>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

size_t mp_loop_smem_bytes(const DevPlan& P, int T, int threads, int cs) {
    size_t b = (size_t)2 * cs * (threads / 32) * sizeof(Entry) + (size_t)T * sizeof(Entry) +
               (size_t)P.ncls * sizeof(DevClass) + (size_t)P.ngam * sizeof(float2) + (size_t)T;
    return (b + 15) & ~(size_t)15;
}

int mp_loop_max_clusters(int threads, int cs, size_t smem) {
    switch (threads) {
        case 1024: return max_clusters<1024>(cs, smem);
        case 512: return max_clusters<512>(cs, smem);
        case 256: return max_clusters<256>(cs, smem);
        case 128: return max_clusters<128>(cs, smem);
        default: return 0;
    }
}

int mp_loop_threads(int nsig, int num_sms) {
    // 512-thread CTAs while every signal has SMs to itself, 256-thread CTAs
    // (two per SM) when there are more signals than SMs
    return nsig <= num_sms ? 512 : 256;
}

// launch shape for B signals: threads per CTA, cluster size and dynamic
// shared memory.  Clusters give a signal several SMs while there are SMs to
// spare; they need every N_w divisible by the cluster size and the per-CTA
// top level to fit on chip.
void mp_loop_shape(const DevPlan& P, const DevSig* hs, int B, int num_sms, int* threads, int* cs,
                   size_t* smem) {
    int nt = mp_loop_threads(B, num_sms);
    int c = B <= 8 ? 16 : B <= 16 ? 8 : B * 4 <= num_sms ? 4 : B * 2 <= num_sms ? 2 : 1;
    int nt_override = 0;
    if (const char* ov = getenv("MPGABOR_LOOP_THREADS")) {  // tuning overrides
        int t = atoi(ov);
        if (t == 128 || t == 256 || t == 512 || t == 1024) nt_override = t;
    }
    if (const char* ov = getenv("MPGABOR_CLUSTER")) {
        int t = atoi(ov);
        if (t == 1 || t == 2 || t == 4 || t == 8 || t == 16) c = t;
    }
    if (nt_override) nt = nt_override;
    for (; c > 1; c >>= 1) {
        // a cluster CTA runs only a few frame jobs per iteration: one warp per
        // scheduler keeps the redundant selection off each other's issue slots
        if (!nt_override) nt = 128;
        bool ok = true;
        int lt = 0;
        for (int b = 0; b < B && ok; ++b) {
            int t = 0;
            for (int w = 0; w < P.W; ++w) {
                if (hs[b].N[w] % c) ok = false;
                t += (int)(hs[b].N[w] / c);
            }
            lt = t > lt ? t : lt;
        }
        if (!ok || lt > TOPCAP) continue;
        const size_t sm = mp_loop_smem_bytes(P, lt, nt, c);
        if (mp_loop_max_clusters(nt, c, sm) < 1) continue;
        *threads = nt;
        *cs = c;
        *smem = sm;
        return;
    }
    int tmax = 1;
    for (int b = 0; b < B; ++b) tmax = hs[b].T > tmax ? hs[b].T : tmax;
    *threads = nt_override ? nt_override : mp_loop_threads(B, num_sms);
    *cs = 1;
    *smem = mp_loop_smem_bytes(P, tmax, nt, 1);
}

cudaError_t launch_mp_loop(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig,
                           long long kmax, double thr_scale, long long budget_ns, size_t smem,
                           int threads, int cs, cudaStream_t st) {
    if (nsig <= 0) return cudaSuccess;
    switch (threads) {
        case 1024: return launch_nt<1024>(P, d_sigs, d_order, nsig, kmax, thr_scale, budget_ns, smem, cs, st);
        case 512: return launch_nt<512>(P, d_sigs, d_order, nsig, kmax, thr_scale, budget_ns, smem, cs, st);
        case 256: return launch_nt<256>(P, d_sigs, d_order, nsig, kmax, thr_scale, budget_ns, smem, cs, st);
        case 128: return launch_nt<128>(P, d_sigs, d_order, nsig, kmax, thr_scale, budget_ns, smem, cs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mpg
