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
// One iteration:
//   1. every thread scans its share of the top level; warp bests are reduced
//      to the CTA best (shared memory + barrier);
//   2. with a cluster, each CTA sends its best to every CTA of the cluster
//      (st.async into distributed shared memory, completing bytes on the
//      receiver's mbarrier) and waits, bounded, for all of them; every warp
//      then takes the same selection, adjusts the coefficient to the
//      real-pair coefficient (eqs. dualatprod / projenfaster) and one thread
//      keeps E in FP64 and writes the atom list;
//   3. warps are assigned to dictionaries (warp w serves w mod W); a warp
//      builds its dictionary's update -- the atom's and the conjugate
//      partner's class tile, the column hull and the touched 32-bin chunks
//      as a bit mask -- and runs one job per owned touched frame: load the
//      frame's level-0 entries together with the touched chunks of the plane
//      and the matching tile entries, subtract both terms (eq.
//      fastkernupdate with the modulation of eq. hkj, looked up in an FP64-
//      rounded table), recompute the touched chunks' level-0 entries, the
//      frame's level-1 entry and its top-level slot; barrier.
//
// Clusters.  A signal may be given a thread-block cluster of CS CTAs (on CS
// SMs) instead of one CTA: frame n of every dictionary belongs to CTA
// n mod CS, which holds its top-level entry and runs its frame jobs.  The
// time limit is decided by CTA 0 and sent with the candidates, so all CTAs
// leave the loop in the same iteration.
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

// index q = (k tau) mod M_u of the column's modulation e^{i 2 pi k tau / M_u}
__device__ __forceinline__ int term_q(const Term& T, int n, int Nv, int av, int Mu, int Mumask) {
    int cc = n - T.Acol;
    if (cc < 0) cc += Nv;
    const int tau = T.tau0 + cc * av;
    if (Mumask) return (int)(((unsigned)T.kk * ((unsigned)tau & (unsigned)Mumask)) & (unsigned)Mumask);
    const unsigned tm = (unsigned)imod(tau, Mu);
    return (int)(((unsigned long long)T.kk * tm) % (unsigned)Mu);
}


__device__ __forceinline__ unsigned mapa_u32(unsigned addr, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 16-byte store into another CTA's shared memory that also completes 16
// bytes of transaction on that CTA's mbarrier
__device__ __forceinline__ void st_async16(unsigned raddr, const Entry& e, unsigned rbar) {
    const unsigned k0 = (unsigned)e.key, k1 = (unsigned)(e.key >> 32);
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
        :
        : "r"(raddr), "r"(k0), "r"(k1), "r"(__float_as_uint(e.val.x)), "r"(__float_as_uint(e.val.y)),
          "r"(rbar)
        : "memory");
}

__device__ __forceinline__ bool xbar_try(unsigned addr, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// one dictionary's part of the update, shared by the warps that serve it;
// all fields are scalars so the struct lives in registers
struct DictJob {
    Term t0, t1;
    int nstart;  // first frame of the hull owned by this CTA
    int cnt;     // owned frames of the hull
    // chunk ranges [l, h): a0, a1 of the atom (na of them), b0, b1 of the
    // partner (nb of them)
    int a0l, a0h, a1l, a1h, b0l, b0h, b1l, b1h;
    int na, nb;
    // the same set as a bit mask over chunks cbase .. cbase + 63 (cwide: the
    // set spans more than 64 chunks and is walked range by range instead)
    int cbase, cend;
    unsigned long long cmask;
    bool cwide;
};

// chunk ranges of a term's stored rows: up to two, as scalars
__device__ __forceinline__ int term_chunks2(const Term& t, int Mv, int Mr, int& l0, int& h0, int& l1,
                                            int& h1) {
    l0 = h0 = l1 = h1 = 0;
    if (!t.active) return 0;
    int n = 0;
    const int e1 = min(min(t.Arow + t.R, Mv), Mr);
    if (e1 > t.Arow) {
        l0 = t.Arow / CHUNK;
        h0 = (e1 - 1) / CHUNK + 1;
        n = 1;
    }
    if (t.Arow + t.R > Mv) {
        const int b1 = min(t.Arow + t.R - Mv, Mr);
        if (b1 > 0) {
            const int l = 0, h = (b1 - 1) / CHUNK + 1;
            if (n == 0) { l0 = l; h0 = h; } else { l1 = l; h1 = h; }
            ++n;
        }
    }
    return n;
}

__device__ __forceinline__ bool in_ranges(const DictJob& J, int c) {
    bool t = false;
    t |= (J.na > 0) & (c >= J.a0l) & (c < J.a0h);
    t |= (J.na > 1) & (c >= J.a1l) & (c < J.a1h);
    t |= (J.nb > 0) & (c >= J.b0l) & (c < J.b0h);
    t |= (J.nb > 1) & (c >= J.b1l) & (c < J.b1h);
    return t;
}


__device__ __forceinline__ void dict_job(const DevDict* sd, const DevPair* sp, const DevClass* scls,
                                         int W, const DevSig& S, int u, int kk, int j, bool edge,
                                         int v, int rank, int CS, DictJob& J) {
    J.t0 = make_term(sd, sp, scls, W, S, u, kk, j, edge, v, 0);
    J.t1 = make_term(sd, sp, scls, W, S, u, kk, j, edge, v, 1);
    const DevDict& Dv = sd[v];
    const int Nv = (int)S.N[v];
    J.cnt = 0;
    J.nstart = 0;
    int lo = 0, hi = 0;
    bool any = false;
    if (J.t0.active) { lo = J.t0.a0; hi = J.t0.a0 + J.t0.C; any = true; }
    if (J.t1.active) {
        if (any) { lo = min(lo, J.t1.a0); hi = max(hi, J.t1.a0 + J.t1.C); }
        else { lo = J.t1.a0; hi = J.t1.a0 + J.t1.C; any = true; }
    }
    if (any) {
        int ns, nf;
        const int nc = hi - lo;
        if (nc >= Nv) { ns = 0; nf = Nv; }
        else { ns = S.Nmask[v] ? (lo & S.Nmask[v]) : imod(lo, Nv); nf = nc; }
        const int i0 = imod(rank - ns, CS);
        J.nstart = ns + i0;
        J.cnt = nf > i0 ? (nf - i0 + CS - 1) / CS : 0;
    }
    J.na = term_chunks2(J.t0, Dv.M, Dv.Mr, J.a0l, J.a0h, J.a1l, J.a1h);
    J.nb = term_chunks2(J.t1, Dv.M, Dv.Mr, J.b0l, J.b0h, J.b1l, J.b1h);
    int clo = 1 << 30, chi = 0;
    if (J.na > 0) { clo = min(clo, J.a0l); chi = max(chi, J.a0h); }
    if (J.na > 1) { clo = min(clo, J.a1l); chi = max(chi, J.a1h); }
    if (J.nb > 0) { clo = min(clo, J.b0l); chi = max(chi, J.b0h); }
    if (J.nb > 1) { clo = min(clo, J.b1l); chi = max(chi, J.b1h); }
    if (chi <= clo) { clo = 0; chi = 0; }
    J.cbase = clo;
    J.cend = chi;
    J.cwide = chi - clo > 64;
    unsigned long long m = 0;
    if (!J.cwide) {
        auto add = [&](int l, int h) {
            const int n = h - l;
            const unsigned long long bits = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
            m |= bits << (l - clo);
        };
        if (J.na > 0) add(J.a0l, J.a0h);
        if (J.na > 1) add(J.a1l, J.a1h);
        if (J.nb > 0) add(J.b0l, J.b0h);
        if (J.nb > 1) add(J.b1l, J.b1h);
    }
    J.cmask = m;
}

__device__ __forceinline__ bool chunk_touched(const DictJob& J, int c) {
    if (!J.cwide) {
        const int d = c - J.cbase;
        return d >= 0 && d < 64 && ((J.cmask >> d) & 1ull);
    }
    return in_ranges(J, c);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_mp_loop(DevPlan P, DevSig* __restrict__ sigs, const int* __restrict__ order,
              long long kmax, double thr_scale, long long budget_ns, int CS, long long reset_it,
              double reset_scale) {
    namespace cg = cooperative_groups;
    constexpr int NWARPS = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevSig S;
    __shared__ DevDict sd[MAXW];
    __shared__ DevPair sp[MAXW * MAXW];
    __shared__ int sstop[2];        // stop decision per iteration parity
    __shared__ int ltb[MAXW + 1];   // local top-level base per dictionary
    __shared__ Entry wsel[NWARPS];  // per-warp bests of the scan
    __shared__ __align__(16) Entry cand[2][16];      // CTA bests of the cluster, per parity
    __shared__ __align__(16) int tmsg[2][4];         // time-limit message of CTA 0, per parity
    __shared__ __align__(8) unsigned long long xbar[2];  // exchange barriers, per parity
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
    const unsigned xb0 = (unsigned)__cvta_generic_to_shared(&xbar[0]);
    const unsigned xb1 = (unsigned)__cvta_generic_to_shared(&xbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xb1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmsg[0][0] = tmsg[1][0] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        int b = 0;
        for (int w = 0; w < W; ++w) {
            ltb[w] = b;
            b += CS > 1 ? (int)(S.N[w] / CS) : S.tbase[w + 1] - S.tbase[w];
        }
        ltb[W] = b;
    }
    __syncthreads();
    const int T = ltb[W];
    Entry* top = reinterpret_cast<Entry*>(smem_raw);
    DevClass* scls = reinterpret_cast<DevClass*>(top + T);
    float2* sgam = reinterpret_cast<float2*>(scls + P.ncls);
    float2* scis = sgam + P.ngam;
    unsigned char* tdirty = reinterpret_cast<unsigned char*>(scis + P.ncis);

    for (int i = tid; i < P.ncls; i += NT) scls[i] = P.cls[i];
    for (int i = tid; i < P.ngam; i += NT) sgam[i] = P.gam[i];
    for (int i = tid; i < P.ncis; i += NT) scis[i] = P.cis[i];
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

    long long k = S.k;
    // FP64 work stays in one thread (the FP64 pipe is narrow on this part):
    // E, and the stop tests that read it, are evaluated there one iteration
    // ahead and published in sstop
    const int KEEPER = NT - 32;
    double E = S.E;
    const double E0 = S.E0;
    const double thr = E0 * thr_scale;
    // resets (Alg. 2): stop the launch for a reset pass once reset_it atoms
    // were selected since the last reset or E dropped below E_out reset_scale
    const bool resets = reset_it > 0 || reset_scale > 0.0;
    const long long k_out = S.k_out;
    const double E_out = S.E_out;
    const unsigned long long t_start = gtimer();
    const float2* __restrict__ tiles = P.tiles;
    const unsigned xbytes = (unsigned)(CS * sizeof(Entry)) + (budget_ns > 0 ? 16u : 0u);
    int stop = 0;
    if (tid == KEEPER) {
        int s0 = 0;
        if (!isfinite(E0)) s0 = MP_STOP_INVALID;
        else if (E <= 0.0) s0 = MP_STOP_NEGENERGY;
        else if (E <= thr) s0 = MP_STOP_SNR;
        else if (k >= kmax) s0 = MP_STOP_KMAX;
        else if (resets && k > k_out &&
                 ((reset_it > 0 && k - k_out >= reset_it) ||
                  (reset_scale > 0.0 && E < E_out * reset_scale)))
            s0 = -3;
        sstop[k & 1] = s0;
    }
    // every CTA's barriers are initialised before anyone sends
    if (CS > 1) cluster.sync(); else __syncthreads();

    // warp -> dictionary service: warp w serves v = w mod W as its slot w / W
    // of nserve(v) warps (or, with fewer warps than dictionaries, v = w,
    // w + NWARPS, ...)
    unsigned long long it = 0;  // iteration counter (exchange parities)
    for (;;) {
        const int par = (int)(it & 1);
        const unsigned xb = par ? xb1 : xb0;
        // ---- 1. scan of the top level, CTA best, cluster exchange ----------
        {
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            for (int i = tid; i < T; i += NT) {
                const Entry e = top[i];
                if (e.key > b.key) b = e;
            }
            const Entry r = warp_max_entry(b);
            if (lane == 0) wsel[warp] = r;
            if (CS > 1 && tid == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xb),
                             "r"(xbytes)
                             : "memory");
        }
        __syncthreads();
        Entry best;
        {
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            if (lane < NWARPS) b = wsel[lane];
            best = warp_max_entry(b);
        }
        if (CS > 1) {
            if (warp == 0) {
                if (lane < CS) {
                    const unsigned laddr = (unsigned)__cvta_generic_to_shared(&cand[par][rank]);
                    st_async16(mapa_u32(laddr, lane), best, mapa_u32(xb, lane));
                }
                if (budget_ns > 0 && rank == 0) {
                    int tf = 0;
                    if (lane == 0) tf = (long long)(gtimer() - t_start) > budget_ns ? 1 : 0;
                    tf = __shfl_sync(FULL, tf, 0);
                    if (lane < CS) {
                        Entry m;
                        m.key = (unsigned long long)(unsigned)tf;
                        m.val = make_float2(0.f, 0.f);
                        const unsigned laddr = (unsigned)__cvta_generic_to_shared(&tmsg[par][0]);
                        st_async16(mapa_u32(laddr, lane), m, mapa_u32(xb, lane));
                    }
                }
            }
            // bounded wait for the CS candidates (and the time-limit message)
            const unsigned long long w0 = gtimer();
            const unsigned xpar = (unsigned)((it >> 1) & 1);
            bool ok = true;
            while (!xbar_try(xb, xpar)) {
                if (gtimer() - w0 > 2000000000ull) {
                    ok = false;
                    break;
                }
            }
            Entry b;
            b.key = 0;
            b.val = make_float2(0.f, 0.f);
            if (lane < CS) b = cand[par][lane];
            best = warp_max_entry(b);
            if (!ok) stop = -2;
        } else if (budget_ns > 0) {
            // single CTA: the time limit is read by one thread before the scan
            // barrier of the next iteration; here it is read after this one
            if (tid == 0) tmsg[par][0] = (long long)(gtimer() - t_start) > budget_ns ? 1 : 0;
            __syncthreads();
        }

        // ---- 2. selection, adjustment, bookkeeping -------------------------
        if (stop == 0) stop = sstop[k & 1];
        if (stop == 0 && budget_ns > 0 && tmsg[par][0]) stop = -1;
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
        const float2* cis_u = scis + sd[u].cis_off;
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
        if (tid == KEEPER) {
            E -= (double)Edf;
            if (rank == 0) {
                mp_atom at;
                at.dict = u;
                at.m = kk;
                at.n = j;
                at.re = cx;
                at.im = cy;
                S.atoms[k] = at;
                S.errs[k] = E;
            }
            int s1 = 0;  // stop tests before the next selection
            if (E <= 0.0) s1 = MP_STOP_NEGENERGY;
            else if (E <= thr) s1 = MP_STOP_SNR;
            else if (k + 1 >= kmax) s1 = MP_STOP_KMAX;
            else if (resets && ((reset_it > 0 && k + 1 - k_out >= reset_it) ||
                                (reset_scale > 0.0 && E < E_out * reset_scale)))
                s1 = -3;  // reset pass (Alg. 2) before the next selection
            sstop[(k + 1) & 1] = s1;
        }
        ++k;
        const float2 c_main = make_float2(cx, cy), c_conj = make_float2(cx, -cy);

        // ---- 3. frame jobs: each warp serves its dictionaries ---------------
        // warp w serves dictionary w mod W as slot w / W of the warps that
        // serve it; with fewer warps than dictionaries it serves w, w +
        // NWARPS, ... alone
        const int v_first = NWARPS >= W ? warp % W : warp;
        const int v_step = NWARPS >= W ? W : NWARPS;
        const int slot = NWARPS >= W ? warp / W : 0;
        for (int v = v_first; v < W; v += v_step) {
            const int nserve = NWARPS >= W ? (NWARPS / W + (v < NWARPS % W ? 1 : 0)) : 1;
            DictJob J;
            dict_job(sd, sp, scls, W, S, u, kk, j, edge, v, rank, CS, J);
            const DevDict& Dv = sd[v];
            const int Nv = (int)S.N[v];
            for (int f = slot; f < J.cnt; f += nserve) {
                int n = J.nstart + f * CS;
                n -= (n >= Nv) ? Nv : 0;
                n -= (n >= Nv) ? Nv : 0;
                // level-0 entries of the whole frame (untouched chunks keep theirs)
                const Entry* l0row = S.l0[v] + (long long)n * Dv.nch;
                Entry l0v[MAXL0];
#pragma unroll
                for (int q = 0; q < MAXL0; ++q) {
                    const int c = lane + 32 * q;
                    if (c < Dv.nch) l0v[q] = l0row[c];
                }
                float2* prow = S.plane[v] + (long long)n * Dv.Mrp;
                const float2 w0 = J.t0.active ? cmul(c_main, cis_u[term_q(J.t0, n, Nv, Dv.a, Mu, Mumask)])
                                              : make_float2(0.f, 0.f);
                const float2 w1 = J.t1.active ? cmul(c_conj, cis_u[term_q(J.t1, n, Nv, Dv.a, Mu, Mumask)])
                                              : make_float2(0.f, 0.f);
                Entry fmax;
                fmax.key = 0;
                fmax.val = make_float2(0.f, 0.f);
                // touched chunks, CB at a time, lowest first (bit mask; a set
                // wider than 64 chunks is walked chunk by chunk)
                unsigned long long mrest = J.cmask;
                int wc = J.cbase;
                for (;;) {
                    int chunk[CB];
                    int cnt = 0;
#pragma unroll
                    for (int q = 0; q < CB; ++q) {
                        chunk[q] = -1;
                        if (!J.cwide) {
                            if (mrest) {
                                const int b = __ffsll((long long)mrest) - 1;
                                mrest &= mrest - 1ull;
                                chunk[q] = J.cbase + b;
                            }
                        } else {
                            while (wc < J.cend && !in_ranges(J, wc)) ++wc;
                            if (wc < J.cend) chunk[q] = wc++;
                        }
                        cnt += chunk[q] >= 0 ? 1 : 0;
                    }
                    if (cnt == 0) break;
                    float2 val[CB], h0[CB], h1[CB];
                    bool hit0[CB], hit1[CB];
#pragma unroll
                    for (int q = 0; q < CB; ++q) {
                        hit0[q] = hit1[q] = false;
                        if (chunk[q] >= 0) {
                            const int m = chunk[q] * CHUNK + lane;
                            val[q] = prow[m];
                            int off;
                            if (m < Dv.Mr) {
                                if (term_hit(J.t0, m, n, Dv.M, Nv, &off)) {
                                    hit0[q] = true;
                                    h0[q] = __ldg(tiles + J.t0.tile + off);
                                }
                                if (term_hit(J.t1, m, n, Dv.M, Nv, &off)) {
                                    hit1[q] = true;
                                    h1[q] = __ldg(tiles + J.t1.tile + off);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < CB; ++q) {
                        if (chunk[q] < 0) continue;
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
                        e.key = (m < Dv.Mr) ? make_key_sel(x2, S.fbase[v] + ((unsigned)n << Dv.msh) + m,
                                                            m, Dv, sgam, P.pedantic)
                                            : 0ull;
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
                    if (cq < Dv.nch && !chunk_touched(J, cq) && l0v[q].key > b.key) b = l0v[q];
                }
                for (int cq = lane + 32 * MAXL0; cq < Dv.nch; cq += 32) {
                    if (chunk_touched(J, cq)) continue;
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
            if (NWARPS >= W) break;  // one dictionary per warp
        }
        __syncthreads();

        // ---- level 2 (groups) of touched frames (single-CTA launches) -------
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
        ++it;
    }
    if (CS > 1) cluster.sync();  // no CTA leaves while others may address it
    if (tid == KEEPER && rank == 0) {
        Sg.k = k;
        Sg.E = E;
        Sg.reset_pending = 0;
        if (stop > 0) {
            Sg.stop = stop;
            Sg.timed_out = 0;
        } else if (stop == -3) {
            Sg.stop = 0;
            Sg.timed_out = 0;
            Sg.reset_pending = 1;
        } else {
            Sg.stop = 0;
            Sg.timed_out = 1;
        }
    }
}

template <int NT>
cudaError_t launch_nt(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig, long long kmax,
                      double thr_scale, long long budget_ns, size_t smem, int cs, cudaStream_t st,
                      long long reset_it, double reset_scale) {
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
    e = cudaLaunchKernelEx(&cfg, k_mp_loop<NT>, P, d_sigs, d_order, kmax, thr_scale, budget_ns, cs,
                           reset_it, reset_scale);
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

size_t mp_loop_smem_bytes(const DevPlan& P, int T, int, int) {
    size_t b = (size_t)T * sizeof(Entry) + (size_t)P.ncls * sizeof(DevClass) +
               (size_t)(P.ngam + P.ncis) * sizeof(float2) + (size_t)T;
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

// feasibility of a requested launch shape (threads per CTA, cluster size)
bool mp_loop_shape_ok(const DevPlan& P, const DevSig* hs, int B, int threads, int c, size_t* smem) {
    if (threads != 128 && threads != 256 && threads != 512 && threads != 1024) return false;
    if (c != 1 && c != 2 && c != 4 && c != 8 && c != 16) return false;
    if (c == 1) {
        int tmax = 1;
        for (int b = 0; b < B; ++b) tmax = hs[b].T > tmax ? hs[b].T : tmax;
        *smem = mp_loop_smem_bytes(P, tmax, threads, 1);
        return *smem <= 227 * 1024;
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
    if (lt > TOPCAP) return false;
    *smem = mp_loop_smem_bytes(P, lt, threads, c);
    return mp_loop_max_clusters(threads, c, *smem) >= 1;
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
                           int threads, int cs, cudaStream_t st, long long reset_it,
                           double reset_scale) {
    if (nsig <= 0) return cudaSuccess;
#define MPG_LAUNCH(NTV)                                                                        \
    launch_nt<NTV>(P, d_sigs, d_order, nsig, kmax, thr_scale, budget_ns, smem, cs, st, reset_it, \
                   reset_scale)
    switch (threads) {
        case 1024: return MPG_LAUNCH(1024);
        case 512: return MPG_LAUNCH(512);
        case 256: return MPG_LAUNCH(256);
        case 128: return MPG_LAUNCH(128);
        default: return cudaErrorInvalidValue;
    }
#undef MPG_LAUNCH
}

}  // namespace mpg
