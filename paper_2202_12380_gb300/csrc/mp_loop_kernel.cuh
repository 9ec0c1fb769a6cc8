// Persistent matching-pursuit loop kernel, included by the translation
// units that instantiate its variants (mp_loop_f32.cu, mp_loop_f64.cu);
// the launch logic is in mp_loop.cu.
//
// Persistent matching-pursuit loop (Alg. 1 with the residual update of
// Alg. 3): one CTA (or one thread-block cluster) per signal, iterating
// selection -> real-pair adjustment -> energy bookkeeping -> coefficient-
// domain update of every dictionary -> max-tree repair, entirely on the
// device.
//
// Max tree (Sec. 5.1), keys only (score bits and inverted flat index).
// Level 0 (per frame and 32-bin chunk) and level 1 (per frame) live in
// global memory next to the coefficient planes; the top level (one key per
// frame, or per group of 2^gshift frames of a single CTA whose frames do not
// fit) lives in shared memory and is scanned every iteration.  It is held as
// two word arrays, scores and inverted flat indices: the scan reads only the
// scores, since top-level positions are ordered like flat indices (by
// dictionary, then frame), so among equal scores the first position holds
// the largest key.  The selected coefficient itself is read from its plane.
//
// One iteration:
//   1. the CTA's best key: warp 0 alone scans a cluster CTA's top level,
//      otherwise every thread scans its share and a barrier combines them;
//   2. with a cluster, each CTA sends its best to every CTA of the cluster
//      (st.async into distributed shared memory, completing bytes on the
//      receiver's mbarrier) and waits, bounded, for all of them; every warp
//      then decodes the same selection;
//   3. the selected coefficient: a single CTA reads it from its plane; in a
//      cluster the CTA owning the frame reads it and sends it to every CTA
//      (second mbarrier), overlapped with step 4;
//   4. warp v builds dictionary v's update for this iteration -- the class
//      tiles of the atom and of its conjugate partner, their first row and
//      column, the modulation index of column 0 and its step, the frames of
//      the column hull owned by this CTA, the list of touched 32-bin chunks
//      and the lanes' touched-chunk masks -- into shared memory; in
//      128-thread CTAs it also issues the loads of its dictionary's first
//      frame job; a spare warp (more warps than dictionaries) adjusts the
//      coefficient to the real-pair coefficient (eqs. dualatprod /
//      projenfaster), keeps E in FP64, writes the atom and the next stop
//      decision; barrier;
//   5. frame jobs: the prefetched one, then the rest dealt to the warps from
//      one flat index.  A job loads the frame's level-0 keys together with
//      the touched chunks of the plane and the matching tile entries,
//      subtracts both terms (eq. fastkernupdate with the modulation of eq.
//      hkj, looked up in an FP64-rounded table), recomputes the touched
//      chunks' level-0 keys, the frame's level-1 key and its top-level slot;
//      barrier;
//   6. (single CTA with grouped top level) the groups of touched frames are
//      rebuilt, one thread per group; barrier.
//
// Clusters.  A signal may be given a thread-block cluster of CS CTAs (on CS
// SMs) instead of one CTA: frame n of every dictionary belongs to CTA
// n mod CS, which holds its top-level key and runs its frame jobs.  The
// time limit is decided by CTA 0 and sent with the candidates, so all CTAs
// leave the loop in the same iteration.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int MAXL0 = 4;   // level-0 entries held per lane (larger frames reload)
constexpr unsigned NOPOS = 0xffffffffu;  // no top-level position
constexpr int CB = 4;      // touched chunks per batch of loads

// One dictionary's part of an iteration's update.  Term 0 is the selected
// atom, term 1 its conjugate partner (M_u - k, j).  A term's tile covers
// rows Arow .. Arow + R - 1 (mod M_v) and frames Acol .. Acol + C - 1
// (mod N_v); column c carries the modulation e^{i 2 pi q / M_u},
// q = qb + c dq (mod M_u).
struct __align__(16) VJob {
    int act0, act1;
    int Arow0, Arow1;
    int R0, R1;
    int Acol0, Acol1;
    int C0, C1;
    int qb0, qb1;
    int dq0, dq1;
    int nstart, cnt;  // owned hull frames nstart + f CS (mod N_v), f < cnt
    long long tile0, tile1;  // float2 offsets of the class tiles
    int nlist;               // touched chunks, listed in the chunk list of v
    int pad[3];
};

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    return cx_t<C2>::make(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// x mod M for x in [-M, 2M)
__device__ __forceinline__ int wrap2(int x, int M) {
    x += x < 0 ? M : 0;
    return x >= M ? x - M : x;
}

__device__ __forceinline__ unsigned mapa_u32(unsigned addr, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 8-byte store into another CTA's shared memory that also completes 8 bytes
// of transaction on that CTA's mbarrier
__device__ __forceinline__ void st_async8(unsigned raddr, unsigned lo, unsigned hi, unsigned rbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];"
        :
        : "r"(raddr), "r"(lo), "r"(hi), "r"(rbar)
        : "memory");
}

// 16-byte form (a double2 coefficient)
__device__ __forceinline__ void st_async16(unsigned raddr, unsigned a, unsigned b, unsigned c,
                                           unsigned d, unsigned rbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, "
        "[%5];"
        :
        : "r"(raddr), "r"(a), "r"(b), "r"(c), "r"(d), "r"(rbar)
        : "memory");
}

// send the selected coefficient (float2 or double2) to CTA `lane`
__device__ __forceinline__ void send_coef(unsigned laddr, int lane, float2 v, unsigned rbar_l) {
    st_async8(mapa_u32(laddr, lane), __float_as_uint(v.x), __float_as_uint(v.y),
              mapa_u32(rbar_l, lane));
}
__device__ __forceinline__ void send_coef(unsigned laddr, int lane, double2 v, unsigned rbar_l) {
    const unsigned long long x = (unsigned long long)__double_as_longlong(v.x);
    const unsigned long long y = (unsigned long long)__double_as_longlong(v.y);
    st_async16(mapa_u32(laddr, lane), (unsigned)x, (unsigned)(x >> 32), (unsigned)y,
               (unsigned)(y >> 32), mapa_u32(rbar_l, lane));
}

// expect this iteration's candidate bytes and the selected coefficient
__device__ __forceinline__ void arm_exchange(unsigned xb, unsigned vb, unsigned xbytes,
                                             unsigned vbytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xb), "r"(xbytes)
                 : "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vb), "r"(vbytes)
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

// Dictionary v's update for the selected atom (u, k, j), built by one warp
// (every lane computes the scalars and returns them; the lanes split the
// chunk list).  POW2:
// every M and a is a power of two, so the class, row and modulation indices
// are shifts and masks.  tmk receives, per lane, which of the chunks
// lane + 32 s (s < MAXL0) are touched.
template <bool POW2>
__device__ __forceinline__ VJob build_vjob(const DevDict* sd, const DevPair* sp,
                                           const DevClass* scls, int W, const DevSig& S, int u,
                                           int kk, int j, bool edge, int v, int rank, int CS,
                                           int cs_sh, int lane, VJob* out,
                                           unsigned short* clist, unsigned char* tmk, int ccap,
                                           int* berr) {
    const DevDict& Du = sd[u];
    const DevDict& Dv = sd[v];
    const DevPair& PR = sp[u * W + v];
    const int Mu = Du.M, Mumask = Du.Mmask, au = Du.a;
    const int Mv = Dv.M, Mr = Dv.Mr, av = Dv.a;
    const int Nv = (int)S.N[v];
    int ct, base_n;
    if (POW2) {
        ct = j & (PR.rt - 1);
        base_n = PR.aratio ? j * PR.aratio : j >> PR.rt_sh;
    } else {
        ct = j % PR.rt;
        base_n = PR.aratio ? j * PR.aratio : (j - ct) / PR.rt;
    }
    int act[2], Arow[2], R[2], Acol[2], Cc[2], a0[2], qb[2], dq[2];
    long long tile[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int kt = t ? Mu - kk : kk;
        int cf, base_m;
        if (POW2) {
            cf = kt & (PR.rf - 1);
            base_m = PR.mratio ? kt * PR.mratio : kt >> PR.rf_sh;
        } else {
            cf = kt % PR.rf;
            base_m = PR.mratio ? kt * PR.mratio : (kt - cf) / PR.rf;
        }
        const DevClass C = scls[PR.cls_base + cf * PR.rt + ct];
        Arow[t] = POW2 ? ((base_m + C.i_lo) & Dv.Mmask) : wrap2(base_m + C.i_lo, Mv);
        R[t] = C.R;
        // any stored row (0 .. M_v/2) inside [Arow, Arow + R) mod M_v ?
        act[t] = (t == 0 || !edge) && C.R > 0 && (Arow[t] < Mr || Arow[t] + C.R > Mv);
        a0[t] = base_n + C.c_lo;
        Acol[t] = wrap2(a0[t], Nv);
        Cc[t] = C.C;
        const int tau0 = C.c_lo * av - ct * au;
        if (POW2) {
            qb[t] = (int)(((unsigned)kt * (unsigned)tau0) & (unsigned)Mumask);
            dq[t] = (int)(((unsigned)kt * (unsigned)av) & (unsigned)Mumask);
        } else {
            qb[t] = (int)lmod((long long)kt * tau0, Mu);
            dq[t] = (int)(((long long)kt * av) % Mu);
        }
        tile[t] = C.off;
    }
    // frames of the column hull of both terms owned by this CTA
    int cnt = 0, nstart = 0;
    if (act[0] | act[1]) {
        const int lo = act[0] && act[1] ? min(a0[0], a0[1]) : (act[0] ? a0[0] : a0[1]);
        const int hi = act[0] && act[1] ? max(a0[0] + Cc[0], a0[1] + Cc[1])
                                        : (act[0] ? a0[0] + Cc[0] : a0[1] + Cc[1]);
        const int nc = hi - lo;
        const int ns = nc >= Nv ? 0 : wrap2(lo, Nv);
        const int nf = nc >= Nv ? Nv : nc;
        const int i0 = (rank - ns) & (CS - 1);
        nstart = ns + i0;
        cnt = nf > i0 ? ((nf - i0 + CS - 1) >> cs_sh) : 0;
    }
    // touched chunks: each term's stored rows form up to two chunk ranges;
    // the lanes walk their concatenation and drop chunks an earlier range
    // already holds
    int rl[4], rh[4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int e1 = min(min(Arow[t] + R[t], Mv), Mr);
        const bool p1 = act[t] && e1 > Arow[t];
        rl[2 * t] = p1 ? Arow[t] >> 5 : 0;
        rh[2 * t] = p1 ? ((e1 - 1) >> 5) + 1 : 0;
        const int b1 = min(Arow[t] + R[t] - Mv, Mr);
        const bool p2 = act[t] && b1 > 0;
        rl[2 * t + 1] = 0;
        rh[2 * t + 1] = p2 ? ((b1 - 1) >> 5) + 1 : 0;
    }
    unsigned mk = 0;
#pragma unroll
    for (int s = 0; s < MAXL0; ++s) {
        const int c = lane + 32 * s;
        bool in = false;
#pragma unroll
        for (int r = 0; r < 4; ++r) in |= c >= rl[r] && c < rh[r];
        mk |= in ? (1u << s) : 0u;
    }
    tmk[lane] = (unsigned char)mk;
    const int p1 = rh[0] - rl[0];
    const int p2 = p1 + rh[1] - rl[1];
    const int p3 = p2 + rh[2] - rl[2];
    const int total = p3 + rh[3] - rl[3];
    int count = 0;
    for (int base = 0; base < total; base += 32) {
        const int idx = base + lane;
        const int r = idx < p1 ? 0 : idx < p2 ? 1 : idx < p3 ? 2 : 3;
        const int c = r == 0 ? rl[0] + idx : r == 1 ? rl[1] + idx - p1
                    : r == 2 ? rl[2] + idx - p2 : rl[3] + idx - p3;
        bool dup = (r > 0 && c >= rl[0] && c < rh[0]);
        dup |= (r > 1 && c >= rl[1] && c < rh[1]);
        dup |= (r > 2 && c >= rl[2] && c < rh[2]);
        const bool keep = idx < total && !dup;
        const unsigned ball = __ballot_sync(FULL, keep);
        const int pos = count + __popc(ball & ((1u << lane) - 1u));
        if (keep && inb(pos, ccap, 1, berr)) clist[pos] = (unsigned short)c;
        count += __popc(ball);
    }
    VJob J;
    {
        J.act0 = act[0];
        J.act1 = act[1];
        J.Arow0 = Arow[0];
        J.Arow1 = Arow[1];
        J.R0 = R[0];
        J.R1 = R[1];
        J.Acol0 = Acol[0];
        J.Acol1 = Acol[1];
        J.C0 = Cc[0];
        J.C1 = Cc[1];
        J.qb0 = qb[0];
        J.qb1 = qb[1];
        J.dq0 = dq[0];
        J.dq1 = dq[1];
        J.nstart = nstart;
        J.cnt = cnt;
        J.tile0 = tile[0];
        J.tile1 = tile[1];
        J.nlist = count;
        J.pad[0] = J.pad[1] = J.pad[2] = 0;
    }
    if (lane == 0) *out = J;
    return J;
}

// e^{i 2 pi q / M}, q < M, from the table of dictionary D: a quarter period
// (the quadrant k of q multiplies by i^k, exactly) or the full period
template <typename C2>
__device__ __forceinline__ C2 cis_at(const C2* t, const DevDict& D, int q) {
    if (D.cis_q == 0) return t[q];
    int k, r;
    if (D.cis_qsh >= 0) {
        k = q >> D.cis_qsh;
        r = q & (D.cis_q - 1);
    } else {
        k = q / D.cis_q;
        r = q - k * D.cis_q;
    }
    const C2 e = t[r];
    const auto x = (k & 1) ? -e.y : e.x;
    const auto y = (k & 1) ? e.x : e.y;
    return (k & 2) ? cx_t<C2>::make(-x, -y) : cx_t<C2>::make(x, y);
}

// tile column of a term for frame n: its first entry in the tile pool, or -1
// when the column misses the frame; cc is the column index
__device__ __forceinline__ long long term_col(int act, int Acol, int C, int R, long long tile, int n,
                                              int Nv, int& cc) {
    cc = n - Acol;
    cc += cc < 0 ? Nv : 0;
    return (act && cc < C) ? tile + (long long)cc * R : -1ll;
}

// weight c e^{i 2 pi q / M_u} of column cc, q = qb + cc dq (mod M_u); zero
// when the column misses the frame
template <typename C2>
__device__ __forceinline__ C2 term_weight(long long tbase, int cc, int qb, int dq,
                                          const DevDict& Du, const C2* cis_u, C2 c) {
    if (tbase < 0) return cx_t<C2>::make(0, 0);
    int q;
    if (Du.Mmask) q = (int)(((unsigned)qb + (unsigned)cc * (unsigned)dq) & (unsigned)Du.Mmask);
    else q = (int)(((long long)qb + (long long)cc * dq) % Du.M);
    return cmul(c, cis_at(cis_u, Du, q));
}

// one frame job in registers: the frame, its level-0 keys, the columns of
// both terms, and the loads of one batch of touched chunks
template <typename C2>
struct JobCtx {
    int v, n, nb;
    int cc0, cc1;
    long long tb0, tb1;
    Key l0v[MAXL0];
    int cq[CB];
    C2 val[CB], h0[CB], h1[CB];
    bool hit[CB];
};

// C2: element type of the coefficient planes, kernel tiles and tables --
// float2, or double2 for MP_COEF_FP64 plans (every step then runs in FP64)
template <int NT, bool POW2, typename C2>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_mp_loop(DevPlan P, DevSig* __restrict__ sigs, const int* __restrict__ order,
              long long kmax, double thr_scale, long long budget_ns, int CS, int topcap,
              long long reset_it, double reset_scale) {
    namespace cg = cooperative_groups;
    using R = typename cx_t<C2>::R;
    constexpr int NWARPS = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevSig S;
    __shared__ DevDict sd[MAXW];
    __shared__ DevPair sp[MAXW * MAXW];
    __shared__ VJob vj[MAXW];
    __shared__ unsigned char tmk[MAXW][32];  // touched chunks lane + 32 s, per lane
    __shared__ int sstop[2];        // stop decision per iteration parity
    __shared__ int ltb[MAXW + 1];   // local top-level base per dictionary
    __shared__ int clo[MAXW + 1];   // chunk-list base per dictionary
    __shared__ int sgs;             // log2 of frames per top-level key (single CTA)
    __shared__ int ndirty;          // dirty top-level groups this iteration
    __shared__ Key wsel[NWARPS];    // per-warp bests of the scan
    __shared__ __align__(8) Key cand[2][16];   // CTA bests of the cluster, per parity
    __shared__ __align__(8) Key tmsg[2];       // time-limit message of CTA 0, per parity
    __shared__ __align__(16) C2 cval[2];       // selected coefficient, per parity
    __shared__ __align__(16) C2 scoef[2];      // adjusted coefficient, per parity
    __shared__ int sbad;                       // a bounded wait gave up
    __shared__ __align__(8) unsigned long long xbar[2];  // candidate barriers, per parity
    __shared__ __align__(8) unsigned long long vbar[2];  // coefficient barriers, per parity
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = CS > 1 ? (int)cluster.block_rank() : 0;
    const int cs_sh = __ffs(CS) - 1;
    DevSig& Sg = sigs[order[blockIdx.x / CS]];
    int* berr = &Sg.bounds;  // bounds-checking build: first failed access site
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
    const unsigned vb0 = (unsigned)__cvta_generic_to_shared(&vbar[0]);
    const unsigned vb1 = (unsigned)__cvta_generic_to_shared(&vbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xb1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(vb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(vb1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmsg[0] = tmsg[1] = 0ull;
        ndirty = 0;
        sbad = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // top level: this CTA's frames (cluster), else every frame, grouped
        // by 2^gs so that at most topcap keys are held
        int gs = 0;
        if (CS == 1) {
            for (;;) {
                long long t = 0;
                for (int w = 0; w < W; ++w) t += (S.N[w] + (1ll << gs) - 1) >> gs;
                if (t <= topcap || gs >= 30) break;
                ++gs;
            }
        }
        sgs = gs;
        int b = 0, c = 0;
        for (int w = 0; w < W; ++w) {
            ltb[w] = b;
            b += CS > 1 ? (int)(S.N[w] / CS) : (int)((S.N[w] + (1ll << gs) - 1) >> gs);
            clo[w] = c;
            c += (P.d[w].nch + 7) & ~7;
        }
        ltb[W] = b;
        clo[W] = c;
    }
    __syncthreads();
    const int T = ltb[W];
    const int gsh = sgs;
    // top level: score words tops[0 .. T), inverted flat indices topl[0 .. T)
    unsigned* tops = reinterpret_cast<unsigned*>(smem_raw);
    unsigned* topl = tops + ((T + 1) & ~1);
    auto set_top = [&](int i, Key key) {
        tops[i] = (unsigned)(key >> 32);
        topl[i] = (unsigned)key;
    };
    // warp-wide best top-level key from each lane's best (score, position);
    // every lane returns it (0 when no lane holds a position)
    auto top_best = [&](unsigned sc, unsigned pos) -> Key {
        const unsigned ms = __reduce_max_sync(FULL, pos == NOPOS ? 0u : sc);
        const unsigned mp = __reduce_min_sync(FULL, (pos != NOPOS && sc == ms) ? pos : NOPOS);
        return mp == NOPOS ? 0ull : (((Key)ms << 32) | topl[mp]);
    };
    DevClass* scls = reinterpret_cast<DevClass*>(topl + ((T + 1) & ~1));
    // the tables start 16-byte aligned (offset from the shared base, so that
    // every pointer below stays a shared-memory pointer)
    const size_t gam_off =
        ((size_t)(reinterpret_cast<unsigned char*>(scls + P.ncls) - smem_raw) + 15) & ~(size_t)15;
    C2* sgam = reinterpret_cast<C2*>(smem_raw + gam_off);
    C2* scis = sgam + P.ngam;
    unsigned* dbits = reinterpret_cast<unsigned*>(scis + P.ncis);  // dirty groups, one bit each
    unsigned short* dlist = reinterpret_cast<unsigned short*>(dbits + ((T + 31) >> 5));
    unsigned short* chl = dlist + ((T + 7) & ~7);  // touched-chunk lists

    for (int i = tid; i < P.ncls; i += NT) scls[i] = P.cls[i];
    {
        const C2* pg = cx_t<C2>::gam(P);
        const C2* pc = cx_t<C2>::cis(P);
        for (int i = tid; i < P.ngam; i += NT) sgam[i] = pg[i];
        for (int i = tid; i < P.ncis; i += NT) scis[i] = pc[i];
    }
    for (int w = 0; w < W; ++w) {
        const int tb = ltb[w], te = ltb[w + 1];
        const Key* l1 = S.l1[w];
        if (CS > 1) {
            for (int i = tid; i < te - tb; i += NT)
                set_top(tb + i, inb((long long)i * CS + rank, S.N[w], 2, berr)
                                    ? l1[(long long)i * CS + rank] : 0ull);
        } else {
            const long long Nw = S.N[w];
            for (int i = tid; i < te - tb; i += NT) {
                const long long f0 = (long long)i << gsh;
                const long long f1 = min(f0 + (1ll << gsh), Nw);
                Key m = 0ull;
                for (long long f = f0; f < f1; ++f)
                    if (inb(f, Nw, 3, berr)) m = l1[f] > m ? l1[f] : m;
                set_top(tb + i, m);
            }
        }
    }
    for (int i = tid; i < ((T + 31) >> 5); i += NT) dbits[i] = 0u;
    // dictionary bases of the flat index, one per lane (lane w < W)
    const unsigned fb_l = lane < W ? S.fbase[lane] : 0xffffffffu;
    constexpr bool PREF = NT == 128;
    const C2* __restrict__ tiles = cx_t<C2>::tiles(P);
    const C2 zero2 = cx_t<C2>::make(0, 0);

    // frame jobs (step 5).  job_begin: the frame n = nstart + f CS of
    // dictionary v, its level-0 keys, both terms' tile columns and the loads
    // of the first batch of touched chunks (nothing here needs the
    // coefficient).  job_end: the update (eq. fastkernupdate with the
    // modulation of eq. hkj), new chunk keys, further batches, the frame
    // maximum and the top level.
    auto load_batch = [&](JobCtx<C2>& x, const VJob& J, int b0) {
        const DevDict& Dv = sd[x.v];
        const int Mv = Dv.M, Mr = Dv.Mr;
        const unsigned short* lst = chl + clo[x.v];
        const C2* prow = reinterpret_cast<const C2*>(S.plane[x.v]) + (long long)x.n * Dv.Mrp;
        const int nb = min(CB, J.nlist - b0);  // uniform
        x.nb = nb;
        auto load_slot = [&](int q) {
            x.cq[q] = q < nb ? (int)lst[b0 + q] : -1;
            const int m = x.cq[q] * CHUNK + lane;
            const bool ok = x.cq[q] >= 0;
            const bool okm = ok && inb((long long)x.n * Dv.Mrp + m, S.N[x.v] * Dv.Mrp, 4, berr);
            x.val[q] = okm ? prow[okm ? m : 0] : zero2;
            int i0 = m - J.Arow0;
            i0 += i0 < 0 ? Mv : 0;
            int i1 = m - J.Arow1;
            i1 += i1 < 0 ? Mv : 0;
            const bool s0 = ok && m < Mr && x.tb0 >= 0 && i0 < J.R0;
            const bool s1 = ok && m < Mr && x.tb1 >= 0 && i1 < J.R1;
            x.h0[q] = s0 && inb(x.tb0 + i0, P.tiles_len, 5, berr) ? __ldg(tiles + x.tb0 + i0) : zero2;
            x.h1[q] = s1 && inb(x.tb1 + i1, P.tiles_len, 6, berr) ? __ldg(tiles + x.tb1 + i1) : zero2;
            x.hit[q] = s0 || s1;
        };
        // all loads first (one round trip), the second pair only when the
        // batch holds more than two chunks
        load_slot(0);
        load_slot(1);
        if (nb > 2) {
            load_slot(2);
            load_slot(3);
        } else {
            x.cq[2] = x.cq[3] = -1;
        }
    };
    auto job_begin = [&](JobCtx<C2>& x, const VJob& J, int v, int f) {
        const DevDict& Dv = sd[v];
        const int Nv = (int)S.N[v];
        int n = J.nstart + f * CS;
        n -= (n >= Nv) ? Nv : 0;
        n -= (n >= Nv) ? Nv : 0;
        x.v = v;
        x.n = n;
        const Key* l0row = S.l0[v] + (long long)n * Dv.nch;
#pragma unroll
        for (int q = 0; q < MAXL0; ++q) {
            const int c = lane + 32 * q;
            x.l0v[q] = c < Dv.nch && inb((long long)n * Dv.nch + c, S.N[v] * Dv.nch, 7, berr)
                           ? l0row[c] : 0ull;
        }
        x.tb0 = term_col(J.act0, J.Acol0, J.C0, J.R0, J.tile0, n, Nv, x.cc0);
        x.tb1 = term_col(J.act1, J.Acol1, J.C1, J.R1, J.tile1, n, Nv, x.cc1);
        load_batch(x, J, 0);
    };
    auto job_end = [&](JobCtx<C2>& x, const VJob& J, C2 c_main, C2 c_conj, int u) {
        const int v = x.v, n = x.n;
        const DevDict& Dv = sd[v];
        const int Mr = Dv.Mr, nch = Dv.nch;
        const C2* cis_u = scis + sd[u].cis_off;
        const C2 w0 = term_weight(x.tb0, x.cc0, J.qb0, J.dq0, sd[u], cis_u, c_main);
        const C2 w1 = term_weight(x.tb1, x.cc1, J.qb1, J.dq1, sd[u], cis_u, c_conj);
        Key* l0row = S.l0[v] + (long long)n * nch;
        C2* prow = reinterpret_cast<C2*>(S.plane[v]) + (long long)n * Dv.Mrp;
        const unsigned fn = S.fbase[v] + ((unsigned)n << Dv.msh);
        const unsigned tm = tmk[v][lane];
        Key tmax = 0ull;  // maximum of the touched chunks' new keys
        Key e[CB];
        // update and key of one slot
        auto update_slot = [&](int q) {
            const int m = x.cq[q] * CHUNK + lane;
            C2 x2 = x.val[q];
            const C2 d0 = cmul(w0, x.h0[q]);
            x2.x -= d0.x;
            x2.y -= d0.y;
            const C2 d1 = cmul(w1, x.h1[q]);
            x2.x -= d1.x;
            x2.y -= d1.y;
            if (x.hit[q] && inb((long long)n * Dv.Mrp + m, S.N[v] * Dv.Mrp, 8, berr)) prow[m] = x2;
            e[q] = (x.cq[q] >= 0 && m < Mr) ? make_key_sel(x2, fn + m, m, Dv, sgam, P.pedantic)
                                            : 0ull;
        };
        for (int b0 = 0; b0 < J.nlist; b0 += CB) {
            if (b0 > 0) load_batch(x, J, b0);
            const int nb = x.nb;
            update_slot(0);
            update_slot(1);
            warp_max_key2(e[0], e[1]);
            if (lane == 0 && inb(x.cq[0], nch, 9, berr)) l0row[x.cq[0]] = e[0];
            tmax = e[0] > tmax ? e[0] : tmax;
            if (nb > 1) {
                if (lane == 1 && inb(x.cq[1], nch, 9, berr)) l0row[x.cq[1]] = e[1];
                tmax = e[1] > tmax ? e[1] : tmax;
            }
            if (nb > 2) {
                update_slot(2);
                update_slot(3);
                warp_max_key2(e[2], e[3]);
                if (lane == 2 && inb(x.cq[2], nch, 9, berr)) l0row[x.cq[2]] = e[2];
                tmax = e[2] > tmax ? e[2] : tmax;
                if (nb > 3) {
                    if (lane == 3 && inb(x.cq[3], nch, 9, berr)) l0row[x.cq[3]] = e[3];
                    tmax = e[3] > tmax ? e[3] : tmax;
                }
            }
        }
        // frame maximum: the touched chunks' new keys and the untouched
        // chunks' stored ones
        Key fb = tmax;
#pragma unroll
        for (int q = 0; q < MAXL0; ++q)
            if (!((tm >> q) & 1u) && x.l0v[q] > fb) fb = x.l0v[q];
        if (nch > 32 * MAXL0) {
            __syncwarp();  // this warp's level-0 stores are visible to its loads
            for (int c = lane + 32 * MAXL0; c < nch; c += 32) fb = l0row[c] > fb ? l0row[c] : fb;
        }
        const Key fr = warp_max_key(fb);
        if (lane == 0) {
            if (inb(n, S.N[v], 10, berr)) S.l1[v][n] = fr;
            if (CS > 1) {
                const int ti = ltb[v] + (n >> cs_sh);
                if (inb(ti, ltb[v + 1], 11, berr)) set_top(ti, fr);
            } else if (gsh == 0) {
                const int ti = ltb[v] + n;
                if (inb(ti, ltb[v + 1], 11, berr)) set_top(ti, fr);
            } else {
                const int gi = ltb[v] + (n >> gsh);
                const unsigned bit = 1u << (gi & 31);
                if (inb(gi, ltb[v + 1], 12, berr) && !(atomicOr(&dbits[gi >> 5], bit) & bit)) {
                    const int di = atomicAdd(&ndirty, 1);
                    if (inb(di, T, 13, berr)) dlist[di] = (unsigned short)gi;
                }
            }
        }
    };

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
    const unsigned xbytes = (unsigned)(CS * sizeof(Key)) + (budget_ns > 0 ? 8u : 0u);
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

    // loop shape: warp 0 alone scans a small cluster top level; with a warp
    // to spare (more warps than dictionaries) the last warp computes the
    // coefficient and keeps the books while the others build the update
    const bool w0scan = CS > 1 && T <= 256;
    const bool early = NWARPS - 1 >= W;
    unsigned long long it = 0;  // iteration counter (exchange parities)
    for (;;) {
        const int par = (int)(it & 1);
        const unsigned xb = par ? xb1 : xb0;
        const unsigned vb = par ? vb1 : vb0;
        const unsigned xpar = (unsigned)((it >> 1) & 1);
        // ---- 1. scan of the top level, CTA best, cluster exchange ----------
        Key best = 0ull;
        if (w0scan) {
            // a cluster CTA with at most 256 top-level keys: warp 0 scans them
            // and sends, the other warps go straight to the wait
            if (warp == 0) {
                // the lane's scores in position order, the first of equal
                // scores kept
                unsigned e[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) e[q] = lane + 32 * q < T ? tops[lane + 32 * q] : 0u;
                unsigned bs = e[0];
                int bq = 0;
#pragma unroll
                for (int q = 1; q < 8; ++q)
                    if (e[q] > bs) {
                        bs = e[q];
                        bq = q;
                    }
                best = top_best(bs, lane + 32 * bq < T ? (unsigned)(lane + 32 * bq) : NOPOS);
                if (lane == 0) arm_exchange(xb, vb, xbytes, (unsigned)sizeof(C2));
            }
        } else {
            // four independent running maxima of the scores (each keeps the
            // first of equal scores), merged at the end
            unsigned s0 = 0u, s1 = 0u, s2 = 0u, s3 = 0u;
            unsigned p0 = NOPOS, p1 = NOPOS, p2 = NOPOS, p3 = NOPOS;
            int i = tid;
            for (; i + 3 * NT < T; i += 4 * NT) {
                const unsigned e0 = tops[i], e1 = tops[i + NT], e2 = tops[i + 2 * NT],
                               e3 = tops[i + 3 * NT];
                if (e0 > s0 || p0 == NOPOS) { s0 = e0; p0 = (unsigned)i; }
                if (e1 > s1 || p1 == NOPOS) { s1 = e1; p1 = (unsigned)(i + NT); }
                if (e2 > s2 || p2 == NOPOS) { s2 = e2; p2 = (unsigned)(i + 2 * NT); }
                if (e3 > s3 || p3 == NOPOS) { s3 = e3; p3 = (unsigned)(i + 3 * NT); }
            }
            for (; i < T; i += NT) {
                const unsigned e0 = tops[i];
                if (e0 > s0 || p0 == NOPOS) { s0 = e0; p0 = (unsigned)i; }
            }
            // merge: higher score, else lower position (NOPOS is the highest)
            auto pick = [](unsigned& sa, unsigned& pa, unsigned sb, unsigned pb) {
                if (pb != NOPOS && (pa == NOPOS || sb > sa || (sb == sa && pb < pa))) {
                    sa = sb;
                    pa = pb;
                }
            };
            pick(s0, p0, s1, p1);
            pick(s2, p2, s3, p3);
            pick(s0, p0, s2, p2);
            const Key r = top_best(s0, p0);
            if (lane == 0) wsel[warp] = r;
            if (CS > 1 && tid == 0) arm_exchange(xb, vb, xbytes, (unsigned)sizeof(C2));
            __syncthreads();
            best = warp_max_key(lane < NWARPS ? wsel[lane] : 0ull);
        }
        if (CS > 1) {
            if (warp == 0) {
                if (lane < CS) {
                    const unsigned laddr = (unsigned)__cvta_generic_to_shared(&cand[par][rank]);
                    st_async8(mapa_u32(laddr, lane), (unsigned)best, (unsigned)(best >> 32),
                              mapa_u32(xb, lane));
                }
                if (budget_ns > 0 && rank == 0) {
                    int tf = 0;
                    if (lane == 0) tf = (long long)(gtimer() - t_start) > budget_ns ? 1 : 0;
                    tf = __shfl_sync(FULL, tf, 0);
                    if (lane < CS) {
                        const unsigned laddr = (unsigned)__cvta_generic_to_shared(&tmsg[par]);
                        st_async8(mapa_u32(laddr, lane), (unsigned)tf, 0u, mapa_u32(xb, lane));
                    }
                }
            }
            // bounded wait for the CS candidates (and the time-limit message)
            const unsigned long long w0 = gtimer();
            bool ok = true;
            while (!xbar_try(xb, xpar)) {
                if (gtimer() - w0 > 2000000000ull) {
                    ok = false;
                    break;
                }
            }
            best = warp_max_key(lane < CS ? cand[par][lane] : 0ull);
            if (!ok) stop = -2;
        } else if (budget_ns > 0) {
            // single CTA: the time limit is read by one thread before the scan
            // barrier of the next iteration; here it is read after this one
            if (tid == 0) tmsg[par] = (long long)(gtimer() - t_start) > budget_ns ? 1ull : 0ull;
            __syncthreads();
        }

        // ---- 2. selection ---------------------------------------------------
        if (stop == 0) stop = sstop[k & 1];
        if (stop == 0 && budget_ns > 0 && tmsg[par]) stop = -1;
        if (stop == 0 && (unsigned)(best >> 32) == 0u) stop = MP_STOP_ZEROMAX;
        if (stop) break;

        const unsigned flat = 0xffffffffu - (unsigned)(best & 0xffffffffull);
        // dictionary of the flat index: the number of bases w >= 1 at or below it
        const int u = __popc(__ballot_sync(FULL, lane > 0 && lane < W && flat >= fb_l));
        const unsigned rel = flat - __shfl_sync(FULL, fb_l, u);
        const int msh = sd[u].msh;
        const int j = (int)(rel >> msh);
        const int kk = (int)(rel & ((1u << msh) - 1u));
        const int Mu = sd[u].M;
        const bool edge = (kk == 0) || (2 * kk == Mu);
        // the selected coefficient: a single CTA reads it from its plane (it
        // wrote it itself); in a cluster the CTA owning frame j reads it and
        // sends it to every CTA of the cluster (bytes completed on vbar),
        // while the update descriptors are built
        C2 rho = zero2;
        const C2* psel = reinterpret_cast<const C2*>(S.plane[u]) + (long long)j * sd[u].Mrp + kk;
        const bool sel_ok = inb((long long)j * sd[u].Mrp + kk, S.N[u] * sd[u].Mrp, 14, berr) &&
                            inb(kk, sd[u].Mr, 14, berr);
        if (CS == 1) {
            if ((!early || warp == NWARPS - 1) && sel_ok) rho = *psel;
        } else if (warp == NWARPS - 1 && (j & (CS - 1)) == rank) {
            C2 r2 = zero2;
            if (lane == 0 && sel_ok) r2 = *psel;
            r2.x = __shfl_sync(FULL, r2.x, 0);
            r2.y = __shfl_sync(FULL, r2.y, 0);
            if (lane < CS) {
                const unsigned laddr = (unsigned)__cvta_generic_to_shared(&cval[par]);
                send_coef(laddr, lane, r2, vb);
            }
        }

        // ---- 3. per-dictionary update descriptors; 4. real-pair adjustment --
        // eqs. dualatprod / projenfaster: coefficient and energy drop in the
        // planes' precision (gamma is zero away from m = 0 and m = M/2), E
        // accumulated in FP64
        // by the keeper thread, which also writes the atom and the next stop
        // decision
        auto adjust = [&](C2 r, R& cx, R& cy) {
            R Edf;
            if (edge) {
                cx = r.x;
                cy = 0.f;
                Edf = r.x * r.x;
            } else {
                const C2 g = gamma_of(sd[u], sgam, kk);
                if (g.x == 0.f && g.y == 0.f) {
                    cx = r.x;
                    cy = r.y;
                    Edf = R(2) * fma(cx, cx, cy * cy);
                } else {
                    const R inv = R(1) / (R(1) - fma(g.x, g.x, g.y * g.y));
                    cx = (r.x - fma(g.x, r.x, g.y * r.y)) * inv;  // rho - conj(gamma) conj(rho)
                    cy = (r.y - fma(g.y, r.x, -g.x * r.y)) * inv;
                    const R c2 = fma(cx, cx, cy * cy), d2 = fma(cx, cx, -cy * cy);
                    Edf = R(2) * (c2 + fma(g.x, d2, R(-2) * g.y * cx * cy));
                }
            }
            if (tid == KEEPER) {
                E -= (double)Edf;
                if (rank == 0 && inb(k, S.cap, 15, berr)) {
                    mp_atom at;
                    at.dict = u;
                    at.m = kk;
                    at.n = j;
                    at.re = (float)cx;
                    at.im = (float)cy;
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
        };
        // bounded wait for the selected coefficient of a cluster
        auto wait_coef = [&]() -> bool {
            const unsigned long long w0 = gtimer();
            while (!xbar_try(vb, xpar))
                if (gtimer() - w0 > 2000000000ull) return false;
            return true;
        };
        // a warp that builds dictionary v's descriptor also issues the loads
        // of v's first owned frame (128-thread CTAs, which have the
        // registers): they fly while the barrier and the coefficient wait
        JobCtx<C2> px;
        bool pref = false;
        for (int v = warp; v < W; v += NWARPS) {
            const VJob Jv = build_vjob<POW2>(sd, sp, scls, W, S, u, kk, j, edge, v, rank, CS,
                                             cs_sh, lane, &vj[v], chl + clo[v], tmk[v],
                                             clo[v + 1] - clo[v], berr);
            if (PREF && v == warp && Jv.cnt > 0) {
                __syncwarp();  // the chunk list was written by this warp's lanes
                job_begin(px, Jv, v, 0);
                pref = true;
            }
        }
        R cx = R(0), cy = R(0);
        if (early && warp == NWARPS - 1) {
            bool ok = true;
            if (CS > 1) {
                ok = wait_coef();
                rho = cval[par];
            }
            adjust(rho, cx, cy);
            if (lane == 0) {
                scoef[par] = cx_t<C2>::make(cx, cy);
                if (!ok) sbad = 1;
            }
        }
        __syncthreads();
        if (early) {
            if (sbad) {
                stop = -2;
                break;
            }
            const C2 c2 = scoef[par];
            cx = c2.x;
            cy = c2.y;
        } else {
            if (CS > 1) {
                if (!wait_coef()) {
                    stop = -2;
                    break;
                }
                rho = cval[par];
            }
            adjust(rho, cx, cy);
        }
        ++k;

        // ---- 5. frame jobs: the prefetched one, then the rest dealt from one
        //         flat index (warps without a prefetched job first) ----------
        {
            const C2 c_main = cx_t<C2>::make(cx, cy), c_conj = cx_t<C2>::make(cx, -cy);
            if (pref) job_end(px, vj[px.v], c_main, c_conj, u);
            // remaining jobs per dictionary (lane w < W), inclusive prefix
            int cw = lane < W ? vj[lane].cnt : 0;
            const int off = (PREF && lane < NWARPS && cw > 0) ? 1 : 0;  // prefetched
            int pre = cw - off;
#pragma unroll
            for (int o = 1; o < MAXW; o <<= 1) {
                const int y = __shfl_up_sync(FULL, pre, o);
                if (lane >= o) pre += y;
            }
            const int nrem = __shfl_sync(FULL, pre, W - 1);
            const int first = PREF ? ((warp - W) % NWARPS + NWARPS) % NWARPS : warp;
            for (int g = first; g < nrem; g += NWARPS) {
                const int v = __popc(__ballot_sync(FULL, lane < W && g >= pre));
                const int f = g - (v > 0 ? __shfl_sync(FULL, pre, (v + 31) & 31) : 0) +
                              __shfl_sync(FULL, off, v);
                JobCtx<C2> x;
                job_begin(x, vj[v], v, f);
                job_end(x, vj[v], c_main, c_conj, u);
            }
        }
        __syncthreads();

        // ---- 6. groups of touched frames (single CTA, grouped top level) ----
        if (CS == 1 && gsh > 0) {
            const int nd = ndirty;
            for (int i = tid; i < nd; i += NT) {
                const int gi = dlist[i];
                int w = 0;
                while (w + 1 < W && ltb[w + 1] <= gi) ++w;
                const int f0 = (gi - ltb[w]) << gsh;
                const int f1 = min(f0 + (1 << gsh), (int)S.N[w]);
                const Key* l1 = S.l1[w];
                Key m2 = 0ull;
                // the group's level-1 keys, eight independent loads at a time
                for (int f = f0; f < f1; f += 8) {
                    Key e8[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        e8[q] = f + q < f1 && inb(f + q, S.N[w], 16, berr) ? l1[f + q] : 0ull;
#pragma unroll
                    for (int q = 0; q < 8; ++q) m2 = e8[q] > m2 ? e8[q] : m2;
                }
                if (inb(gi, T, 17, berr)) set_top(gi, m2);
                dbits[gi >> 5] = 0u;
            }
            __syncthreads();
            if (tid == 0) ndirty = 0;
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

using LoopKernel_t = void (*)(DevPlan, DevSig*, const int*, long long, double, long long, int,
                              int, long long, double);

// the loop instantiation for a CTA size (0 if unsupported)
template <typename C2>
LoopKernel_t loop_kernel_t(int threads, bool pow2) {
    switch (threads) {
        case 512: return pow2 ? k_mp_loop<512, true, C2> : k_mp_loop<512, false, C2>;
        case 256: return pow2 ? k_mp_loop<256, true, C2> : k_mp_loop<256, false, C2>;
        case 128: return pow2 ? k_mp_loop<128, true, C2> : k_mp_loop<128, false, C2>;
        default: return nullptr;
    }
}
}  // namespace
}  // namespace mpg
