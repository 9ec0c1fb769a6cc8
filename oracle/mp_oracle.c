/*
 * FP64 CPU oracle for matching pursuit on multi-Gabor dictionaries.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's cpu_baseline / reference legs may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * It restates, in plain and slow double precision, what Prusa, Holighaus and
 * Balazs, "Fast Matching Pursuit with Multi-Gabor Dictionaries" (ACM TOMS
 * 47(3), 2021) compute:
 *
 *   ora_kernel   cross-Gram kernel h_{u,v} = D_u^* g_v on the common grid
 *                (Sec. 4, eqs. GramKern / hkj, Sec. 4.2), by direct sum.
 *   ora_dgt      analysis c = D^* x of one reduced Gabor dictionary
 *                (eq. gabdict, Sec. 5 initialisation), by direct sum.
 *   ora_mp_coef  coefficient-domain MP with the truncated Gram matrix
 *                (Alg. 1 with G_eps of eq. truncgram, the residual update of
 *                Alg. 3, real atom pairs of eqs. dualatprod / projenfaster).
 *   ora_mp_plain plain signal-domain MP with real atom pairs (Sec. 2.2 and
 *                eqs. dualatprod / projenfaster with the exact <d, conj d>).
 *   ora_synth    real-signal synthesis from an atom list (eq. idgtreal).
 *
 * Conventions (readings of the paper where it is silent):
 *  - windows are zero-centred: array index i holds g(t) with t = i - w/2;
 *  - signals are circular (indices mod L); atoms
 *      d_{m,n}(l) = g(l - n a) exp(i 2 pi m (l - n a) / M);
 *  - the reduced dictionary keeps m = 0 .. M/2 (M even);
 *  - threshold is absolute: an entry is kept when |h| > eps;
 *  - selection is argmax |rho|^2 over all (w, n, m); ties go to the lowest
 *    (w, n, m) in that lexicographic order;
 *  - for m in {0, M/2} the conjugate partner is missing: c = Re rho,
 *    energy drop c^2, one kernel subtraction;
 *  - otherwise gamma = <d, conj d> (from the truncated own kernel in the
 *    coefficient-domain variant, exact in the plain one),
 *    c = (rho - conj(gamma) conj(rho)) / (1 - |gamma|^2), energy drop per
 *    eq. projenfaster, and both the atom and its conjugate partner
 *    (frequency M - m, coefficient conj(c)) are subtracted wherever their
 *    kernels land inside the reduced rows 0 .. M_v/2;
 *  - stop tests before each selection, in this order: E <= 0 (energy
 *    estimate exhausted), E <= E0 10^(-snr/10) (target reached),
 *    k >= Kmax, and after the search a zero maximum.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORA_PI 3.14159265358979323846

enum { ORA_STOP_SNR = 1, ORA_STOP_KMAX = 2, ORA_STOP_NEGENERGY = 3, ORA_STOP_ZEROMAX = 4 };

static int64_t imod(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}

/* floor division for possibly negative numerators */
static int64_t ifloordiv(int64_t x, int64_t d) {
    int64_t q = x / d;
    if ((x % d != 0) && ((x < 0) != (d < 0))) q -= 1;
    return q;
}

static int imin(int x, int y) { return x < y ? x : y; }
static int imax(int x, int y) { return x > y ? x : y; }

/* e^{i 2 pi q / M} for q = 0..M-1 */
static cplx* cis_table(int M) {
    cplx* t = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    for (int q = 0; q < M; ++q) {
        double th = 2.0 * ORA_PI * (double)q / (double)M;
        t[q] = cos(th) + I * sin(th);
    }
    return t;
}

/* ------------------------------------------------------------------------ */
/* kernels (Sec. 4, 4.2)                                                    */
/* ------------------------------------------------------------------------ */

/* Geometry of h_{u,v}: common grid a_min = min(a_u, a_v), M_max = max(M_u,
 * M_v); tau runs over multiples of a_min for which the window supports
 * t in [-w_u/2, w_u/2) and t - tau in [-w_v/2, w_v/2) overlap. */
void ora_kernel_dims(int wu, int au, int Mu, int wv, int av, int Mv,
                     int* Mx, int* an, int* tau_min, int* ntau) {
    int a_min = imin(au, av);
    int M_max = imax(Mu, Mv);
    int lo = -wu / 2 - wv / 2 + 1;      /* smallest tau with overlap */
    int hi = wu / 2 - 1 + wv / 2;       /* largest tau with overlap  */
    int tmin = (int)(-ifloordiv(-lo, a_min)) * a_min; /* ceil(lo/a)*a */
    int tmax = (int)ifloordiv(hi, a_min) * a_min;
    *Mx = M_max;
    *an = a_min;
    *tau_min = tmin;
    *ntau = (tmax - tmin) / a_min + 1;
}

/* h[(it * Mx + delta) * 2 + {0,1}] = h_{u,v}(delta, tau_min + it * a_min),
 *   h_{u,v}(delta, tau) = sum_t g_u(t) g_v(t - tau) e^{-i 2 pi delta (t - tau) / M_max}
 * which is <d^u_{k,j}, d^v_{m,n}> with the phase e^{i 2 pi k tau / M_u}
 * removed, tau = n a_v - j a_u and delta = m M_max/M_v - k M_max/M_u
 * (derivation of eq. GramKern extended to cross-Gram matrices, Sec. 4.2). */
void ora_kernel(const double* gu, int wu, int au, int Mu,
                const double* gv, int wv, int av, int Mv, double* h) {
    int Mx, an, tmin, ntau;
    ora_kernel_dims(wu, au, Mu, wv, av, Mv, &Mx, &an, &tmin, &ntau);
    cplx* cs = cis_table(Mx);
    for (int it = 0; it < ntau; ++it) {
        int tau = tmin + it * an;
        int t0 = imax(-wu / 2, tau - wv / 2);
        int t1 = imin(wu / 2 - 1, tau + wv / 2 - 1);
        for (int d = 0; d < Mx; ++d) {
            cplx acc = 0.0;
            /* q = d (t - tau) mod M_max, advanced by d per step in t */
            int64_t q = imod((int64_t)d * (t0 - tau), Mx);
            for (int t = t0; t <= t1; ++t) {
                double p = gu[t + wu / 2] * gv[t - tau + wv / 2];
                acc += p * conj(cs[q]);
                q += d;
                if (q >= Mx) q -= Mx;
            }
            h[((size_t)it * Mx + d) * 2 + 0] = creal(acc);
            h[((size_t)it * Mx + d) * 2 + 1] = cimag(acc);
        }
    }
    free(cs);
}

/* ------------------------------------------------------------------------ */
/* analysis (eq. gabdict, reduced dictionary)                               */
/* ------------------------------------------------------------------------ */

/* out[(n * (M/2+1) + m) * 2 + {0,1}] = <x, d_{m,n}>
 *   = sum_{t=-w/2}^{w/2-1} x((n a + t) mod L) g(t) e^{-i 2 pi m t / M} */
void ora_dgt(const double* x, int64_t L, const double* g, int w, int a, int M, double* out) {
    int Mr = M / 2 + 1;
    int64_t N = L / a;
    cplx* cs = cis_table(M);
    double* f = (double*)malloc(sizeof(double) * (size_t)w);
    for (int64_t n = 0; n < N; ++n) {
        for (int i = 0; i < w; ++i) {
            int t = i - w / 2;
            f[i] = x[imod(n * a + t, L)] * g[i];
        }
        for (int m = 0; m < Mr; ++m) {
            cplx acc = 0.0;
            /* q = m t mod M for t = i - w/2, advanced by m per step */
            int64_t q = imod((int64_t)m * (-(w / 2)), M);
            for (int i = 0; i < w; ++i) {
                acc += f[i] * conj(cs[q]);
                q += m;
                if (q >= M) q -= M;
            }
            out[((size_t)n * Mr + m) * 2 + 0] = creal(acc);
            out[((size_t)n * Mr + m) * 2 + 1] = cimag(acc);
        }
    }
    free(f);
    free(cs);
}

/* ------------------------------------------------------------------------ */
/* synthesis (eq. idgtreal)                                                 */
/* ------------------------------------------------------------------------ */

/* y = sum over atoms of  c d + conj(c) conj(d)  (just c d at m in {0, M/2}) */
void ora_synth(int W, const int* wl, const int* av, const int* Mv, const double* gcat,
               int64_t K, const int32_t* dict, const int32_t* mm, const int64_t* nn,
               const double* cre, const double* cim, int64_t L, double* y) {
    int64_t off[64];
    int64_t o = 0;
    for (int w = 0; w < W; ++w) { off[w] = o; o += wl[w]; }
    memset(y, 0, sizeof(double) * (size_t)L);
    for (int64_t k = 0; k < K; ++k) {
        int u = dict[k];
        int w = wl[u], a = av[u], M = Mv[u];
        const double* g = gcat + off[u];
        int m = mm[k];
        int64_t n = nn[k];
        cplx c = cre[k] + I * cim[k];
        int edge = (m == 0) || (2 * m == M);
        for (int i = 0; i < w; ++i) {
            int t = i - w / 2;
            double th = 2.0 * ORA_PI * (double)imod((int64_t)m * t, M) / (double)M;
            cplx d = g[i] * (cos(th) + I * sin(th));
            double v = edge ? creal(c * d) : 2.0 * creal(c * d);
            y[imod(n * a + t, L)] += v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* shared MP bookkeeping                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int W;
    int w[64], a[64], M[64], Mr[64];
    int64_t N[64];
    const double* g[64];
    int64_t L;
    cplx* rho[64];          /* residual coefficients, [N][Mr] */
    double* fbest[64];      /* per frame: max |rho|^2 */
    int* farg[64];          /* per frame: its (lowest) bin */
    double* fsecond[64];    /* per frame: second largest |rho|^2 */
    unsigned char* touched[64];
    int pedantic;           /* selection score = energy drop of eq. projenfaster */
    cplx* gam[64];          /* <d_m, conj d_m> used by the score, m = 0..M/2 */
} mpstate;

/* eq. projenfaster: energy removed by subtracting the real pair with the
 * least-squares coefficient of eq. dualatprod (c^2 for m in {0, M/2}) */
static double pair_energy(cplx rho, cplx gamma, int edge) {
    if (edge) return creal(rho) * creal(rho);
    double ag2 = creal(gamma) * creal(gamma) + cimag(gamma) * cimag(gamma);
    cplx c = (rho - conj(gamma) * conj(rho)) / (1.0 - ag2);
    double x = creal(c), y = cimag(c);
    return 2.0 * (x * x + y * y + creal(gamma) * (x * x - y * y) - 2.0 * cimag(gamma) * x * y);
}

/* selection score of coefficient m of dictionary v: |rho|^2 (Sec. 5.1 as
 * used in practice) or, pedantic, the pair energy drop (Sec. 5) */
static double score(const mpstate* s, int v, int m, cplx r) {
    if (!s->pedantic) return creal(r) * creal(r) + cimag(r) * cimag(r);
    int edge = (m == 0) || (2 * m == s->M[v]);
    return pair_energy(r, s->gam[v][m], edge);
}

static void frame_rescan(mpstate* s, int v, int64_t n) {
    int Mr = s->Mr[v];
    const cplx* r = s->rho[v] + (size_t)n * Mr;
    double b = -1.0, b2 = -1.0;
    int arg = 0;
    for (int m = 0; m < Mr; ++m) {
        double sc = score(s, v, m, r[m]);
        if (sc > b) { b2 = b; b = sc; arg = m; }
        else if (sc > b2) { b2 = sc; }
    }
    s->fbest[v][n] = b;
    s->farg[v][n] = arg;
    s->fsecond[v][n] = b2;
}

static int state_init(mpstate* s, int W, const int* wl, const int* a, const int* M,
                      const double* gcat, int64_t L) {
    memset(s, 0, sizeof(*s));
    if (W < 1 || W > 64) return -1;
    s->W = W;
    s->L = L;
    int64_t o = 0;
    for (int w = 0; w < W; ++w) {
        s->w[w] = wl[w]; s->a[w] = a[w]; s->M[w] = M[w];
        s->Mr[w] = M[w] / 2 + 1;
        s->N[w] = L / a[w];
        s->g[w] = gcat + o;
        o += wl[w];
        size_t P = (size_t)s->N[w] * s->Mr[w];
        s->rho[w] = (cplx*)calloc(P, sizeof(cplx));
        s->fbest[w] = (double*)malloc(sizeof(double) * (size_t)s->N[w]);
        s->fsecond[w] = (double*)malloc(sizeof(double) * (size_t)s->N[w]);
        s->farg[w] = (int*)malloc(sizeof(int) * (size_t)s->N[w]);
        s->touched[w] = (unsigned char*)calloc((size_t)s->N[w], 1);
        s->gam[w] = (cplx*)calloc((size_t)s->Mr[w], sizeof(cplx));
    }
    return 0;
}

static void state_free(mpstate* s) {
    for (int w = 0; w < s->W; ++w) {
        free(s->rho[w]); free(s->fbest[w]); free(s->fsecond[w]);
        free(s->farg[w]); free(s->touched[w]); free(s->gam[w]);
    }
}

static void analyse_all(mpstate* s, const double* x) {
    for (int w = 0; w < s->W; ++w) {
        double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)s->N[w] * s->Mr[w]);
        ora_dgt(x, s->L, s->g[w], s->w[w], s->a[w], s->M[w], tmp);
        size_t P = (size_t)s->N[w] * s->Mr[w];
        for (size_t p = 0; p < P; ++p) s->rho[w][p] = tmp[2 * p] + I * tmp[2 * p + 1];
        free(tmp);
        for (int64_t n = 0; n < s->N[w]; ++n) frame_rescan(s, w, n);
    }
}

/* argmax over all frames; returns best score, writes position and runner-up */
static double select_max(const mpstate* s, int* bu, int* bk, int64_t* bj, double* second) {
    double best = -1.0, sec = -1.0;
    int u = 0, k = 0;
    int64_t j = 0;
    for (int w = 0; w < s->W; ++w) {
        for (int64_t n = 0; n < s->N[w]; ++n) {
            double f = s->fbest[w][n];
            if (f > best) {
                sec = best > s->fsecond[w][n] ? best : s->fsecond[w][n];
                best = f; u = w; k = s->farg[w][n]; j = n;
            } else if (f > sec) {
                sec = f;
            }
        }
    }
    *bu = u; *bk = k; *bj = j;
    *second = sec;
    return best;
}

/* full scan, used only as a cross-check of the per-frame bookkeeping */
static double select_full(const mpstate* s, int* bu, int* bk, int64_t* bj) {
    double best = -1.0;
    for (int w = 0; w < s->W; ++w)
        for (int64_t n = 0; n < s->N[w]; ++n)
            for (int m = 0; m < s->Mr[w]; ++m) {
                cplx r = s->rho[w][(size_t)n * s->Mr[w] + m];
                double sc = score(s, w, m, r);
                if (sc > best) { best = sc; *bu = w; *bk = m; *bj = n; }
            }
    return best;
}

/* eqs. dualatprod / projenfaster (with conj(gamma) in the numerator, which
 * is the least-squares solution; it equals the printed form for real gamma) */
static cplx dual_coef(cplx rho, cplx gamma, double* Edrop) {
    double ag2 = creal(gamma) * creal(gamma) + cimag(gamma) * cimag(gamma);
    cplx c = (rho - conj(gamma) * conj(rho)) / (1.0 - ag2);
    double x = creal(c), y = cimag(c);
    *Edrop = 2.0 * (x * x + y * y + creal(gamma) * (x * x - y * y) - 2.0 * cimag(gamma) * x * y);
    return c;
}

#define ORA_FLAG_FULLSCAN 1
#define ORA_FLAG_PEDANTIC 2

typedef struct {
    int32_t* dict; int32_t* m; int64_t* n;
    double* re; double* im; double* E;
    double* s1; double* s2;
} atom_out;

/* stop tests before selection; returns 0 to continue */
static int stop_before(double E, double thr, int64_t k, int64_t kmax) {
    if (E <= 0.0) return ORA_STOP_NEGENERGY;
    if (E <= thr) return ORA_STOP_SNR;
    if (k >= kmax) return ORA_STOP_KMAX;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* coefficient-domain MP with G_eps (Alg. 1, eq. truncgram, Alg. 3)         */
/* ------------------------------------------------------------------------ */

typedef struct { int delta; int tau; cplx h; } kentry;

typedef struct {
    int Mx, an, tmin, ntau;
    int nent;
    kentry* ent;       /* entries with |h| > eps */
    cplx* full;        /* full kernel [ntau][Mx] (for gamma on the diagonal) */
} kern;

/* subtract coef * G_eps(., (u, kk, j)) from all reduced rows of dictionary v
 * (the conjugate partner is handled by the caller with kk -> M_u - kk) */
static void kernel_subtract(mpstate* s, const kern* K, int u, int v, int kk, int64_t j, cplx coef) {
    int Mu = s->M[u], Mv = s->M[v], au = s->a[u], avv = s->a[v];
    int Mx = K->Mx;
    int64_t kf = (int64_t)kk * (Mx / Mu);     /* k on the common grid */
    int fr = Mx / Mv;                          /* frequency subsampling */
    int64_t Nv = s->N[v];
    int Mr = s->Mr[v];
    for (int e = 0; e < K->nent; ++e) {
        const kentry* E = &K->ent[e];
        int64_t num = (int64_t)E->tau + j * au;  /* = n a_v */
        if (imod(num, avv) != 0) continue;
        int64_t n = imod(num / avv, Nv);
        int64_t mf = imod(kf + E->delta, Mx);     /* = m M_max / M_v */
        if (mf % fr != 0) continue;
        int m = (int)(mf / fr);
        if (m >= Mr) continue;
        /* modulation of eq. hkj: e^{i 2 pi k tau / M_u} */
        double th = 2.0 * ORA_PI * (double)imod((int64_t)kk * E->tau, Mu) / (double)Mu;
        cplx ph = cos(th) + I * sin(th);
        s->rho[v][(size_t)n * Mr + m] -= coef * ph * E->h;
        s->touched[v][n] = 1;
    }
}

/* Alg. 2: approximate coefficient-domain MP with resets.  Before each
 * selection, after the stop tests: when resets are enabled (reset_it > 0 or
 * reset_db < 0) and at least one atom was selected since the last reset, and
 * either reset_it selections have been made since it or the estimate has
 * fallen by more than |reset_db| dB below the energy at the last reset,
 * 10 log10(E_k / E_out) < reset_db, the residual is recomputed in the signal
 * domain, r_out = x - (synthesis of all atoms so far), E_out = E_k =
 * ||r_out||^2, the coefficients are re-analysed from r_out, and the stop
 * tests are applied again.  reset_it = 0 and reset_db = 0 disable resets. */
int ora_mp_coef_reset(int W, const int* wl, const int* a, const int* M, const double* gcat,
                      const double* x, int64_t L, double eps, int64_t kmax, double target_db,
                      int flags, int64_t reset_it, double reset_db,
                      int32_t* o_dict, int32_t* o_m, int64_t* o_n, double* o_re, double* o_im,
                      double* o_E, double* o_s1, double* o_s2,
                      int64_t* n_atoms, int* stop_reason, double* E0_out, double* planes_out,
                      int64_t* n_resets);

int ora_mp_coef(int W, const int* wl, const int* a, const int* M, const double* gcat,
                const double* x, int64_t L, double eps, int64_t kmax, double target_db, int flags,
                int32_t* o_dict, int32_t* o_m, int64_t* o_n, double* o_re, double* o_im,
                double* o_E, double* o_s1, double* o_s2,
                int64_t* n_atoms, int* stop_reason, double* E0_out, double* planes_out) {
    int64_t nr = 0;
    return ora_mp_coef_reset(W, wl, a, M, gcat, x, L, eps, kmax, target_db, flags, 0, 0.0,
                             o_dict, o_m, o_n, o_re, o_im, o_E, o_s1, o_s2, n_atoms, stop_reason,
                             E0_out, planes_out, &nr);
}

int ora_mp_coef_reset(int W, const int* wl, const int* a, const int* M, const double* gcat,
                      const double* x, int64_t L, double eps, int64_t kmax, double target_db,
                      int flags, int64_t reset_it, double reset_db,
                      int32_t* o_dict, int32_t* o_m, int64_t* o_n, double* o_re, double* o_im,
                      double* o_E, double* o_s1, double* o_s2,
                      int64_t* n_atoms, int* stop_reason, double* E0_out, double* planes_out,
                      int64_t* n_resets) {
    mpstate s;
    if (state_init(&s, W, wl, a, M, gcat, L)) return -1;

    /* precompute kernels for all ordered pairs (Sec. 4.1, 4.2) */
    kern* K = (kern*)calloc((size_t)W * W, sizeof(kern));
    for (int u = 0; u < W; ++u)
        for (int v = 0; v < W; ++v) {
            kern* k = &K[u * W + v];
            ora_kernel_dims(s.w[u], s.a[u], s.M[u], s.w[v], s.a[v], s.M[v],
                            &k->Mx, &k->an, &k->tmin, &k->ntau);
            double* h = (double*)malloc(sizeof(double) * 2 * (size_t)k->ntau * k->Mx);
            ora_kernel(s.g[u], s.w[u], s.a[u], s.M[u], s.g[v], s.w[v], s.a[v], s.M[v], h);
            k->full = (cplx*)malloc(sizeof(cplx) * (size_t)k->ntau * k->Mx);
            int cnt = 0;
            for (size_t p = 0; p < (size_t)k->ntau * k->Mx; ++p) {
                k->full[p] = h[2 * p] + I * h[2 * p + 1];
                if (cabs(k->full[p]) > eps) cnt++;
            }
            k->ent = (kentry*)malloc(sizeof(kentry) * (size_t)(cnt > 0 ? cnt : 1));
            k->nent = 0;
            for (int it = 0; it < k->ntau; ++it)
                for (int d = 0; d < k->Mx; ++d) {
                    cplx hv = k->full[(size_t)it * k->Mx + d];
                    if (cabs(hv) > eps) {
                        kentry* E = &k->ent[k->nent++];
                        E->delta = d;
                        E->tau = k->tmin + it * k->an;
                        E->h = hv;
                    }
                }
            free(h);
        }
    /* <d_m, conj d_m> from the truncated own kernel (Sec. 5.2) */
    for (int u = 0; u < W; ++u) {
        const kern* Kuu = &K[u * W + u];
        int it0 = (0 - Kuu->tmin) / Kuu->an;
        for (int m = 1; 2 * m < s.M[u]; ++m) {
            cplx gv = Kuu->full[(size_t)it0 * Kuu->Mx + imod((int64_t)s.M[u] - 2 * m, s.M[u])];
            s.gam[u][m] = cabs(gv) > eps ? gv : 0.0;
        }
    }
    s.pedantic = (flags & ORA_FLAG_PEDANTIC) != 0;

    analyse_all(&s, x);
    double E0 = 0.0;
    for (int64_t l = 0; l < L; ++l) E0 += x[l] * x[l];
    double E = E0;
    double thr = E0 * pow(10.0, -target_db / 10.0);
    int64_t k = 0;
    int stop = 0;
    const int resets = reset_it > 0 || reset_db < 0.0;
    double E_out = E0;
    int64_t k_out = 0;
    *n_resets = 0;
    double* rout = resets ? (double*)malloc(sizeof(double) * (size_t)L) : NULL;
    for (;;) {
        stop = stop_before(E, thr, k, kmax);
        if (stop) break;
        if (resets && k > k_out &&
            ((reset_it > 0 && k - k_out >= reset_it) ||
             (reset_db < 0.0 && 10.0 * log10(E / E_out) < reset_db))) {
            /* r_out = x - D c for all atoms so far (eq. idgtreal) */
            ora_synth(W, wl, a, M, gcat, k, o_dict, o_m, o_n, o_re, o_im, L, rout);
            double Er = 0.0;
            for (int64_t l = 0; l < L; ++l) {
                rout[l] = x[l] - rout[l];
                Er += rout[l] * rout[l];
            }
            E = E_out = Er;
            k_out = k;
            analyse_all(&s, rout);
            (*n_resets)++;
            continue;
        }
        int u, kk;
        int64_t j;
        double sec;
        double best = select_max(&s, &u, &kk, &j, &sec);
        if (flags & ORA_FLAG_FULLSCAN) {
            int u2 = 0, k2 = 0; int64_t j2 = 0;
            double b2 = select_full(&s, &u2, &k2, &j2);
            if (b2 != best || u2 != u || k2 != kk || j2 != j) { stop = -99; break; }
        }
        if (!(best > 0.0)) { stop = ORA_STOP_ZEROMAX; break; }
        cplx rho = s.rho[u][(size_t)j * s.Mr[u] + kk];
        int Mu = s.M[u];
        cplx c;
        double Ed;
        int edge = (kk == 0) || (2 * kk == Mu);
        if (edge) {
            c = creal(rho);
            Ed = creal(rho) * creal(rho);
        } else {
            /* <d, conj d> read off the truncated own kernel at tau = 0,
             * frequency offset (M - k) - k; zero when below threshold */
            const kern* Kuu = &K[u * W + u];
            int it0 = (0 - Kuu->tmin) / Kuu->an;
            cplx gam = Kuu->full[(size_t)it0 * Kuu->Mx + imod((int64_t)Mu - 2 * kk, Mu)];
            if (!(cabs(gam) > eps)) gam = 0.0;
            c = dual_coef(rho, gam, &Ed);
        }
        E -= Ed;
        if (o_dict) {
            o_dict[k] = u; o_m[k] = kk; o_n[k] = j;
            o_re[k] = creal(c); o_im[k] = cimag(c); o_E[k] = E;
            if (o_s1) { o_s1[k] = sqrt(best); o_s2[k] = sec > 0 ? sqrt(sec) : 0.0; }
        }
        /* Alg. 3: subtract the atom and its conjugate partner in every dictionary */
        for (int v = 0; v < W; ++v) {
            kernel_subtract(&s, &K[u * W + v], u, v, kk, j, c);
            if (!edge) kernel_subtract(&s, &K[u * W + v], u, v, Mu - kk, j, conj(c));
        }
        for (int v = 0; v < W; ++v)
            for (int64_t n = 0; n < s.N[v]; ++n)
                if (s.touched[v][n]) { frame_rescan(&s, v, n); s.touched[v][n] = 0; }
        k++;
    }
    *n_atoms = k;
    *stop_reason = stop;
    if (E0_out) *E0_out = E0;
    if (planes_out) {
        size_t o = 0;
        for (int w = 0; w < W; ++w) {
            size_t P = (size_t)s.N[w] * s.Mr[w];
            for (size_t p = 0; p < P; ++p) {
                planes_out[2 * (o + p)] = creal(s.rho[w][p]);
                planes_out[2 * (o + p) + 1] = cimag(s.rho[w][p]);
            }
            o += P;
        }
    }
    for (int i = 0; i < W * W; ++i) { free(K[i].ent); free(K[i].full); }
    free(K);
    free(rout);
    state_free(&s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* plain signal-domain MP (Sec. 2.2) with real atom pairs                   */
/* ------------------------------------------------------------------------ */

static void reanalyse_frame(mpstate* s, const double* r, int v, int64_t n, const cplx* cs) {
    int w = s->w[v], a = s->a[v], M = s->M[v], Mr = s->Mr[v];
    const double* g = s->g[v];
    cplx* out = s->rho[v] + (size_t)n * Mr;
    for (int m = 0; m < Mr; ++m) {
        cplx acc = 0.0;
        for (int i = 0; i < w; ++i) {
            int t = i - w / 2;
            acc += r[imod(n * a + t, s->L)] * g[i] * conj(cs[imod((int64_t)m * t, M)]);
        }
        out[m] = acc;
    }
}

int ora_mp_plain(int W, const int* wl, const int* a, const int* M, const double* gcat,
                 const double* x, int64_t L, int64_t kmax, double target_db, int flags,
                 int32_t* o_dict, int32_t* o_m, int64_t* o_n, double* o_re, double* o_im,
                 double* o_E, double* o_s1, double* o_s2,
                 int64_t* n_atoms, int* stop_reason, double* E0_out, double* resid_out) {
    mpstate s;
    if (state_init(&s, W, wl, a, M, gcat, L)) return -1;
    double* r = (double*)malloc(sizeof(double) * (size_t)L);
    memcpy(r, x, sizeof(double) * (size_t)L);
    cplx* cs[64];
    for (int w = 0; w < W; ++w) cs[w] = cis_table(s.M[w]);
    /* exact <d_m, conj d_m> = sum_t g(t)^2 e^{i 4 pi m t / M} */
    for (int w = 0; w < W; ++w)
        for (int m = 1; 2 * m < s.M[w]; ++m) {
            cplx acc = 0.0;
            for (int i = 0; i < s.w[w]; ++i) {
                int t = i - s.w[w] / 2;
                acc += s.g[w][i] * s.g[w][i] * cs[w][imod((int64_t)2 * m * t, s.M[w])];
            }
            s.gam[w][m] = acc;
        }
    s.pedantic = (flags & ORA_FLAG_PEDANTIC) != 0;
    analyse_all(&s, r);
    double E0 = 0.0;
    for (int64_t l = 0; l < L; ++l) E0 += x[l] * x[l];
    double E = E0;
    double thr = E0 * pow(10.0, -target_db / 10.0);
    int64_t k = 0;
    int stop = 0;
    for (;;) {
        stop = stop_before(E, thr, k, kmax);
        if (stop) break;
        int u, kk;
        int64_t j;
        double sec;
        double best = select_max(&s, &u, &kk, &j, &sec);
        if (flags & ORA_FLAG_FULLSCAN) {
            int u2 = 0, k2 = 0; int64_t j2 = 0;
            double b2 = select_full(&s, &u2, &k2, &j2);
            if (b2 != best || u2 != u || k2 != kk || j2 != j) { stop = -99; break; }
        }
        if (!(best > 0.0)) { stop = ORA_STOP_ZEROMAX; break; }
        int w = s.w[u], au = s.a[u], Mu = s.M[u];
        const double* g = s.g[u];
        cplx rho = s.rho[u][(size_t)j * s.Mr[u] + kk];
        int edge = (kk == 0) || (2 * kk == Mu);
        cplx c;
        double Ed;
        if (edge) {
            c = creal(rho);
            Ed = creal(rho) * creal(rho);
        } else {
            /* exact <d, conj d> = sum_l d(l)^2 */
            cplx gam = 0.0;
            for (int i = 0; i < w; ++i) {
                int t = i - w / 2;
                cplx d = g[i] * cs[u][imod((int64_t)kk * t, Mu)];
                gam += d * d;
            }
            c = dual_coef(rho, gam, &Ed);
        }
        E -= Ed;
        if (o_dict) {
            o_dict[k] = u; o_m[k] = kk; o_n[k] = j;
            o_re[k] = creal(c); o_im[k] = cimag(c); o_E[k] = E;
            if (o_s1) { o_s1[k] = sqrt(best); o_s2[k] = sec > 0 ? sqrt(sec) : 0.0; }
        }
        /* subtract the real atom (pair) in the signal domain */
        for (int i = 0; i < w; ++i) {
            int t = i - w / 2;
            cplx d = g[i] * cs[u][imod((int64_t)kk * t, Mu)];
            double v = edge ? creal(c * d) : 2.0 * creal(c * d);
            r[imod(j * au + t, L)] -= v;
        }
        /* re-analyse every frame whose window overlaps the atom's support */
        for (int v = 0; v < W; ++v) {
            int64_t lo = j * au - w / 2, hi = j * au + w / 2 - 1;   /* atom support */
            int wv = s.w[v], av = s.a[v];
            /* frames n with [n a_v - w_v/2, n a_v + w_v/2 - 1] meeting [lo, hi] */
            int64_t n0 = -ifloordiv(-(lo - wv / 2 + 1), av);
            int64_t n1 = ifloordiv(hi + wv / 2, av);
            if (n1 - n0 + 1 >= s.N[v]) { n0 = 0; n1 = s.N[v] - 1; }
            for (int64_t nn = n0; nn <= n1; ++nn) {
                int64_t n = imod(nn, s.N[v]);
                reanalyse_frame(&s, r, v, n, cs[v]);
                frame_rescan(&s, v, n);
            }
        }
        k++;
    }
    *n_atoms = k;
    *stop_reason = stop;
    if (E0_out) *E0_out = E0;
    if (resid_out) memcpy(resid_out, r, sizeof(double) * (size_t)L);
    for (int w = 0; w < W; ++w) free(cs[w]);
    free(r);
    state_free(&s);
    return 0;
}
