/*
 * mpgabor -- matching pursuit on multi-Gabor dictionaries, GB300 (sm_103a).
 *
 * C ABI of the GPU library libmpgabor.so.  It decomposes real signals x over
 * the concatenation of W Gabor dictionaries D_w = D_(g_w, a_w, M_w)
 * (eq. gabdict, Sec. 2.1) with the coefficient-domain matching pursuit of
 * Alg. 1, using the truncated Gram matrix G_eps (eq. truncgram) in the
 * kernel form of eqs. GramKern / hkj / fastkernupdate and the cross-kernels
 * of Sec. 4.2, with real atom pairs (eqs. idgtreal, dualatprod,
 * projenfaster) and the residual update of Alg. 3.
 *
 * Conventions shared by all calls
 *  - Windows are caller-supplied real arrays of even length w; element i is
 *    g(t) with t = i - w/2 (the window is zero-centred on the circle).  The
 *    library uses them as given (normalise them to unit l2 norm for MP in the
 *    paper's sense).
 *  - Signals are real float32, circular of length L.  L must be a multiple of
 *    every a_w and every M_w, and L >= w_u + w_v for all pairs u, v.
 *  - Coefficients are kept for the reduced dictionary, m = 0 .. M_w/2.
 *  - Atoms are reported as (w, m, n, c): the signal part is
 *    c d + conj(c) conj(d) for 0 < m < M_w/2 and c d for m in {0, M_w/2}
 *    (eq. idgtreal), d(l) = g(l - n a) exp(i 2 pi m (l - n a) / M).
 *  - Device pointers are used on the plan's CUDA stream; the caller owns all
 *    input and output buffers, the library owns everything it allocates.
 *  - Every int-returning call returns MP_OK (0) or a negative MP_E* code and
 *    never aborts; mp_last_error() then describes the failure (thread-local).
 *  - Not thread-safe per object: one host thread at a time per plan / state.
 */
#ifndef MPGABOR_H
#define MPGABOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mp_plan mp_plan;   /* opaque: dictionaries, kernels, tables */
typedef struct mp_state mp_state; /* opaque: coefficient planes, trees, atoms */

/* one selected real atom (pair) */
typedef struct {
    int32_t dict; /* dictionary index w, 0 .. W-1 */
    int32_t m;    /* frequency index, 0 .. M_w/2 */
    int64_t n;    /* frame (time shift) index, 0 .. L/a_w - 1 */
    float re;     /* adjusted coefficient c (eq. dualatprod) */
    float im;
} mp_atom;

enum {
    MP_OK = 0,
    MP_EINVAL = -1,     /* bad argument */
    MP_ENOTCOMPAT = -2, /* dictionary set violates the compatibility rules of Sec. 2.1 */
    MP_ENOMEM = -3,     /* device or host allocation failed */
    MP_ECUDA = -4,      /* a CUDA call failed */
    MP_ETIMEOUT = -5    /* mp_run hit its time limit; the state stays valid */
};

/* per-signal stop reason reported by mp_run */
enum {
    MP_STOP_NONE = 0,      /* not stopped yet (time limit reached) */
    MP_STOP_SNR = 1,       /* E_k <= ||x||^2 10^(-target/10) */
    MP_STOP_KMAX = 2,      /* K_max atoms selected */
    MP_STOP_NEGENERGY = 3, /* energy estimate E_k <= 0 (Sec. 6.1 rule) */
    MP_STOP_ZEROMAX = 4,   /* all coefficients are zero */
    MP_STOP_INVALID = 5    /* the signal holds NaN or Inf */
};

/* mp_plan_create flags (bit set) */
enum {
    MP_ANALYSIS_FP32 = 0,   /* analysis as an FP32 DFT-GEMM on the SIMT cores (default) */
    MP_ANALYSIS_BF16X3 = 1, /* analysis as a split-BF16 three-product DFT-GEMM on tcgen05;
                               needs every a a multiple of 64 and every w/2 a multiple of a */
    MP_PEDANTIC = 2,        /* select by the real-pair energy drop of eq. projenfaster
                               ("pedantic", Sec. 5) instead of |rho|^2 */
    MP_COEF_FP64 = 4        /* FP64 coefficient planes, kernel tiles, modulation and
                               <d, conj d> tables, FP64 analysis (DFT-GEMM on the FP64
                               pipe): the paper's precision (Sec. 6), for parity runs;
                               not combinable with MP_ANALYSIS_BF16X3 */
};

/*
 * Build a plan for W dictionaries (Sec. 4.1-4.2, Sec. 5 initialisation).
 *   windows[w]  host pointer to win_len[w] doubles (zero-centred window)
 *   a[w], M[w]  time shift and number of channels; M even, M/a integer; all
 *               a pairwise divisible by the smaller one, all M pairwise
 *               dividing the larger one (Sec. 2.1 compatibility)
 *   kern_thr    eps >= 0 of eq. truncgram, absolute: kernel entries with
 *               |h| <= eps are dropped (Fig. 1 uses 1e-4, i.e. -80 dB)
 *   flags       MP_ANALYSIS_* | MP_PEDANTIC
 *   cuda_stream cudaStream_t used by every call on this plan (NULL: legacy)
 * Computes on the device, in FP64, every cross-kernel h_{u,v} on the common
 * grid (a_min, M_max), thresholds it, splits it into dense FP32 tiles per
 * grid alignment class (and FP64 tiles with MP_COEF_FP64), and derives
 * <d, conj d> for every own-dictionary frequency.  Cost and memory are
 * independent of the signal length.
 * Returns MP_EINVAL / MP_ENOTCOMPAT on bad input, MP_ECUDA / MP_ENOMEM on
 * device failure; *out is set only on success.  Synchronises the stream.
 */
int mp_plan_create(mp_plan** out, int W, const double* const* windows, const int* win_len,
                   const int* a, const int* M, double kern_thr, unsigned flags,
                   void* cuda_stream);
void mp_plan_destroy(mp_plan* plan);

/*
 * Plan introspection (tests and tools).
 * mp_plan_kernel_dims: geometry of h_{u,v}: M_max, a_min, smallest tau and
 * number of tau values (multiples of a_min where the windows overlap).
 * mp_plan_kernel_fp64: copies the untruncated FP64 kernel computed on the
 * device, h[(it * M_max + delta) * 2 + {0,1}] = h_{u,v}(delta, tau_min +
 * it a_min), h_{u,v}(delta, tau) = sum_t g_u(t) g_v(t - tau)
 * e^{-i 2 pi delta (t - tau) / M_max}; host buffer of 2 ntau M_max doubles.
 * mp_plan_tile_info: for alignment class (cf, ct) of pair (u, v) writes
 * info[0..6] = {rf, rt, R, C, i_lo, c_lo, n_nonzero}: the class tile holds
 * T[c][i] = h_eps(delta = (i_lo + i) rf - cf, tau = (c_lo + c) a_v - ct a_u)
 * for i < R, c < C.  mp_plan_tile copies it (R C complex floats, host).
 * mp_plan_gamma copies <d, conj d> (thresholded, FP32) for k = 0 .. M_u/2.
 */
int mp_plan_kernel_dims(const mp_plan* plan, int u, int v, int* M_max, int* a_min,
                        int* tau_min, int* ntau);
int mp_plan_kernel_fp64(const mp_plan* plan, int u, int v, double* h_host, int64_t cap_doubles);
int mp_plan_tile_info(const mp_plan* plan, int u, int v, int cf, int ct, int* info7);
int mp_plan_tile(const mp_plan* plan, int u, int v, int cf, int ct, float* tile_host,
                 int64_t cap_floats);
int mp_plan_gamma(const mp_plan* plan, int u, float* gamma_host, int64_t cap_floats);

/*
 * Analysis, Alg. 1 initialisation: rho_0 = D_w^* x for every dictionary
 * (reduced rows m = 0 .. M_w/2), E_0 = ||x||^2 in FP64, and the max trees.
 *   B        number of signals (>= 1); each is decomposed independently
 *   x_dev[b] device pointer to L[b] floats (read only during the call's
 *            stream work): device memory of the plan's device, managed or
 *            page-locked host memory; a pageable host address or memory of
 *            another device is MP_EINVAL (checked with
 *            cudaPointerGetAttributes when the plan's stream is not being
 *            captured; the signals are copied into the state by one kernel
 *            per 256 signals)
 * If *state is NULL a new state is allocated; if it is non-NULL it must come
 * from the same plan with the same B and lengths and is reused (all previous
 * atoms are discarded).  Asynchronous on the plan's stream; reusing a state,
 * mp_analyze (device pointers) followed by mp_run_async can be captured into
 * a CUDA graph (the tensor-core error check is skipped while capturing).
 * mp_analyze_host is the same with host pointers; it copies each signal to
 * the device inside the call (end-to-end path).
 */
int mp_analyze(const mp_plan* plan, mp_state** state, int B, const float* const* x_dev,
               const int64_t* L);
int mp_analyze_host(const mp_plan* plan, mp_state** state, int B, const float* const* x_host,
                    const int64_t* L);

/* copies the current residual coefficients rho of signal sig, dictionary w
 * to host: (L/a_w) x (M_w/2+1) complex floats, frame-major. */
int mp_state_coefficients(const mp_state* state, int sig, int w, float* host, int64_t cap_floats);

/*
 * Matching pursuit, Alg. 1 with Alg. 3, for every signal of the state, in
 * one persistent launch (one CTA per signal).  Per iteration: select the
 * coefficient of largest |rho|^2 over all dictionaries (ties: lowest
 * (w, n, m)); adjust it to the real-pair coefficient c (eq. dualatprod with
 * conj(gamma); c = Re rho at m in {0, M/2}); E_{k+1} = E_k - energy drop
 * (eq. projenfaster, FP64); subtract c G_eps(., p) and, for the conjugate
 * partner, conj(c) G_eps(., conj p) from every dictionary's coefficients.
 * Stop tests run before each selection: E_k <= 0, then
 * 10 log10(E_0 / E_k) >= target_snr_db, then k >= K_max (K_max counts all
 * atoms of the state, so a second call continues a decomposition), then a
 * zero maximum.
 * Outputs (host arrays of B, may be NULL): atoms so far, stop reason,
 * 10 log10(E_0 / E_k).  Synchronous.  Returns MP_ETIMEOUT if the time limit
 * (mp_state_set_time_limit) ended the launch first; call again to go on.
 * mp_run_async only enqueues the launch (no outputs, no synchronisation),
 * e.g. for stream capture; read results with mp_get_status.
 */
int mp_run(mp_state* state, int64_t K_max, double target_snr_db, int64_t* n_atoms,
           int* stop_reason, double* final_snr_db);
int mp_run_async(mp_state* state, int64_t K_max, double target_snr_db);
int mp_get_status(mp_state* state, int64_t* n_atoms, int* stop_reason, double* final_snr_db);
/* seconds of device time after which a launch returns MP_ETIMEOUT (<= 0: none) */
int mp_state_set_time_limit(mp_state* state, double seconds);

/*
 * Launch shape of the MP loop (tuning): threads per CTA (128, 256 or 512)
 * and CTAs per signal (thread-block cluster of 1, 2, 4, 8 or 16; more
 * than one needs every N_w = L/a_w divisible by it and each CTA's share of
 * the frames to fit in shared memory).  The default is chosen from the
 * number of signals and dictionaries (up to 8 signals: 16-CTA clusters,
 * 128 threads per CTA for up to three dictionaries, 512 for more; many
 * signals: one CTA each); threads = cluster = 0 restores it.  Returns
 * MP_EINVAL for a shape this state cannot run.  mp_state_get_launch reports
 * the current shape.  Results do not depend on the shape.
 */
int mp_state_set_launch(mp_state* state, int threads, int cluster);
int mp_state_get_launch(const mp_state* state, int* threads, int* cluster);

/*
 * Top level of the max tree in a one-CTA-per-signal launch (tuning; the
 * tree of Sec. 5.1 with its upper level on chip).  The CTA scans one key per
 * frame each iteration, or one per group of 2^g frames when the signal has
 * more frames than max_keys (the smallest g that fits; touched groups are
 * rebuilt from the per-frame keys after each update).  max_keys: a power of
 * two from 64 to the CTA size's cap (16384 keys for 512 threads, 8192 for
 * 256, 4096 for 128), or 0 for that cap (or the largest smaller one whose
 * top level fits in shared memory).  MP_EINVAL for other values, for a
 * launch with clusters (a cluster CTA holds its own frames ungrouped), or
 * when the top level does not fit.  mp_state_set_launch resets it to the
 * default.  mp_state_get_top_keys reports it (0 for cluster launches).
 * Results do not depend on it.
 */
int mp_state_set_top_keys(mp_state* state, int max_keys);
int mp_state_get_top_keys(const mp_state* state, int* max_keys);

/*
 * Launch order of the signals (tuning, no counterpart in the paper).  With
 * more signals than the GPU runs at once, the MP launch starts the signals
 * in order and a CTA that finishes takes the next; by default the longer
 * signal starts first.  work (host array of B non-negative numbers, e.g.
 * the atoms each signal needed in an earlier run of similar signals)
 * starts the signals with the most work first, so that the longest
 * pursuits do not end up in the last wave; NULL restores the default.
 * Results do not depend on the order.  Synchronises the plan's stream (call
 * it outside a stream capture).  MP_EINVAL for a negative or non-finite
 * entry.
 */
int mp_state_set_work_hint(mp_state* state, const double* work);

/*
 * Resets, Alg. 2 (the paper's reset options, Sec. 7): mp_run interrupts the
 * coefficient-domain pursuit of a signal before a selection when
 * reset_every > 0 selections were made since its last reset, or when
 * reset_err_db < 0 and the estimate fell below it, 10 log10(E_k / E_out) <
 * reset_err_db, E_out the energy at the last reset.  The reset synthesises
 * all atoms selected so far (eq. idgtreal), takes the signal-domain
 * residual r_out = x - x_hat, sets E_k = E_out = ||r_out||^2 (FP64) and
 * re-analyses r_out; the pursuit then continues (stop tests first).  The
 * atom list keeps growing across resets.  Both 0: no resets (default).
 * Returns MP_EINVAL for reset_every < 0 or reset_err_db > 0.
 */
int mp_state_set_resets(mp_state* state, int64_t reset_every, double reset_err_db);

/* copy the atom list of signal sig (host buffer of cap atoms); *n = count */
int mp_get_atoms(const mp_state* state, int sig, mp_atom* out_host, int64_t cap, int64_t* n);
/* energy estimates E_k after each atom (host doubles); *n = count */
int mp_get_errors(const mp_state* state, int sig, double* E_host, int64_t cap, int64_t* n);

/*
 * Synthesis (eq. idgtreal) of signal sig's atoms into y_dev (device, L
 * floats, overwritten), and the true residual SNR 10 log10(||x||^2 /
 * ||x - y||^2) in FP64 if true_snr_db is non-NULL (synchronous then).  The
 * signal is read from the library's own device copy made by mp_analyze.
 */
int mp_synthesize(const mp_state* state, int sig, float* y_dev, double* true_snr_db);

void mp_state_destroy(mp_state* state);

/*
 * Allocation-free decomposition of one signal (no counterpart in the paper:
 * it is an operational variant of mp_analyze + mp_run).
 *
 * For callers that cannot call cudaMalloc while they decompose: real-time
 * audio threads that must not block on the device allocator (cudaMalloc may
 * synchronise the device and take unbounded time), and processes held to a
 * fixed device-memory budget or whose device memory belongs to their own
 * pool allocator.  The plan is created beforehand (that call allocates);
 * this call then allocates nothing: the coefficient planes, max trees and
 * bookkeeping live in one file-scope device array of 32 MiB that every GPU
 * loading the library holds until the process exits.
 *   x_dev       device pointer to L floats (input)
 *   atoms_dev   device buffer of K_max mp_atom (output, atoms in order)
 *   errors_dev  device buffer of K_max doubles for E_k (output) or NULL
 *   n_atoms, stop_reason, final_snr_db  host outputs or NULL; if all three
 *               are NULL the call is asynchronous on the plan's stream,
 *               otherwise it synchronises the stream and fills them
 * Same method, kernels and results as mp_analyze + mp_run on one signal
 * with the FP32 analysis (no time limit, no resets).  Returns
 * MP_ENOTCOMPAT for a plan made with MP_ANALYSIS_BF16X3 (this call runs the
 * FP32 analysis only), MP_EINVAL if the current device is not the plan's,
 * and MP_EINVAL with a message if the signal needs more than the 32 MiB
 * array (about L = 2^18 with three dictionaries of 512..2048 channels fits);
 * use mp_analyze / mp_run for those.
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) -- make that first call before any stream capture.
 * All calls on a device share the array and each call rewrites every part
 * of it it uses; calls that overlap on the GPU (other streams or threads)
 * race on it and must be serialised by the caller.
 */
int mp_decompose_static(const mp_plan* plan, const float* x_dev, int64_t L, int64_t K_max,
                        double target_snr_db, mp_atom* atoms_dev, double* errors_dev,
                        int64_t* n_atoms, int* stop_reason, double* final_snr_db);

/* message of the last failure on this host thread ("" if none) */
const char* mp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MPGABOR_H */
