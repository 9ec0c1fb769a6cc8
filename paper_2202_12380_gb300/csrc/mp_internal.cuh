// Internal data layout shared by the CUDA translation units of libmpgabor.
//
// Device memory layout (per signal, per dictionary w):
//   plane[w]  residual coefficients rho_w(m, n), float2, frame-major
//             [N_w][Mrp_w] with Mrp_w = 32 * ceil((M_w/2 + 1) / 32); bins
//             m >= M_w/2 + 1 are zero padding and never selected
//   l0[w]     max-tree level 0: one key per (frame, 32-bin chunk)
//   l1[w]     max-tree level 1: one key per frame
// The MP launch keeps the top level (one key per frame, or per group of
// 2^gshift consecutive frames of one dictionary when the frames do not fit)
// in shared memory.  A key packs the selection score and the coefficient's
// flat index:
//   key = (float bits of |rho|^2) << 32 | (0xffffffff - flat index),
//   flat = fbase[w] + n * 2^msh_w + m   (2^msh_w >= M_w/2 + 1),
// so an unsigned max over keys is the argmax of |rho|^2 with ties broken
// towards the lowest (w, n, m).  |rho|^2 >= 0, so its float bits order like
// the values.  The tree holds keys only: the selected coefficient itself is
// read from its plane.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "mpgabor.h"

namespace mpg {

constexpr int MAXW = 8;          // dictionaries per plan
constexpr int CHUNK = 32;        // bins per level-0 entry (one warp)
constexpr int TOPCAP = 16384;    // top-level keys held in shared memory per single CTA
constexpr int TOPCAP_CLUSTER = 24576;  // own frames a cluster CTA may hold (if they fit)

using Key = unsigned long long;

struct DevDict {
    int wlen, a, M, Mr, nch, Mrp;  // Mr = M/2+1 stored bins, Mrp padded to CHUNK
    int gam_lo, gam_hi, gam_off;   // compact <d, conj d> table (see mp_plan.cu)
    int g_off;                     // offset of the FP32 window in DevPlan::g32
    int msh;                       // flat-index row stride 2^msh >= Mr
    int Mmask;                     // M - 1 if M is a power of two, else 0
    int cis_off;                   // offset of the modulation table in DevPlan::cis
    int cis_q;                     // M/4 if 4 divides M (the table holds e^{i 2 pi q / M},
                                   // q < M/4; quadrants are exact multiples by i), else 0
                                   // (the table holds all q < M)
    int cis_qsh;                   // log2(M/4) if M/4 is a power of two, else -1
};

struct DevPair {
    int rf, rt;      // alignment classes in frequency / time
    int cls_base;    // first class descriptor of the pair
    int rf_sh, rt_sh;  // log2(rf), log2(rt), or -1 if not a power of two
    int mratio;      // M_v / M_u when M_v >= M_u, else 0
    int aratio;      // a_u / a_v when a_v <= a_u, else 0
    int pad;
};

// Dense tile of one alignment class: T[c * R + i] = h_eps(delta, tau) with
// delta = (i_lo + i) rf - cf and tau = (c_lo + c) a_v - ct a_u.
struct DevClass {
    long long off;   // float2 offset in the tile pool
    int R, C, i_lo, c_lo;
};

struct DevPlan {
    int W;
    int ncls;  // class descriptors
    int ngam;  // entries of the compact <d, conj d> pool
    int ncis;  // entries of the modulation tables
    int pedantic;  // selection by the pair energy drop (MP_PEDANTIC)
    int pow2;      // every M_w and a_w is a power of two
    DevDict d[MAXW];
    DevPair p[MAXW * MAXW];
    const DevClass* cls;
    const float2* tiles;
    const float2* gam;
    const float* g32;
    const float2* cis;  // e^{i 2 pi q / M_w} per dictionary (FP64-rounded to FP32)
    long long tiles_len;  // entries of the tile pool (bounds-checking build)
    // MP_COEF_FP64: the same tables in FP64 (tile offsets as in `tiles`)
    int fp64;
    const double2* tiles64;
    const double2* gam64;
    const double2* cis64;
};

// Coefficient planes hold float2 entries, or double2 ones when the plan has
// MP_COEF_FP64 (DevPlan::fp64); `plane` is then reinterpreted as double2*.
struct DevSig {
    long long L;
    long long N[MAXW];
    int Nmask[MAXW];  // N_w - 1 if N_w is a power of two, else 0
    unsigned fbase[MAXW + 1];
    float2* plane[MAXW];
    Key* l0[MAXW];
    Key* l1[MAXW];
    mp_atom* atoms;
    double* errs;
    long long cap;
    const float* x;  // device copy of the signal
    // dynamic state, written back by the MP launch
    long long k;
    double E;
    double E0;
    int stop;
    int timed_out;
    // resets (Alg. 2): residual and synthesis buffers, the last reset's
    // atom count and energy, and the hand-over flags between launches
    float* r;
    float* y;
    long long k_out;
    double E_out;
    int reset_pending;  // the MP launch stopped for a reset
    int reanalyze;      // analysis kernels act on this signal (reset pass)
    int use_r;          // the analysis reads r instead of x
    int bounds;         // bounds-checking build (MP_CHECK_BOUNDS): first failed
                        // access site of the MP loop, 0 if none (always 0 otherwise)
};

// ---- host launchers implemented in the .cu files -------------------------
// analysis: rho = A * frames for dictionary w of the listed signals
// flagged: act only on signals whose `reanalyze` flag is set (reset pass)
cudaError_t launch_analysis_sgemm(const float* A, int Arows, int Kp, int w_len, int a, int Mrp,
                                  int nsig, const long long* d_tile_prefix, const DevSig* d_sigs,
                                  int dict, long long total_frame_tiles, cudaStream_t st,
                                  int flagged = 0);
// FP64 analysis (MP_COEF_FP64): the same DFT-GEMM with FP64 matrix and
// accumulation into double2 planes
cudaError_t launch_analysis_dgemm(const double* A, int Arows, int Kp, int w_len, int a, int Mrp,
                                  int nsig, const long long* d_tile_prefix, const DevSig* d_sigs,
                                  int dict, long long total_frame_tiles, cudaStream_t st,
                                  int flagged = 0);
// device-to-device copy of up to GATHER_MAX signals in one launch (the
// pointers and lengths travel as kernel parameters, so the launch can be
// captured in a CUDA graph)
constexpr int GATHER_MAX = 256;
struct GatherArgs {
    const float* src[GATHER_MAX];
    float* dst[GATHER_MAX];
    long long len[GATHER_MAX];
};
cudaError_t launch_gather_signals(const GatherArgs& g, int n, cudaStream_t st);
// E_0 = E = ||x||^2 (FP64) of every signal and a fresh pursuit state.
// d_part: scratch of nsig * ENERGY_PARTS doubles (partial sums).
constexpr int ENERGY_PARTS = 64;
cudaError_t launch_energy(DevSig* d_sigs, int nsig, double* d_part, cudaStream_t st);
// reset pass: r = x - y for flagged signals, then E = E_out = ||r||^2
// (d_part as for launch_energy)
cudaError_t launch_reset_residual(DevSig* d_sigs, int nsig, double* d_part, cudaStream_t st);
cudaError_t launch_tree_build(const DevPlan& P, const DevSig* d_sigs, int nsig,
                              const long long* d_frame_prefix, long long total_frames, int dict,
                              cudaStream_t st, int flagged = 0);
// launch shape of the MP loop: threads per CTA, CTAs per signal (cluster),
// top-level keys a single CTA may hold (the loop groups frames to fit), and
// the dynamic shared memory; threads = 0 means no shape fits
struct LoopShape {
    int threads = 0;
    int cs = 1;
    int topcap = 0;
    size_t smem = 0;
};
// reset_it > 0: reset after that many selections since the last reset;
// reset_scale > 0: reset once E < E_out reset_scale
cudaError_t launch_mp_loop(const DevPlan& P, DevSig* d_sigs, const int* d_order, int nsig,
                           long long kmax, double thr_scale, long long budget_ns,
                           const LoopShape& shape, cudaStream_t st, long long reset_it = 0,
                           double reset_scale = 0.0);
void mp_loop_shape(const DevPlan& P, const DevSig* hs, int B, int num_sms, LoopShape* out);
bool mp_loop_shape_ok(const DevPlan& P, const DevSig* hs, int B, int threads, int c,
                      LoopShape* out);
// one CTA per signal with a top level of at most cap keys (a power of two
// in 64 .. the CTA size's default cap); false if it does not fit
bool mp_loop_shape_single_cap(const DevPlan& P, const DevSig* hs, int B, int threads, int cap,
                              LoopShape* out);
cudaError_t launch_synth(const DevPlan& P, const DevSig* d_sig, long long natoms, float* y,
                         long long L, cudaStream_t st);
cudaError_t launch_resid_energy(const DevSig* d_sig, const float* y, long long L,
                                double* d_partials, int nparts, cudaStream_t st);

// tensor-core (split-BF16) analysis, mp_analysis_tc.cu.  Tiles are 128 rows
// of A by bn = 128 or 256 frames; analysis_tc_frames picks bn from the row
// tiles, the tile count with 256 frames and the frames both widths cover.
int analysis_tc_frames(long long nrow, long long tiles256, long long frames128,
                       long long frames256, int num_sms);
cudaError_t launch_split_rows(const float* src, int rows, int cols, int src_ld, int cols_p,
                              void* hi, void* lo, cudaStream_t st);
cudaError_t launch_split_segments(const DevSig* d_sigs, int nsig, const long long* seg_off,
                                  const long long* seg_len, int pad, void* hi, void* lo,
                                  cudaStream_t st, int flagged = 0);
cudaError_t launch_analysis_tc(const void* tmaps, int bn, int Arows, int Kp, int a, int Mrp,
                               int nsig, const long long* d_tile_prefix, const int* d_brow,
                               const DevSig* d_sigs, int dict, long long total_tiles, int* d_err,
                               cudaStream_t st, int flagged = 0);
// encodes a 2-D BF16 tensor map with a 64 x box_rows box and 128-byte
// swizzle (mp_plan.cu); returns false on failure
bool encode_bf16_map(void* map, const void* base, unsigned long long inner,
                     unsigned long long outer, unsigned long long row_bytes,
                     unsigned box_rows = 128);

size_t mp_loop_smem_bytes(const DevPlan& P, int T, int threads, int cs);
int mp_loop_threads(int nsig, int num_sms);
int mp_loop_max_clusters(int threads, int cs, size_t smem, bool fp64 = false);

}  // namespace mpg

namespace mpg {
// NVTX range over one C-ABI call (visible in nsys / ncu timelines; NVTX v3
// is header-only and costs nothing when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace mpg

// error helpers (mp_api.cu)
extern "C" void mpg_set_error(const char* fmt, ...);

#ifdef __cplusplus
#include <vector>

// host side of an mp_plan (opaque in the C ABI)
struct mp_plan {
    int W;
    int wlen[mpg::MAXW], a[mpg::MAXW], M[mpg::MAXW];
    double eps;
    unsigned flags;
    cudaStream_t stream;
    int device;
    int num_sms;
    mpg::DevPlan dp;  // device view (pointers below)
    // geometry of every ordered pair (u, v), index u * W + v
    int Mx[mpg::MAXW * mpg::MAXW], an[mpg::MAXW * mpg::MAXW];
    int tmin[mpg::MAXW * mpg::MAXW], ntau[mpg::MAXW * mpg::MAXW];
    double2* d_kern[mpg::MAXW * mpg::MAXW];  // untruncated FP64 kernels [ntau][Mx]
    std::vector<mpg::DevClass> cls;
    std::vector<int> cls_nnz;
    std::vector<float> gam_full[mpg::MAXW];  // <d, conj d>, (M/2+1) complex
    mpg::DevClass* d_cls;
    float2* d_tiles;
    long long tiles_len;
    float2* d_gam;
    float* d_g32;
    float2* d_cis32;
    float* d_A[mpg::MAXW];  // FP32 DFT matrices for the analysis, [Arows][Akp]
    double* d_A64[mpg::MAXW];  // FP64 DFT matrices (MP_COEF_FP64), same shape
    double2* d_tiles64;        // FP64 class tiles (MP_COEF_FP64)
    double2* d_gam64;          // FP64 compact <d, conj d> (MP_COEF_FP64)
    double2* d_cis64;          // FP64 modulation tables (MP_COEF_FP64)
    int Arows[mpg::MAXW], Akp[mpg::MAXW];
    // split-BF16 analysis (MP_ANALYSIS_BF16X3): A = A_hi + A_lo, [Arows][Kp64]
    void* d_Ahi[mpg::MAXW];
    void* d_Alo[mpg::MAXW];
    int Kp64[mpg::MAXW];
    alignas(64) unsigned char tmA[mpg::MAXW][2][128];  // CUtensorMap of A_hi, A_lo
};
#endif
