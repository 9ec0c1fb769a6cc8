// Precision form of the analysis (Sec. 5 initialisation): the reduced DGT as
// a split-BF16 three-product GEMM on the tcgen05 tensor cores, FP32
// accumulation in tensor memory.
//
//   rho(m, n) = sum_i A(2m + {0,1}, i) B(i, n),   A = windowed cos / -sin rows,
//   B(i, n) = x((n a + i - w/2) mod L),
//   A = A_hi + A_lo, B = B_hi + B_lo (BF16 pairs), and
//   A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi   (the A_lo B_lo term is dropped).
//
// B is never materialised: the signal is written once into a padded BF16
// segment per signal (x_hi, x_lo) and read through a 2-D TMA view whose rows
// have length a.  Because a is a multiple of 64 and w/2 a multiple of a, the
// 64 K-values i = q a + r (r in [r0, r0 + 64)) of one K block lie in one row
// offset q, so the B tile of frames n0 .. n0+127 is the plain box
// rows n0 + q .. n0 + q + 127, columns r0 .. r0 + 63 of that view.
//
// The output is cut into 128 (rows of A) x BN (frames) tiles, BN = 128 or
// 256, taken by a persistent grid of one CTA per SM: a TMA producer thread
// streams the K blocks of the CTA's tiles through a ring of 3 (BN = 128) or
// 2 (BN = 256) stages of 128B-swizzled K-major tiles, an MMA thread issues
// tcgen05.mma (M=128, N=BN, K=16; three products per K step) into one of two
// BN-column TMEM accumulators and releases stages with tcgen05.commit, and
// four epilogue warps read the other accumulator with tcgen05.ld and write
// complex coefficients to the frame-major plane.  A 256-frame tile loads
// 96 KB of operands per K block for twice the products of a 128-frame tile
// (64 KB), so the operand traffic per flop falls by a quarter; the host takes
// it when there are many tiles (batches), where the loads set the pace.  Every mbarrier wait is bounded (2 s of device time); on
// expiry the CTA records an error, waits (bounded) for its in-flight copies
// and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int TBM = 128, TBK = 64;
constexpr int TILE_BYTES = TBM * TBK * 2;  // 16 KB: one A operand tile (128 rows)
constexpr int STG_BYTES = 32 * TBM * 4;    // epilogue staging: 32 frames x 128 rows of FP32

// shared-memory layout of the BN-frame form: the ring (A_hi, A_lo, B_hi,
// B_lo per stage), 128 bytes of barriers, the epilogue staging, and 1024
// bytes for the alignment of the ring
template <int BN>
struct TcCfg {
    static constexpr int STAGES = BN == 256 ? 2 : 3;
    static constexpr int B_BYTES = BN * TBK * 2;
    static constexpr int STAGE_BYTES = 2 * TILE_BYTES + 2 * B_BYTES;
    static constexpr int STG_OFF = STAGES * STAGE_BYTES + 128;
    static constexpr int SMEM = STG_OFF + STG_BYTES + 1024;
    static constexpr int ACC_COLS = 2 * BN;  // two accumulators
};
static_assert(TcCfg<256>::SMEM <= 227 * 1024, "256-frame ring exceeds shared memory");
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false (and the error flag) when the time limit expires
__device__ bool mbar_wait(unsigned addr, unsigned parity, int* err) {
    const unsigned long long t0 = gtime();
    while (!mbar_try(addr, parity)) {
        if (gtime() - t0 > WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// 64-bit shared-memory matrix descriptor: K-major tile, 128-byte swizzle,
// 8-row core groups 1024 bytes apart
__device__ __forceinline__ unsigned long long sw128_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)(16u >> 4) << 16;
    d |= (unsigned long long)(1024u >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, K-major A and B
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int c0, int c1,
                                            unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        :
        : "r"(dst), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void umma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                          unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ int find_tile_sig(const long long* prefix, int nsig, long long t) {
    int lo = 0, hi = nsig - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent form: gridDim.x CTAs (one per SM) take the 128 x BN output
// tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (row tiles of one frame
// tile consecutive, so neighbouring CTAs share the frame operand in L2).
// Warp 4 lane 0 streams the K blocks of all its tiles through the TMA ring;
// warp 5 lane 0 issues the MMAs of tile i into TMEM accumulator i mod 2
// (2 x BN columns) once the epilogue has drained it, and commits it;
// warps 0-3 (TMEM lanes 0-127) read accumulator i mod 2 and write the plane
// while the MMAs of tile i + 1 run.  Per tile the MMAs run in the same order
// as one CTA per tile would, so the planes are bitwise the same.
constexpr int TC_THREADS = 192;

struct TileOf {
    int s;       // signal
    int n0, r0;  // first frame, first row of A
    bool skip;   // reset pass: signal not flagged
};

template <int BN>
__device__ __forceinline__ TileOf tile_of(long long t, int nrow, const long long* tprefix, int nsig,
                                          const DevSig* sigs, int flagged) {
    TileOf o;
    const long long ft = t / nrow;
    o.r0 = (int)(t - ft * nrow) * TBM;
    o.s = find_tile_sig(tprefix, nsig, ft);
    o.n0 = (int)((ft - tprefix[o.s]) * BN);
    o.skip = flagged && !sigs[o.s].reanalyze;
    return o;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_analysis_tc(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                  const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                  int Kp, int a, int Mrp, int nsig, const long long* __restrict__ tprefix,
                  const int* __restrict__ brow, const DevSig* __restrict__ sigs, int dict,
                  long long ntiles, int nrow, int* __restrict__ err, int flagged) {
    using Cfg = TcCfg<BN>;
    constexpr int STAGES = Cfg::STAGES, STAGE_BYTES = Cfg::STAGE_BYTES, ACC_COLS = Cfg::ACC_COLS;
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    // barriers: full[s], empty[s], tfull[2], tempty[2], drained
    const unsigned bar0 = base + STAGES * STAGE_BYTES;
    const unsigned full0 = bar0, empty0 = bar0 + 8 * STAGES;
    const unsigned tfull0 = bar0 + 16 * STAGES, tempty0 = tfull0 + 16, drained = tempty0 + 16;
    volatile unsigned* tmem_slot =
        reinterpret_cast<volatile unsigned*>(gbase + STAGES * STAGE_BYTES + 16 * STAGES + 40);
    __shared__ volatile int failed;
    __shared__ volatile int tile_ok;  // epilogue: the accumulator of this tile is ready
    float* stg = reinterpret_cast<float*>(gbase + Cfg::STG_OFF);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = Kp / TBK;

    if (threadIdx.x == 0) {
        failed = 0;
        for (int i = 0; i < STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * i));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tempty0 + 8 * i));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(drained));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(ACC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 4) {
        // ---- TMA producer ------------------------------------------------
        if (lane == 0) {
            long long kc = 0;  // K blocks issued by this CTA
            for (long long t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
                const TileOf T = tile_of<BN>(t, nrow, tprefix, nsig, sigs, flagged);
                if (T.skip) continue;
                const int row0 = brow[T.s] + T.n0;
                for (int kb = 0; kb < nk; ++kb, ++kc) {
                    const int st = (int)(kc % STAGES);
                    const unsigned rnd = (unsigned)(kc / STAGES);
                    if (kc >= STAGES && !mbar_wait(empty0 + 8 * st, (rnd - 1) & 1, err)) {
                        failed = 1;
                        break;
                    }
                    const unsigned fb = full0 + 8 * st;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"(STAGE_BYTES)
                                 : "memory");
                    const unsigned sb = base + st * STAGE_BYTES;
                    const int k0 = kb * TBK;
                    const int q = k0 / a, rr = k0 - q * a;
                    tma_load_2d(sb, &tAh, k0, T.r0, fb);
                    tma_load_2d(sb + TILE_BYTES, &tAl, k0, T.r0, fb);
                    tma_load_2d(sb + 2 * TILE_BYTES, &tBh, rr, row0 + q, fb);
                    tma_load_2d(sb + 2 * TILE_BYTES + Cfg::B_BYTES, &tBl, rr, row0 + q, fb);
                }
            }
            if (failed) {
                // let the copies in flight land before the CTA can exit (bounded)
                const long long k0 = kc > STAGES ? kc - STAGES : 0;
                for (long long k = k0; k < kc; ++k)
                    mbar_wait(full0 + 8 * (int)(k % STAGES), (unsigned)(k / STAGES) & 1, err);
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer ----------------------------------------------------
        if (lane == 0) {
            const unsigned idesc = idesc_bf16(TBM, BN);
            long long kc = 0, tc = 0;
            for (long long t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
                const TileOf T = tile_of<BN>(t, nrow, tprefix, nsig, sigs, flagged);
                if (T.skip) continue;
                const int b = (int)(tc & 1);
                const unsigned use = (unsigned)(tc >> 1);
                if (use >= 1 && !mbar_wait(tempty0 + 8 * b, (use - 1) & 1, err)) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned acc = tmem + (unsigned)(b * BN);
                for (int kb = 0; kb < nk; ++kb, ++kc) {
                    const int st = (int)(kc % STAGES);
                    const unsigned rnd = (unsigned)(kc / STAGES);
                    if (!mbar_wait(full0 + 8 * st, rnd & 1, err)) {
                        failed = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned sb = base + st * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TBK / 16; ++kk) {
                        const unsigned off = kk * 32;
                        const unsigned long long ah = sw128_desc(sb + off);
                        const unsigned long long al = sw128_desc(sb + TILE_BYTES + off);
                        const unsigned long long bh = sw128_desc(sb + 2 * TILE_BYTES + off);
                        const unsigned long long bl =
                            sw128_desc(sb + 2 * TILE_BYTES + Cfg::B_BYTES + off);
                        umma_bf16(acc, ah, bh, idesc, (kb | kk) != 0);
                        umma_bf16(acc, ah, bl, idesc, 1);
                        umma_bf16(acc, al, bh, idesc, 1);
                    }
                    umma_commit(empty0 + 8 * st);
                }
                if (failed) break;
                umma_commit(tfull0 + 8 * b);
                ++tc;
            }
            // every MMA this thread issued has completed before the CTA ends
            umma_commit(drained);
            mbar_wait(drained, 0, err);
        }
    } else {
        // ---- epilogue: warps 0-3, TMEM lanes 32 w .. 32 w + 31 -------------
        // Thread 0 waits for the accumulator and shares the outcome behind a
        // named barrier of the four warps, so they leave together on failure.
        // Each 32-frame chunk is transposed through shared memory and written
        // as 16-byte stores, one frame's 64 bins (512 B) per row of threads.
        const int rl = warp * 32 + lane;
        long long tc = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileOf T = tile_of<BN>(t, nrow, tprefix, nsig, sigs, flagged);
            if (T.skip) continue;
            const int b = (int)(tc & 1);
            const unsigned use = (unsigned)(tc >> 1);
            if (threadIdx.x == 0)
                tile_ok = (mbar_wait(tfull0 + 8 * b, use & 1, err) && !failed) ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (!tile_ok) {
                if (threadIdx.x == 0) failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const DevSig& S = sigs[T.s];
            const long long N = S.N[dict];
            float2* plane = S.plane[dict];
            const int mb = T.r0 >> 1;  // first bin of the tile
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                unsigned v[32];
                const unsigned taddr =
                    tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(b * BN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                    "%9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, "
                    "%24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                      "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                      "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[j * TBM + rl] = __uint_as_float(v[j]);
                asm volatile("bar.sync 1, 128;" ::: "memory");
                // 32 frames x 32 float4 (two bins each): 8 per thread
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int q = threadIdx.x + 128 * i;
                    const int j = q >> 5, p = q & 31;
                    const long long n = T.n0 + c0 + j;
                    const int m0 = mb + 2 * p;
                    if (n < N && m0 < Mrp)
                        *reinterpret_cast<float4*>(plane + n * Mrp + m0) =
                            *reinterpret_cast<const float4*>(stg + j * TBM + 4 * p);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
            }
            // accumulator b may be overwritten now
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * b)
                             : "memory");
            ++tc;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ACC_COLS));
}

// hi = bf16(v), lo = bf16(v - hi), rows of length cols padded with zeros to
// cols_p
__global__ void k_split_rows(const float* __restrict__ src, int rows, int cols, int src_ld,
                             int cols_p, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * cols_p) return;
    const int r = (int)(idx / cols_p), c = (int)(idx % cols_p);
    const float v = c < cols ? src[(long long)r * src_ld + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// padded signal segment: seg[j] = x((j - pad) mod L) for j < seg_len
__global__ void k_split_segment(const DevSig* __restrict__ sigs, const long long* __restrict__ seg_off,
                                const long long* __restrict__ seg_len, int pad,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                int flagged) {
    const DevSig& S = sigs[blockIdx.y];
    if (flagged && !S.reanalyze) return;
    const float* xin = S.use_r ? S.r : S.x;
    const long long off = seg_off[blockIdx.y], len = seg_len[blockIdx.y];
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < len;
         j += (long long)gridDim.x * blockDim.x) {
        const float v = xin[lmod(j - pad, S.L)];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[off + j] = h;
        lo[off + j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

}  // namespace

cudaError_t launch_split_rows(const float* src, int rows, int cols, int src_ld, int cols_p,
                              void* hi, void* lo, cudaStream_t st) {
    const long long n = (long long)rows * cols_p;
    k_split_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        src, rows, cols, src_ld, cols_p, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t launch_split_segments(const DevSig* d_sigs, int nsig, const long long* seg_off,
                                  const long long* seg_len, int pad, void* hi, void* lo,
                                  cudaStream_t st, int flagged) {
    dim3 grid(256, (unsigned)nsig);
    k_split_segment<<<grid, 256, 0, st>>>(d_sigs, seg_off, seg_len, pad, (__nv_bfloat16*)hi,
                                          (__nv_bfloat16*)lo, flagged);
    return cudaGetLastError();
}

int analysis_tc_frames(long long nrow, long long tiles256, long long frames128,
                       long long frames256, int num_sms) {
    // 256-frame tiles when every SM gets at least four of them and the wider
    // tiles pad the frames by at most a quarter more than 128-frame tiles do
    // (on GB300 the 256-frame form was faster on a batch of 256 signals even
    // at 14 % more padded frames: the operand loads, not the MMAs, set the
    // pace there)
    return nrow * tiles256 >= 4ll * num_sms && 4 * frames256 <= 5 * frames128 ? 256 : 128;
}

cudaError_t launch_analysis_tc(const void* tmaps /* 4 CUtensorMap */, int bn, int Arows, int Kp,
                               int a, int Mrp, int nsig, const long long* d_tile_prefix,
                               const int* d_brow, const DevSig* d_sigs, int dict,
                               long long total_tiles, int* d_err, cudaStream_t st, int flagged) {
    if (total_tiles <= 0) return cudaSuccess;
    if (bn != 128 && bn != 256) return cudaErrorInvalidValue;
    auto kf = bn == 256 ? k_analysis_tc<256> : k_analysis_tc<128>;
    const int smem = bn == 256 ? TcCfg<256>::SMEM : TcCfg<128>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap* m = static_cast<const CUtensorMap*>(tmaps);
    // one CTA per SM (the shared memory allows no second one, so the CTA
    // holds the SM's tensor memory alone), each looping over the tiles
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nrow = Arows / TBM;
    const long long ntiles = total_tiles * nrow;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
    kf<<<grid, TC_THREADS, smem, st>>>(m[0], m[1], m[2], m[3], Kp, a, Mrp, nsig, d_tile_prefix,
                                       d_brow, d_sigs, dict, ntiles, nrow, d_err, flagged);
    return cudaGetLastError();
}

}  // namespace mpg
