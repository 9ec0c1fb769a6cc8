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
// One CTA computes a 128 (rows of A) x 128 (frames) tile: warp 0 issues TMA
// loads into a 3-stage ring (128B-swizzled K-major tiles), one thread of
// warp 1 issues tcgen05.mma (M=128, N=128, K=16; three products per K step)
// into a 128-column TMEM accumulator and releases stages with
// tcgen05.commit; all four warps then read the accumulator with tcgen05.ld
// and write complex coefficients to the frame-major plane.  Every mbarrier
// wait is bounded (2 s of device time); on expiry the CTA records an error,
// waits (bounded) for its in-flight copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mp_common_dev.cuh"
#include "mp_internal.cuh"

namespace mpg {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64, STAGES = 3;
constexpr int TILE_BYTES = TBM * TBK * 2;           // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;         // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM = STAGES * STAGE_BYTES + 1024 + 256;
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

__global__ void __launch_bounds__(128, 1)
    k_analysis_tc(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                  const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                  int Kp, int a, int Mrp, int nsig, const long long* __restrict__ tprefix,
                  const int* __restrict__ brow, const DevSig* __restrict__ sigs, int dict,
                  int* __restrict__ err, int flagged) {
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    const unsigned bar0 = base + STAGES * STAGE_BYTES;  // full[s], empty[s], done
    const unsigned full0 = bar0, empty0 = bar0 + 8 * STAGES, done = bar0 + 16 * STAGES;
    volatile unsigned* tmem_slot = reinterpret_cast<volatile unsigned*>(gbase + STAGES * STAGE_BYTES + 16 * STAGES + 8);
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long gt = blockIdx.x;
    const int s = find_tile_sig(tprefix, nsig, gt);
    const DevSig& S = sigs[s];
    if (flagged && !S.reanalyze) return;  // uniform per CTA, before any barrier
    const long long N = S.N[dict];
    const int n0 = (int)((gt - tprefix[s]) * TBN);
    const int r0 = blockIdx.y * TBM;
    const int nk = Kp / TBK;
    const int row0 = brow[s] + n0;

    if (threadIdx.x == 0) {
        failed = 0;
        for (int i = 0; i < STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * i));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer --------------------------------------------------
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int st = kb % STAGES, round = kb / STAGES;
            if (kb >= STAGES && !mbar_wait(empty0 + 8 * st, (round - 1) & 1, err)) {
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
            tma_load_2d(sb, &tAh, k0, r0, fb);
            tma_load_2d(sb + TILE_BYTES, &tAl, k0, r0, fb);
            tma_load_2d(sb + 2 * TILE_BYTES, &tBh, rr, row0 + q, fb);
            tma_load_2d(sb + 3 * TILE_BYTES, &tBl, rr, row0 + q, fb);
            issued = kb + 1;
        }
        if (failed) {
            // let copies in flight land before the CTA can exit (bounded)
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, err);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----------------------------------------------------
        const unsigned idesc = idesc_bf16(TBM, TBN);
        for (int kb = 0; kb < nk; ++kb) {
            const int st = kb % STAGES, round = kb / STAGES;
            if (!mbar_wait(full0 + 8 * st, round & 1, err) || failed) {
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
                const unsigned long long bl = sw128_desc(sb + 3 * TILE_BYTES + off);
                umma_bf16(tmem, ah, bh, idesc, (kb | kk) != 0);
                umma_bf16(tmem, ah, bl, idesc, 1);
                umma_bf16(tmem, al, bh, idesc, 1);
            }
            umma_commit(empty0 + 8 * st);
        }
        umma_commit(done);
    }
    __syncwarp();

    // ---- epilogue: TMEM -> complex plane ----------------------------------
    const bool ok = mbar_wait(done, 0, err) && !failed;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = r0 + warp * 32 + lane;
        const int m = row >> 1;
        float2* plane = S.plane[dict];
#pragma unroll 1
        for (int c0 = 0; c0 < TBN; c0 += 32) {
            unsigned v[32];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
                "%26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                  "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                  "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float re = __uint_as_float(v[j]);
                const float im = __shfl_down_sync(FULL, re, 1);
                const long long n = n0 + c0 + j;
                if (!(lane & 1) && n < N && m < Mrp) plane[n * Mrp + m] = make_float2(re, im);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN));
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

int analysis_tc_smem() { return TC_SMEM; }

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

cudaError_t launch_analysis_tc(const void* tmaps /* 4 CUtensorMap */, int Arows, int Kp, int a,
                               int Mrp, int nsig, const long long* d_tile_prefix, const int* d_brow,
                               const DevSig* d_sigs, int dict, long long total_tiles, int* d_err,
                               cudaStream_t st, int flagged) {
    if (total_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_analysis_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM);
    if (e != cudaSuccess) return e;
    const CUtensorMap* m = static_cast<const CUtensorMap*>(tmaps);
    dim3 grid((unsigned)total_tiles, (unsigned)(Arows / TBM));
    k_analysis_tc<<<grid, 128, TC_SMEM, st>>>(m[0], m[1], m[2], m[3], Kp, a, Mrp, nsig,
                                              d_tile_prefix, d_brow, d_sigs, dict, d_err, flagged);
    return cudaGetLastError();
}

}  // namespace mpg
