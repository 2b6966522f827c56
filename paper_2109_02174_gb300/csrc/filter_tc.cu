// Ramp filter Q = P * H (the convolution stated after Eq. 2) as a dense
// Toeplitz contraction on the 5th-generation tensor cores:
//     Q[i][n] = sum_k P[i][k] T[n][k],   T[n][k] = tau h(n - k),
// an (A x D) . (D x D)^T GEMM.  FP32 accuracy from TF32 units by the 3xTF32
// split: x = x_hi + x_lo with x_hi = tf32(x) (round to nearest) and
// x_lo = x - x_hi, and P T ~= P_hi T_hi + P_hi T_lo + P_lo T_hi, each product
// accumulated in FP32 in tensor memory.  T_hi and T_lo are plan tables.
//
// One CTA per 128 x 128 output tile (rows m0.., output bins n0 = 126 t - 1 ..)
// of one slice; one launch covers every slice that shares the plan:
//   warp 0 (lane 0) issues tcgen05.mma, K-chunk after K-chunk (32 columns);
//   warp 1 (lane 0) brings T_hi/T_lo tiles in with 2D TMA (128-byte swizzle);
//   warps 2..9 load the sinogram rows with coalesced loads (the next chunk's
//   values are in flight while the current ones are stored), split them into
//   tf32 hi/lo and store both in the same swizzled layout, then run the
//   epilogue: tcgen05.ld of the accumulators, (mid, slope) pairs of
//   consecutive bins, stores to the filtered rows.
// Tiles step by 126 output pairs and overlap by two columns so every pair's
// two bins sit in one tile; the row n0 = -1 of the first tile is out of bounds
// for TMA and arrives as zeros, which is Q[-1] = 0.  A NSTAGE-deep mbarrier
// ring (full: data landed, empty: MMAs done reading) keeps loads and MMAs
// overlapped.  The tensor core's FP32 accumulation loses low bits at every
// accumulate step, and a ramp-filtered sinogram row is 50-250 times smaller
// than the sums it comes from, so partial sums never stay in tensor memory for
// long: every 32-wide K-chunk gets a fresh accumulator (a ring of four TMEM
// blocks, all 512 columns) that the epilogue warps add into FP32 registers
// (correctly rounded) as soon as its MMAs complete, then hand back to the MMA
// warp.  The lo parts are rounded to tf32 (to nearest) before they reach the
// tensor core, so its truncation of them leaves no sign-correlated error.
// Every wait is bounded (the run-time limit of WaitHook); on a timeout the CTA
// records the status and every warp stops: the MMA warp then waits (bounded)
// for the MMAs it committed, the TMA warp for the loads it issued, and the
// CTA releases its tensor memory and exits with nothing in flight.  For
// tests, the first CTA can withhold the loader warps' arrival on one stage,
// which makes the MMA warp's wait on it run out.
#include "fbp_internal.h"
#include "filter_tc.cuh"
#include "lambert.cuh"
#include "ptx.cuh"
#include "waithook.cuh"

#include <cstring>

namespace fbp {
namespace {

constexpr int kBM = 128;      // output rows per tile (TMEM lanes)
constexpr int kBN = 128;      // output bins per tile (TMEM columns)
constexpr int kStep = 126;    // output pairs per tile
constexpr int kBK = 32;       // fp32 elements per 128-byte swizzle row
constexpr int kStages = 3;
constexpr int kAcc = 4;       // accumulator slots (TMEM column blocks), ring
constexpr int kTile = kBM * kBK * 4;          // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTile;        // A_hi, A_lo, B_hi, B_lo
constexpr int kLoadWarps = 8;  // warps 2..9: sinogram split, then epilogue
constexpr int kThreads = 32 * (2 + kLoadWarps);
constexpr int kRowsPerLoader = kBM / kLoadWarps;  // 16

__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// 8-row x 128-byte atoms stacked 1024 bytes apart along M/N.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 1024 B
    d |= (uint64_t)1 << 46;                            // descriptor version (sm_100)
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major,
// M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 1 accumulator column of this thread's lane.
__device__ __forceinline__ float tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

// Columns an epilogue warp accumulates: half 0 takes columns 0..63 plus
// column 64 (pairs 0..63), half 1 columns 64..127 (pairs 64..125).  Column j
// holds Q[n0 + j]; pair p0 + j takes columns j and j + 1.
template <int H>
__device__ __forceinline__ void add_block(uint32_t tmem_block, int quarter, float (&sum)[2][32],
                                          float &extra)
{
    constexpr int C0 = H ? 2 : 0;
    const uint32_t lane_base = tmem_block + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float w[16];
            tmem_ld16(lane_base + (uint32_t)((C0 + cc) * 32 + 16 * h), w);
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[cc][16 * h + j] += w[j];
        }
    }
    if (H == 0) extra += tmem_ld1(lane_base + 64u);
}

template <int H>
__device__ __forceinline__ void store_half(const float (&v)[2][32], float extra, float *row, int p0,
                                           int npairs)
{
    constexpr int C0 = H ? 2 : 0;
    constexpr int J0 = H ? 64 : 0;
    constexpr int J1 = H ? kStep : 64;
#pragma unroll
    for (int j = J0; j < J1; j += 2) {
        if (p0 + j < npairs) {
            const int l = j - C0 * 32;
            const float a0 = v[l / 32][l % 32];
            const float a1 = v[(l + 1) / 32][(l + 1) % 32];
            const float a2 = (l + 2 < 64) ? v[(l + 2) / 32][(l + 2) % 32] : extra;
            *reinterpret_cast<float4 *>(row + 2 * (p0 + j)) =
                make_float4((a0 + a1) * 0.5f, a1 - a0, (a1 + a2) * 0.5f, a2 - a1);
        }
    }
}

struct TcArgs {
    const float *sino[kTcMaxSlices];
    float *q[kTcMaxSlices];  // filtered pairs [A][pitch]
    int ld[kTcMaxSlices];
    int A;
    int D;
    int pitch;
    int nk;       // K chunks
    int m_tiles;  // row tiles per slice
    float i0;     // > 0: intensity input, converted on load
    float ln_i0;
    int *status;
};

// INTENSITY: the sinogram holds intensities (plan option i0), converted when
// the loaders split them; a separate instantiation, since the kernel sits at
// its register limit and the plain path should not pay for the conversion.
template <bool INTENSITY>
__global__ void __launch_bounds__(kThreads, 1)
    filter_tc_kernel(const __grid_constant__ CUtensorMap t_hi, const __grid_constant__ CUtensorMap t_lo,
                     const TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t s0 = smem_addr(smem);
    const uint32_t base = (s0 + 1023u) & ~1023u;  // 1024-byte aligned: swizzle atoms
    unsigned char *bp = smem + (base - s0);
    const uint32_t bar_full_a = base + kStages * kStageBytes;      // [kStages], 128 arrivals
    const uint32_t bar_full_b = bar_full_a + 8 * kStages;          // [kStages], TMA bytes
    const uint32_t bar_empty = bar_full_b + 8 * kStages;           // [kStages], MMA commit
    const uint32_t bar_acc_full = bar_empty + 8 * kStages;         // [kAcc], MMA commit
    const uint32_t bar_acc_free = bar_acc_full + 8 * kAcc;         // [kAcc], epilogue warps
    uint32_t *tmem_slot =
        reinterpret_cast<uint32_t *>(bp + kStages * kStageBytes + 8 * (3 * kStages + 2 * kAcc));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int n_tile = blockIdx.x;
    const int sl = blockIdx.y / args.m_tiles;
    const int m0 = (blockIdx.y - sl * args.m_tiles) * kBM;
    const float *sino = args.sino[sl];
    const int ld = args.ld[sl];
    const int n0 = n_tile * kStep - 1;  // first output bin of the tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full_a + 8 * s, 32 * kLoadWarps);
            mbar_init(bar_full_b + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int a = 0; a < kAcc; ++a) {
            mbar_init(bar_acc_full + 8 * a, 1);
            mbar_init(bar_acc_free + 8 * a, kLoadWarps);
        }
        *abort_flag = 0;
        fence_proxy_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kAcc * kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        *reinterpret_cast<volatile int *>(args.status) = FBP_ERR_TIMEOUT;
        *abort_flag = 1;
    };
    const WaitHook hook = g_wait_hook;
    const unsigned long long lim = wait_limit_ns(hook);

    if (warp == 0) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int committed = -1;  // last K chunk whose MMAs were committed
            for (int kc = 0; kc < args.nk && !*abort_flag; ++kc) {
                const int s = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait_bounded(bar_full_a + 8 * s, ph, lim) ||
                    !mbar_wait_bounded(bar_full_b + 8 * s, ph, lim)) {
                    fail();
                    break;
                }
                const int blk = kc % kAcc;
                if (kc >= kAcc &&
                    !mbar_wait_bounded(bar_acc_free + 8 * blk, (uint32_t)(kc / kAcc - 1) & 1u,
                                       lim)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t st = base + s * kStageBytes;
                const uint32_t a_hi = st, a_lo = st + kTile, b_hi = st + 2 * kTile,
                               b_lo = st + 3 * kTile;
                const uint32_t d = tmem + (uint32_t)(blk * kBN);
#pragma unroll
                for (int kk = 0; kk < kBK / 8; ++kk) {  // K = 8 tf32 = 32 bytes per MMA
                    const uint32_t off = 32u * kk;
                    mma_tf32(d, sw128_desc(a_hi + off), sw128_desc(b_lo + off), kk > 0 ? 1u : 0u);
                    mma_tf32(d, sw128_desc(a_lo + off), sw128_desc(b_hi + off), 1u);
                    mma_tf32(d, sw128_desc(a_hi + off), sw128_desc(b_hi + off), 1u);
                }
                mma_commit(bar_empty + 8 * s);     // stage s free once these MMAs have read it
                mma_commit(bar_acc_full + 8 * blk);  // chunk kc's partial sums are ready
                committed = kc;
            }
            // stopped early: the MMAs already issued finish before the tensor
            // memory they write is released (a commit tracks all earlier ones)
            if (*abort_flag && committed >= 0)
                (void)mbar_wait_bounded(bar_empty + 8 * (committed % kStages),
                                        (uint32_t)(committed / kStages) & 1u, lim);
        }
        __syncwarp();
    } else if (warp == 1) {
        // -------------------------------------------------------- T tiles by TMA
        if (lane == 0) {
            int issued = 0;  // K chunks whose T tiles were requested
            for (int kc = 0; kc < args.nk && !*abort_flag; ++kc) {
                const int s = kc % kStages;
                const uint32_t use = (uint32_t)(kc / kStages);
                if (use > 0 && !mbar_wait_bounded(bar_empty + 8 * s, (use - 1) & 1u, lim)) {
                    fail();
                    break;
                }
                const uint32_t st = base + s * kStageBytes;
                mbar_arrive_expect_tx(bar_full_b + 8 * s, 2 * kTile);
                tma_load_2d(st + 2 * kTile, &t_hi, kc * kBK, n0, bar_full_b + 8 * s);
                tma_load_2d(st + 3 * kTile, &t_lo, kc * kBK, n0, bar_full_b + 8 * s);
                issued = kc + 1;
            }
            // stopped early: the last kStages requests (each its stage's latest
            // phase) land before the CTA leaves
            if (*abort_flag)
                for (int j = (issued > kStages ? issued - kStages : 0); j < issued; ++j)
                    (void)mbar_wait_bounded(bar_full_b + 8 * (j % kStages),
                                            (uint32_t)(j / kStages) & 1u, lim);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- A split, then epilogue
        const int withhold =
            withheld_stage(hook, kWithholdFilterTc, blockIdx.x == 0 && blockIdx.y == 0);
        const int cw = warp - 2;  // rows 16 cw .. 16 cw + 15 of the tile
        const int quarter = warp & 3;   // TMEM lanes 32 quarter .. +31 = tile rows
        const int half = (warp - 2) / 4;
        float sum[2][32];
        float extra = 0.0f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int j = 0; j < 32; ++j) sum[c][j] = 0.0f;
        // Add chunk kc2's accumulator into the FP32 sums, then free it.
        auto drain = [&](int kc2) -> bool {
            const int blk = kc2 % kAcc;
            if (!mbar_wait_bounded(bar_acc_full + 8 * blk, (uint32_t)(kc2 / kAcc) & 1u, lim)) {
                fail();
                return false;
            }
            tc_fence_after();
            if (half == 0)
                add_block<0>(tmem + (uint32_t)(blk * kBN), quarter, sum, extra);
            else
                add_block<1>(tmem + (uint32_t)(blk * kBN), quarter, sum, extra);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(bar_acc_free + 8 * blk);
            return true;
        };
        float cur[kRowsPerLoader], nxt[kRowsPerLoader];
        auto load_chunk = [&](int kc, float (&v)[kRowsPerLoader]) {
            const int k = kc * kBK + lane;
#pragma unroll
            for (int i = 0; i < kRowsPerLoader; ++i) {
                const int m = m0 + cw * kRowsPerLoader + i;
                v[i] = (m < args.A && k < args.D) ? __ldg(&sino[(size_t)m * ld + k]) : 0.0f;
            }
        };
        bool ok = true;
        if (args.nk > 0) load_chunk(0, cur);
        for (int kc = 0; kc < args.nk && ok; ++kc) {
            const int s = kc % kStages;
            const uint32_t use = (uint32_t)(kc / kStages);
            if (kc + 1 < args.nk) load_chunk(kc + 1, nxt);
            if (*abort_flag) {
                ok = false;
                break;
            }
            if (use > 0 && !mbar_wait_bounded(bar_empty + 8 * s, (use - 1) & 1u, lim)) {
                fail();
                ok = false;
                break;
            }
            unsigned char *a_hi = bp + s * kStageBytes;
            unsigned char *a_lo = a_hi + kTile;
#pragma unroll
            for (int i = 0; i < kRowsPerLoader; ++i) {
                const int r = cw * kRowsPerLoader + i;
                float x = cur[i];
                // intensities: converted here, a chunk after their loads were issued
                if constexpr (INTENSITY)
                    if (m0 + r < args.A && kc * kBK + lane < args.D)
                        x = line_integral(x, args.i0, args.ln_i0);
                const uint32_t hi = tf32_rna(x);
                const uint32_t lo = tf32_rna(x - __uint_as_float(hi));
                // 128-byte swizzle: 16-byte chunk (lane / 4) XOR (row mod 8)
                const uint32_t off = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 +
                                                ((((lane >> 2) ^ (r & 7)) << 4) | ((lane & 3) << 2)));
                *reinterpret_cast<uint32_t *>(a_hi + off) = hi;
                *reinterpret_cast<uint32_t *>(a_lo + off) = lo;
            }
            fence_proxy_async_smem();  // generic-proxy stores -> tensor-core reads
            // (tests only: the first CTA may withhold one stage's arrival)
            if (kc != withhold) mbar_arrive_cta(bar_full_a + 8 * s);
#pragma unroll
            for (int i = 0; i < kRowsPerLoader; ++i) cur[i] = nxt[i];
            if (kc >= 1) ok = drain(kc - 1);  // the previous chunk's MMAs are (nearly) done
        }
        if (ok && args.nk > 0) ok = drain(args.nk - 1);
        if (ok && !*abort_flag) {
            const int m = m0 + quarter * 32 + lane;
            if (m < args.A) {
                float *row = args.q[sl] + (size_t)m * args.pitch;
                if (half == 0)
                    store_half<0>(sum, extra, row, n_tile * kStep, args.pitch / 2);
                else
                    store_half<1>(sum, extra, row, n_tile * kStep, args.pitch / 2);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kAcc * kBN)
                     : "memory");
    }
}

}  // namespace

cudaError_t set_wait_hook_filter_tc(const WaitHook &h) { return write_wait_hook(h); }

size_t filter_tc_smem_bytes()
{
    return (size_t)kStages * kStageBytes + 8 * (3 * kStages + 2 * kAcc) + 16 + 1024;
}

cudaError_t launch_filter_tc_many(const Plan &p, const float *const *sinos, const int *lds,
                                  float *const *qs, int n, cudaStream_t s)
{
    const size_t smem = filter_tc_smem_bytes();
    const bool intensity = p.i0 > 0.0;
    cudaError_t e = cudaFuncSetAttribute(intensity ? filter_tc_kernel<true> : filter_tc_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int b = 0; b < n; b += kTcMaxSlices) {
        const int cnt = (n - b < kTcMaxSlices) ? n - b : kTcMaxSlices;
        TcArgs a;
        std::memset(&a, 0, sizeof a);
        for (int i = 0; i < cnt; ++i) {
            a.sino[i] = sinos[b + i];
            a.q[i] = qs[b + i];
            a.ld[i] = lds[b + i];
        }
        a.A = p.A;
        a.D = p.D;
        a.pitch = p.pitch;
        a.nk = (p.D + kBK - 1) / kBK;
        a.m_tiles = (p.A + kBM - 1) / kBM;
        a.i0 = p.i0f;
        a.ln_i0 = p.ln_i0f;
        a.status = p.d_status;
        dim3 grid((p.pitch / 2 + kStep - 1) / kStep, a.m_tiles * cnt);
        if (intensity)
            filter_tc_kernel<true><<<grid, kThreads, smem, s>>>(p.tc->t_hi, p.tc->t_lo, a);
        else
            filter_tc_kernel<false><<<grid, kThreads, smem, s>>>(p.tc->t_hi, p.tc->t_lo, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t prepare_filter_tc(const Plan &p)
{
    return cudaFuncSetAttribute(p.i0 > 0.0 ? filter_tc_kernel<true> : filter_tc_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)filter_tc_smem_bytes());
}

cudaError_t launch_filter_tc(const Plan &p, const float *sino, int ld, float *q, cudaStream_t s)
{
    return launch_filter_tc_many(p, &sino, &ld, &q, 1, s);
}

}  // namespace fbp
