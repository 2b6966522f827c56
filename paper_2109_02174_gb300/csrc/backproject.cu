// FP32 backprojection (Eq. 2): pixel-driven, gather-only, deterministic.
//
// Input: the filtered sinogram in interpolation-ready form, row i holding for
// every bin k = -1 .. n_det-1 the pair
//     (mid_k, slope_k) = ((Q[k] + Q[k+1]) / 2,  Q[k+1] - Q[k]),
// Q being zero outside [0, n_det).  With k = floor(u) and w = u - k - 1/2,
//     lerp(Q_i, u) = mid_k + w * slope_k                      (one FMA).
//
// Persistent, warp-specialised kernel.  The launch owns a list of work items,
// each one TX x TY pixel tile of one slice (one launch may hold many slices of
// different sizes; see BpLaunch); CTA b takes items b, b + grid, b + 2 grid, ...
// or, given a launch counter, the next untaken item whenever its ring has room
// (which balances uneven items and CTAs that start late behind another launch)
//   - warp NCW (the producer) walks the items' angle chunks: for each angle
//     its lanes compute, in FP64, the first pair of the detector window the
//     tile touches and the tile-local coordinate offset; lane 0 then issues
//     one 2D TMA load per angle into a ring of NSTAGE shared-memory stages
//     (pairs outside the detector arrive as zeros: TMA out-of-bounds fill,
//     which is the zero extension of the interpolation);
//   - warps 0..NCW-1 (consumers) wait for a stage's mbarrier, accumulate its
//     angles into per-thread registers, and release the stage on a second
//     mbarrier.  There is no block-wide barrier in the loop.
// Per update a consumer computes the local coordinate v = u - base - 1/2 with
// an FMA, rounds it with v + 1.5*2^23 (the integer lands in the low mantissa
// bits and gives the shared-memory address directly), forms w = v - round(v),
// loads the (mid, slope) pair and adds mid + w*slope.  Pixel pairs go through
// the packed f32x2 FMA/ADD.  The local coordinate (|v| < window) keeps the FP32
// position error near 1e-5 bins where the global detector coordinate is large.
//
// Every pixel sums its angles in order 0..A-1 in registers: no atomics, no
// cross-CTA reduction, the same bits on every run and in every batch.
//
// Point pairs (plans whose tiling is point-symmetric about the image centre):
// a work item is a tile and its mirror image through the centre, and each
// consumer thread computes a pixel and its mirrored partner from one detector
// position, which takes the position, rounding and fraction off the FP32 pipe
// for half of the updates (the same saving two slices of a batch get from
// sharing them).  A plan uses them in every path (alone, batched, served), so
// its results are the same bits everywhere.
//
// Every mbarrier wait is bounded (the run-time limit of WaitHook).  A consumer
// whose wait runs out records FBP_ERR_TIMEOUT and leaves; a producer whose
// wait for a free stage runs out records it, waits (bounded again) for the
// TMA loads it issued into the ring to land, and leaves, so no bulk copy is
// in flight when the CTA exits.  For tests, the first CTA can withhold one
// stage's arrival (no TMA issued for it), which makes those waits run out.
#include <cstring>
#include <type_traits>

#include "backproject.cuh"
#include "ptx.cuh"
#include "waithook.cuh"

namespace fbp {
namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;
static_assert(kStatusBounds == FBP_ERR_BOUNDS, "status code of the index checks");

__device__ __forceinline__ float2 lds_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ float2 lds_h2_as_f2(uint32_t addr)
{
    uint32_t h;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(h) : "r"(addr));
    __half2 v = *reinterpret_cast<__half2 *>(&h);
    return __half22float2(v);
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t h;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(h) : "r"(addr));
    return h;
}

// acc + mid + w slope for an FP16 (mid, slope) pair (mid in the low half),
// in FP32 with the FP16 operands taken as they are (no conversion); the
// weight is the low (LO) or high half of the packed f16 pair w2.
template <bool LO>
__device__ __forceinline__ float acc_pair_f16(float acc, uint32_t pair, uint32_t w2)
{
    if constexpr (LO)
        asm("{\n\t.reg .b16 m, s, wl, wh;\n\tmov.b32 {m, s}, %1;\n\tmov.b32 {wl, wh}, %2;\n\t"
            "add.rn.f32.f16 %0, m, %0;\n\tfma.rn.f32.f16 %0, wl, s, %0;\n\t}"
            : "+f"(acc) : "r"(pair), "r"(w2));
    else
        asm("{\n\t.reg .b16 m, s, wl, wh;\n\tmov.b32 {m, s}, %1;\n\tmov.b32 {wl, wh}, %2;\n\t"
            "add.rn.f32.f16 %0, m, %0;\n\tfma.rn.f32.f16 %0, wh, s, %0;\n\t}"
            : "+f"(acc) : "r"(pair), "r"(w2));
    return acc;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <typename PairT>
struct PairTraits;
template <>
struct PairTraits<float> {
    static constexpr int kBytes = 8;   // one (mid, slope) pair
    static constexpr int kAlign = 2;   // pairs per 16 bytes: window start granularity
    static constexpr int kShift = 3;   // log2(kBytes)
};
template <>
struct PairTraits<__half> {
    static constexpr int kBytes = 4;
    static constexpr int kAlign = 4;
    static constexpr int kShift = 2;
};

template <int NSTAGE, int CH>
struct Layout {
    int row;    // bytes per staged window row (128-byte multiple)
    int stage;  // bytes per stage
    int prm;    // offset of params [NSTAGE][CH] float4
    int full;   // offset of full barriers [NSTAGE]
    int empty;  // offset of empty barriers [NSTAGE]
    int items;  // offset of the work item of each stage [NSTAGE] int
    int total;  // bytes including 128 of alignment slack
    __host__ __device__ static Layout make(int wp_max, int pair_bytes, int group)
    {
        Layout L;
        L.row = ((wp_max * pair_bytes + 127) / 128) * 128;
        L.stage = group * CH * L.row;
        L.prm = NSTAGE * L.stage;
        L.full = L.prm + NSTAGE * CH * 16;
        L.empty = L.full + NSTAGE * 8;
        L.items = L.empty + NSTAGE * 8;
        L.total = L.items + NSTAGE * 4 + 128;
        return L;
    }
};

// Work item -> (slice, item within the slice) through the prefix sums of the
// slices' item counts.
template <int MAXS>
__device__ __forceinline__ int2 item_of(const BpLaunch<MAXS> &P, int item)
{
    int lo = 0, hi = P.n_slices - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (item < P.tile_end[mid]) hi = mid; else lo = mid + 1;
    }
    return make_int2(lo, item - (lo > 0 ? P.tile_end[lo - 1] : 0));
}

// Launch bounds: the block size and a minimum of one resident CTA per SM,
// which leaves the register budget to the compiler's scheduling of the angle
// loop.  Measured against the default budget (62 registers) and against a cap
// for eight CTAs per SM: batched 64 x 512^2 x 720 at tile 32x32 / 32 angles
// per stage 4547 vs 3935 Gupdates/s, one 512^2 slice 2866 vs 1998, one 2048^2
// slice 3746 vs 3643; the cap for eight CTAs was never faster.
//
// G rows of window per angle and stage: G = 1, one tile of one slice; G = 2,
// either the same tile of two slices of one plan (PP = false) or, with point
// pairs (PP = true), a tile A and its point-symmetric partner B of one slice.
// A pixel at (x, y) and its partner at (-x, -y) have detector coordinates u and
// n_det - 1 - u, so the partner's pair index within B's window is K - j (K per
// tile pair and angle, from the two window starts) and its weight is -w: one
// position computation serves both pixels.
template <typename PairT, bool KAHAN, int WX, int WY, int CH, int G, int MAXS, bool PP>
__global__ void __launch_bounds__(32 * (WX * WY + 1), 1)
    bp_persistent_kernel(const __grid_constant__ BpLaunch<MAXS> P)
{
    static_assert(G == 1 || G == 2, "one or two rows per item");
    static_assert(!(KAHAN && G == 2) || sizeof(PairT) == 4, "two-row Kahan items: FP32 pairs");
    static_assert(!PP || G == 2, "point pairs stage two rows per angle");
    constexpr int NCW = WX * WY;           // consumer warps
    constexpr int TX = 8 * WX;             // tile width  (warp footprint 8 wide)
    constexpr int TY = 32 * WY;            // tile height (warp covers 32 rows)
    constexpr int PPT = 8;                 // pixels per consumer thread (rows ly0 + 4j)
    constexpr int NSTAGE = bp_stages(CH, G);
    using TR = PairTraits<PairT>;
    using L_t = Layout<NSTAGE, CH>;
    static_assert(CH <= 32, "one producer lane per angle of a chunk");

    extern __shared__ __align__(128) unsigned char smem[];
    const L_t L = L_t::make(P.wp_max, TR::kBytes, G);
    const uint32_t base_addr = (smem_addr(smem) + 127u) & ~127u;
    unsigned char *base_ptr = smem + (base_addr - smem_addr(smem));
    float4 *prm = reinterpret_cast<float4 *>(base_ptr + L.prm);
    volatile int *stage_items = reinterpret_cast<volatile int *>(base_ptr + L.items);
    const uint32_t full0 = base_addr + (uint32_t)L.full;
    const uint32_t empty0 = base_addr + (uint32_t)L.empty;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, NCW);
        }
        fence_proxy_async_smem();
    }
    __syncthreads();

    // single-slice launches (MAXS = 1) always stride: no counter code in them
    const bool dyn = MAXS > 1 && P.sched != nullptr;
    const WaitHook hook = g_wait_hook;
    const unsigned long long lim = wait_limit_ns(hook);

    if (warp == NCW) {
        // ------------------------------------------------------------ producer
        // The next work item comes from the launch's counter (P.sched: taken
        // when the ring has room for the item's first stage, so a CTA that
        // started late or drew cheap items takes more; every stage records its
        // item for the consumers, and a stage recording -1 ends their loop) or,
        // without one, by striding (b, b + grid, ...), which the consumers
        // follow on their own.
        const int withhold = withheld_stage(hook, kWithholdBackproject, blockIdx.x == 0);
        auto wait_empty = [&](uint32_t i) -> bool {
            const uint32_t use = i / NSTAGE;
            bool ok = true;
            if (use > 0) ok = mbar_wait_bounded(empty0 + 8u * (i % NSTAGE), (use - 1) & 1u, lim);
            return __all_sync(0xffffffffu, ok);
        };
        // A wait for stage i's slot ran out: record it, then let the loads
        // issued into the ring (stages i - NSTAGE .. i - 1, each its latest
        // phase) land before leaving.
        auto give_up = [&](uint32_t i) {
            if (lane == 0) {
                *reinterpret_cast<volatile int *>(P.status) = FBP_ERR_TIMEOUT;
                for (uint32_t j = (i >= (uint32_t)NSTAGE ? i - NSTAGE : 0u); j < i; ++j)
                    if ((int)j != withhold)
                        (void)mbar_wait_bounded(full0 + 8u * (j % NSTAGE), (j / NSTAGE) & 1u, lim);
            }
            __syncwarp();
        };
        uint32_t it = 0;
        int item = blockIdx.x;
        for (;;) {
            if (!dyn && item >= P.n_items) return;  // the consumers stride too
            if (!wait_empty(it)) {
                give_up(it);
                return;
            }
            if (dyn) {
                int v = 0;
                if (lane == 0) v = atomicAdd(P.sched, 1);
                item = __shfl_sync(0xffffffffu, v, 0);
            }
            if (item >= P.n_items) {
                if (lane == 0) {
                    const int s = (int)(it % NSTAGE);
                    stage_items[s] = -1;
                    mbar_arrive(full0 + 8u * s);  // no bytes: completes the phase
                    // the last CTA past the end leaves the counter at zero for
                    // the next launch that uses it
                    if (atomicAdd(P.sched + 1, 1) == (int)gridDim.x - 1) {
                        atomicExch(P.sched, 0);
                        atomicExch(P.sched + 1, 0);
                    }
                }
                return;
            }
            const int2 wi = item_of(P, item);
            const BpSlice &S = P.slices[wi.x];
            const int tx = wi.y % S.tiles_x, ty = wi.y / S.tiles_x;
            const double x0 = (double)(tx * TX) - S.half_n;
            const double y0 = (double)(ty * TY) - S.half_n;
            // point pairs: the partner tile's origin (tile tiles - 1 - item)
            const int tb = S.tiles - 1 - wi.y;
            const double x0b = (double)((tb % S.tiles_x) * TX) - S.half_n;
            const double y0b = (double)((tb / S.tiles_x) * TY) - S.half_n;
            const int nch = (S.A + CH - 1) / CH;
            for (int cc = 0; cc < nch; ++cc, ++it) {
                const int s = (int)(it % NSTAGE);
                if (cc > 0 && !wait_empty(it)) {
                    give_up(it);
                    return;
                }
                const int a0 = cc * CH;
                const int na = min(CH, S.A - a0);
                int pb = 0, pbb = 0;
                if (lane < na) {
                    const double2 cs = S.trig64[a0 + lane];
                    const double ex = fmin(0.0, (double)(TX - 1) * cs.x) +
                                      fmin(0.0, (double)(TY - 1) * cs.y);
                    const double u0 = x0 * cs.x + y0 * cs.y + S.half_d;
                    // first pair of the window: pair p holds bin k = p - 1; start
                    // one bin below floor(umin), aligned down to 16 bytes.
                    pb = __double2int_rd(u0 + ex) & ~(TR::kAlign - 1);
                    const int base = pb - 1;  // bin of the window's first pair
                    int w4 = 0;
                    if constexpr (PP) {
                        const double u0b = x0b * cs.x + y0b * cs.y + S.half_d;
                        pbb = __double2int_rd(u0b + ex) & ~(TR::kAlign - 1);
                        // partner pair index K - j, K = n_det - pb - pbb
                        w4 = (int)(2.0 * S.half_d + 1.0) - pb - pbb;
                    }
                    prm[s * CH + lane] = make_float4((float)cs.x, (float)cs.y,
                                                     (float)(u0 - (double)base - 0.5),
                                                     __int_as_float(w4));
                }
                if (lane == 0) stage_items[s] = item;
                __syncwarp();
                // (tests only: a withheld stage gets neither its arrival nor its loads)
                const bool fill = (int)it != withhold;
                // rows of the item: a single slice in a two-slice launch stages one
                const int rows = (G == 2 && !PP && S.image2 == nullptr) ? 1 : G;
                if (lane == 0 && fill) {
                    const uint32_t bar = full0 + 8u * s;
                    mbar_arrive_expect_tx(bar, (uint32_t)(rows * na * S.wp * TR::kBytes));
                }
                __syncwarp();
                // each lane issues its own angle's load(s) (x in elements of PairT);
                // row g of the item lands in rows g*CH .. g*CH + CH-1 of the stage
                if (lane < na && fill) {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (g >= rows) break;
                        // two slices: the same window of each slice's rows; point
                        // pairs: the partner tile's window of the one slice
                        const int xg = (PP && g) ? pbb : pb;
                        tma_load_2d(base_addr + (uint32_t)(s * L.stage + (g * CH + lane) * L.row),
                                    &P.maps[PP ? wi.x : G * wi.x + g], 2 * xg, a0 + lane,
                                    full0 + 8u * s);
                    }
                }
            }
            if (!dyn) item += gridDim.x;
        }
    }

    // ---------------------------------------------------------------- consumers
    const int lx = (warp % WX) * 8 + (lane & 7);
    const int ly0 = (warp / WX) * 32 + (lane >> 3);
    const float lxf = (float)lx;
    float2 ypair[PPT / 2];
#pragma unroll
    for (int jj = 0; jj < PPT / 2; ++jj)
        ypair[jj] = make_float2((float)(ly0 + 8 * jj), (float)(ly0 + 8 * jj + 4));
    const float2 kM2 = make_float2(kMagic, kMagic);
    const float2 kNegM2 = make_float2(-kMagic, -kMagic);
    const float2 kNeg1 = make_float2(-1.0f, -1.0f);

    auto wait_full = [&](uint32_t i) -> bool {
        const bool ok = mbar_wait_bounded(full0 + 8u * (i % NSTAGE), (i / NSTAGE) & 1u, lim);
        return __all_sync(0xffffffffu, ok);
    };
    uint32_t it = 0;
    int item = blockIdx.x;
    for (;;) {
        if (dyn) {
            if (!wait_full(it)) {
                if (lane == 0) *reinterpret_cast<volatile int *>(P.status) = FBP_ERR_TIMEOUT;
                return;
            }
            item = stage_items[it % NSTAGE];
            if (item < 0) break;
        } else if (item >= P.n_items) {
            break;
        }
        const int2 wi = item_of(P, item);
        const BpSlice &S = P.slices[wi.x];
        const int tx = wi.y % S.tiles_x, ty = wi.y / S.tiles_x;
        const int nch = (S.A + CH - 1) / CH;
        float acc[G][PPT];
        float cmp[KAHAN ? G : 1][KAHAN ? PPT : 1];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int j = 0; j < PPT; ++j) acc[g][j] = 0.0f;
#pragma unroll
        for (int g = 0; g < (KAHAN ? G : 1); ++g)
#pragma unroll
            for (int j = 0; j < (KAHAN ? PPT : 1); ++j) cmp[g][j] = 0.0f;

        // The item's angle chunks; GC = rows of the item actually staged (a
        // two-slice launch also carries single slices: their second row is
        // absent).  false: a wait ran out.
        auto chunks = [&](auto gcv) -> bool {
        constexpr int GC = decltype(gcv)::value;
        for (int cc = 0; cc < nch; ++cc, ++it) {
            const int s = (int)(it % NSTAGE);
            if ((cc > 0 || !dyn) && !wait_full(it)) {
                if (lane == 0) *reinterpret_cast<volatile int *>(P.status) = FBP_ERR_TIMEOUT;
                return false;
            }
            const int na = min(CH, S.A - cc * CH);
            const uint32_t stage_addr = base_addr + (uint32_t)(s * L.stage);
            const float4 *pp = prm + s * CH;
#pragma unroll 2
            for (int a = 0; a < na; ++a) {
                const float4 p = pp[a];
                const uint32_t cb =
                    stage_addr + (uint32_t)(a * L.row) - (kMagicBits << TR::kShift);
                // point pairs: the partner reads pair K - j of its row (CH rows on)
                const uint32_t cbb = stage_addr + (uint32_t)((CH + a) * L.row) +
                                     ((uint32_t)__float_as_int(p.w) << TR::kShift) +
                                     (kMagicBits << TR::kShift);
                const float xc = fmaf(lxf, p.x, p.z);
                const float2 xc2 = make_float2(xc, xc);
                const float2 s2 = make_float2(p.y, p.y);
#pragma unroll
                for (int jj = 0; jj < PPT / 2; ++jj) {
                    const float2 v = __ffma2_rn(ypair[jj], s2, xc2);
                    const float2 t = __fadd2_rn(v, kM2);
                    const float2 kf = __fadd2_rn(t, kNegM2);
                    const float2 w = __ffma2_rn(kf, kNeg1, v);
                    uint32_t ux = __float_as_uint(t.x), uy = __float_as_uint(t.y);
#ifdef FBP_CHECK_BOUNDS
                    // debug builds: the pair index must lie in the staged window
                    ux = (uint32_t)check_index((int)(ux - kMagicBits), S.wp - hook.shrink,
                                               P.status, kCheckBackproject) + kMagicBits;
                    uy = (uint32_t)check_index((int)(uy - kMagicBits), S.wp - hook.shrink,
                                               P.status, kCheckBackproject) + kMagicBits;
#endif
                    const uint32_t o0 = (ux << TR::kShift) + cb;
                    const uint32_t o1 = (uy << TR::kShift) + cb;
                    // FP16 pairs: the two fractions as an f16 pair (low: w.x)
                    uint32_t w16 = 0;
                    if constexpr (TR::kBytes == 4 && !KAHAN)
                        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w16) : "f"(w.y), "f"(w.x));
#pragma unroll
                    for (int g = 0; g < GC; ++g) {
                        uint32_t a0, a1;
                        if constexpr (PP) {
                            a0 = g ? cbb - (ux << TR::kShift) : o0;
                            a1 = g ? cbb - (uy << TR::kShift) : o1;
#ifdef FBP_CHECK_BOUNDS
                            if (g) {
                                // the partner's index K - j in its own window
                                const int kk = __float_as_int(p.w);
                                const int jx = (int)(ux - kMagicBits), jy = (int)(uy - kMagicBits);
                                const uint32_t row_b = stage_addr + (uint32_t)((CH + a) * L.row);
                                a0 = row_b + ((uint32_t)check_index(kk - jx, S.wp - hook.shrink,
                                                                    P.status, kCheckBackproject)
                                              << TR::kShift);
                                a1 = row_b + ((uint32_t)check_index(kk - jy, S.wp - hook.shrink,
                                                                    P.status, kCheckBackproject)
                                              << TR::kShift);
                            }
#endif
                        } else {
                            const uint32_t go = (uint32_t)(g * CH * L.row);
                            a0 = o0 + go;
                            a1 = o1 + go;
                        }
                        if constexpr (TR::kBytes == 4 && !KAHAN) {
                            // the partner's weight is -w: flip both sign bits
                            const uint32_t wg = (PP && g) ? (w16 ^ 0x80008000u) : w16;
                            acc[g][2 * jj] = acc_pair_f16<true>(acc[g][2 * jj], lds_u32(a0), wg);
                            acc[g][2 * jj + 1] =
                                acc_pair_f16<false>(acc[g][2 * jj + 1], lds_u32(a1), wg);
                            continue;
                        }
                        float2 q0, q1;
                        if constexpr (TR::kBytes == 8) {
                            q0 = lds_f2(a0);
                            q1 = lds_f2(a1);
                        } else {
                            q0 = lds_h2_as_f2(a0);
                            q1 = lds_h2_as_f2(a1);
                        }
                        // the partner's weight is -w
                        const float wx = (PP && g) ? -w.x : w.x;
                        const float wy = (PP && g) ? -w.y : w.y;
                        const float v0 = fmaf(wx, q0.y, q0.x);
                        const float v1 = fmaf(wy, q1.y, q1.x);
                        if constexpr (KAHAN) {
                            const int gk = KAHAN ? g : 0;
                            const float y0 = v0 - cmp[gk][2 * jj];
                            const float t0 = acc[g][2 * jj] + y0;
                            cmp[gk][2 * jj] = (t0 - acc[g][2 * jj]) - y0;
                            acc[g][2 * jj] = t0;
                            const float y1 = v1 - cmp[gk][2 * jj + 1];
                            const float t1 = acc[g][2 * jj + 1] + y1;
                            cmp[gk][2 * jj + 1] = (t1 - acc[g][2 * jj + 1]) - y1;
                            acc[g][2 * jj + 1] = t1;
                        } else {
                            acc[g][2 * jj] += v0;
                            acc[g][2 * jj + 1] += v1;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8u * s);
        }
        return true;
        };
        // single slice in a two-slice launch: its own loop, no second row
        const bool solo = G == 2 && !PP && S.image2 == nullptr;
        const bool ok = solo ? chunks(std::integral_constant<int, 1>())
                             : chunks(std::integral_constant<int, G>());
        if (!ok) return;

        if constexpr (PP) {
            // tile A and, mirrored through the image centre, its partner
            // (tilings with n a multiple of the tile: every pixel is inside)
            const int col = tx * TX + lx;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int row = ty * TY + ly0 + 4 * j;
                S.image[(size_t)row * S.n + col] = acc[0][j] * S.scale;
                S.image[(size_t)(S.n - 1 - row) * S.n + (S.n - 1 - col)] = acc[1][j] * S.scale;
            }
        } else {
            const int col = tx * TX + lx;
            if (col < S.n) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float *img = g ? S.image2 : S.image;
                    if (img == nullptr) break;  // a single slice of a two-slice launch
#pragma unroll
                    for (int j = 0; j < PPT; ++j) {
                        const int row = ty * TY + ly0 + 4 * j;
                        if (row < S.n) img[(size_t)row * S.n + col] = acc[g][j] * S.scale;
                    }
                }
            }
        }
        if (!dyn) item += gridDim.x;
    }
}

template <typename PairT, bool KAHAN, int WX, int WY, int CH, int G, int MAXS, bool PP>
cudaError_t launch_one(const BpLaunch<MAXS> &P, int grid_limit, cudaStream_t s)
{
    using L_t = Layout<bp_stages(CH, G), CH>;
    const L_t L = L_t::make(P.wp_max, PairTraits<PairT>::kBytes, G);
    auto kern = bp_persistent_kernel<PairT, KAHAN, WX, WY, CH, G, MAXS, PP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L.total);
    if (e != cudaSuccess) return e;
    const int threads = 32 * (WX * WY + 1);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, L.total);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (grid_limit < 0) return cudaSuccess;  // preparation only: the kernel is loaded
    int grid = sms * (per_sm > 0 ? per_sm : 1);
    if (grid_limit > 0 && grid > grid_limit) grid = grid_limit;
    if (grid > P.n_items) grid = P.n_items;
    if (grid < 1) grid = 1;
    kern<<<grid, threads, L.total, s>>>(P);
    return cudaGetLastError();
}

template <typename PairT, bool KAHAN, int WX, int WY, int G, int MAXS, bool PP>
cudaError_t by_chunk(const BpLaunch<MAXS> &P, int chunk, int grid_limit, cudaStream_t s)
{
    if (chunk == 8) return launch_one<PairT, KAHAN, WX, WY, 8, G, MAXS, PP>(P, grid_limit, s);
    if (chunk == 32) return launch_one<PairT, KAHAN, WX, WY, 32, G, MAXS, PP>(P, grid_limit, s);
    if (chunk == 16) return launch_one<PairT, KAHAN, WX, WY, 16, G, MAXS, PP>(P, grid_limit, s);
    return cudaErrorInvalidValue;
}

template <int WX, int WY, int MAXS>
cudaError_t by_variant(const BpLaunch<MAXS> &P, const BpConfig &c, int grid_limit, cudaStream_t s)
{
    // Kahan sums with two rows per item: FP32 pairs only (with FP16 pairs the
    // storage, not the sum, sets the error)
    if (c.point_pairs) {
        // one slice per item, a tile and its partner
        if (c.group != 1 || (c.kahan && c.half_pairs)) return cudaErrorInvalidValue;
        if (c.kahan) return by_chunk<float, true, WX, WY, 2, MAXS, true>(P, c.chunk, grid_limit, s);
        if (!c.half_pairs)
            return by_chunk<float, false, WX, WY, 2, MAXS, true>(P, c.chunk, grid_limit, s);
        return by_chunk<__half, false, WX, WY, 2, MAXS, true>(P, c.chunk, grid_limit, s);
    }
    if (c.group == 2) {
        if constexpr (MAXS > 1) {
            if (c.kahan && c.half_pairs) return cudaErrorInvalidValue;
            if (c.kahan)
                return by_chunk<float, true, WX, WY, 2, MAXS, false>(P, c.chunk, grid_limit, s);
            if (!c.half_pairs)
                return by_chunk<float, false, WX, WY, 2, MAXS, false>(P, c.chunk, grid_limit, s);
            return by_chunk<__half, false, WX, WY, 2, MAXS, false>(P, c.chunk, grid_limit, s);
        }
        return cudaErrorInvalidValue;
    }
    if (!c.half_pairs && !c.kahan)
        return by_chunk<float, false, WX, WY, 1, MAXS, false>(P, c.chunk, grid_limit, s);
    if (!c.half_pairs && c.kahan)
        return by_chunk<float, true, WX, WY, 1, MAXS, false>(P, c.chunk, grid_limit, s);
    if (c.half_pairs && !c.kahan)
        return by_chunk<__half, false, WX, WY, 1, MAXS, false>(P, c.chunk, grid_limit, s);
    return by_chunk<__half, true, WX, WY, 1, MAXS, false>(P, c.chunk, grid_limit, s);
}

template <int MAXS>
cudaError_t dispatch(const BpLaunch<MAXS> &P, const BpConfig &c, int grid_limit, cudaStream_t s)
{
    if (c.wx == 4 && c.wy == 2) return by_variant<4, 2, MAXS>(P, c, grid_limit, s);
    if (c.wx == 4 && c.wy == 1) return by_variant<4, 1, MAXS>(P, c, grid_limit, s);
    if (c.wx == 1 && c.wy == 1) return by_variant<1, 1, MAXS>(P, c, grid_limit, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t set_wait_hook_backproject(const WaitHook &h) { return write_wait_hook(h); }

cudaError_t launch_backproject(const BpLaunch<1> &P, const BpConfig &c, cudaStream_t s)
{
    return dispatch<1>(P, c, 0, s);
}

cudaError_t prepare_backproject(const Plan &p)
{
    BpLaunch<1> L;
    std::memset(&L, 0, sizeof L);
    L.wp_max = p.bp_wp;
    return dispatch<1>(L, bp_config(p), -1, nullptr);
}

cudaError_t launch_backproject_batch(const BpLaunch<kBpMaxSlices> &P, const BpConfig &c,
                                     int grid_limit, cudaStream_t s)
{
    return dispatch<kBpMaxSlices>(P, c, grid_limit, s);
}

}  // namespace fbp
