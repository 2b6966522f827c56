// FP32 backprojection (Eq. 2): pixel-driven, gather-only, deterministic.
//
// Work item = one tile of TX x TY pixels (one CTA).  Angles are processed in
// chunks of CH.  For every angle the detector window the tile needs (wraw
// bins starting at a 16-byte-aligned bin `base`) is brought into shared memory
// by a 2D TMA load out of the filtered sinogram [A][pitch]; bins outside
// [0, n_det) arrive as zeros (TMA out-of-bounds fill), which is exactly the
// zero extension of the interpolation.  Two chunks are in flight (double
// buffer, one mbarrier per stage).
//
// Each staged window is rewritten once into (A'_k, B_k) pairs,
//   B_k  = Q[base+k+1] - Q[base+k]
//   A'_k = Q[base+k] - (k - 1/2) B_k
// so that with the local coordinate v = u - base - 1/2 and k = round(v),
//   lerp(Q, u) = Q[base+k] + (u - base - k) B_k = A'_k + v B_k,
// one FMA per update.  k is taken from the bits of v + 1.5*2^23 (the sum is
// rounded to an integer that lands in the low mantissa bits), so there is no
// float-to-int conversion on the hot path.  v is a tile-local coordinate
// (|v| < wraw), which keeps the FP32 position error near 1e-5 bins even where
// the global detector coordinate is in the thousands.
//
// Every pixel sums its angles in order 0..A-1 in its own registers: no
// atomics, no cross-CTA reduction, the same bits on every run.
#include "fbp_internal.h"
#include "ptx.cuh"

namespace fbp {
namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;

struct BpArgs {
    const double2 *trig64;  // (cos, sin) / tau per angle
    float *image;
    int *status;
    int n;
    int A;
    int wraw;
    int nchunks;
    float scale;    // pi / A
    double half_n;  // (n - 1) / 2
    double half_d;  // (n_det - 1) / 2
};

// Shared-memory layout (byte offsets from a 128-byte aligned origin).
struct BpSmem {
    int raw_row;  // bytes per staged raw row (128-byte multiple: TMA destination alignment)
    int tab_row;  // bytes per (A', B) row
    int raw;      // [2][CH] raw rows
    int tab;      // [CH] (A', B) rows
    int prm;      // [2][CH] float4 (c, s, off, base bits) of the staged chunk
    int cur;      // [CH] float4 of the chunk being computed
    int bar;      // [2] mbarriers
    int total;    // bytes including the alignment slack
    __host__ __device__ static BpSmem make(int wraw, int ch)
    {
        BpSmem s;
        s.raw_row = ((wraw * 4 + 127) / 128) * 128;
        s.tab_row = (wraw - 1) * 8;
        s.raw = 0;
        s.tab = s.raw + 2 * ch * s.raw_row;
        s.prm = ((s.tab + ch * s.tab_row + 15) / 16) * 16;
        s.cur = s.prm + 2 * ch * 16;
        s.bar = s.cur + ch * 16;
        s.total = s.bar + 16 + 128;
        return s;
    }
};

template <int TX, int TY, int NT, int CH>
struct BpCfg {
    static constexpr int kWarps = NT / 32;
    static constexpr int kWX = TX / 8;  // warp footprint is 8 x 4 pixels
    static constexpr int kWY = kWarps / kWX;
    static constexpr int kYStride = 4 * kWY;
    static constexpr int kPPT = TY / kYStride;  // pixels per thread
    static_assert(TX % 8 == 0 && kWX >= 1 && kWarps % kWX == 0, "tile width vs warps");
    static_assert(TY % kYStride == 0 && kPPT >= 1, "tile height vs warps");
    static_assert(CH <= 32, "one producer lane per angle of a chunk");
};

template <int TX, int TY, int NT, int CH>
__global__ void __launch_bounds__(NT)
    bp_f32_kernel(const __grid_constant__ CUtensorMap qmap, const BpArgs args)
{
    using C = BpCfg<TX, TY, NT, CH>;
    extern __shared__ __align__(128) unsigned char smem[];
    const BpSmem L = BpSmem::make(args.wraw, CH);
    const uint32_t pad = (128u - (smem_addr(smem) & 127u)) & 127u;
    unsigned char *base_ptr = smem + pad;
    float4 *prm = reinterpret_cast<float4 *>(base_ptr + L.prm);
    float4 *cur = reinterpret_cast<float4 *>(base_ptr + L.cur);
    const uint32_t bar0 = smem_addr(base_ptr + L.bar);
    const uint32_t raw0 = smem_addr(base_ptr + L.raw);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int col0 = blockIdx.x * TX;
    const int row0 = blockIdx.y * TY;
    const double x0 = (double)col0 - args.half_n;
    const double y0 = (double)row0 - args.half_n;
    const int wraw = args.wraw;
    const int wt = wraw - 1;

    if (tid == 0) {
        prefetch_tensor_map(&qmap);
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();

    // Producer: warp 0 computes each angle's window base and local offset in
    // FP64 (one lane per angle), then lane 0 issues the chunk's TMA loads.
    auto produce = [&](int cc, int s) {
        const int a0 = cc * CH;
        const int na = min(CH, args.A - a0);
        if (lane < na) {
            const double2 cs = args.trig64[a0 + lane];
            const double u0 = x0 * cs.x + y0 * cs.y + args.half_d;
            const double umin = u0 + fmin(0.0, (double)(TX - 1) * cs.x) +
                                fmin(0.0, (double)(TY - 1) * cs.y);
            const int base = (__double2int_rd(umin) - 1) & ~3;
            prm[s * CH + lane] = make_float4((float)cs.x, (float)cs.y,
                                             (float)(u0 - (double)base - 0.5),
                                             __int_as_float(base));
        }
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            const uint32_t bar = bar0 + 8u * s;
            mbar_arrive_expect_tx(bar, (uint32_t)(na * wraw * 4));
            for (int a = 0; a < na; ++a) {
                const int base = __float_as_int(prm[s * CH + a].w);
                tma_load_2d(raw0 + (uint32_t)((s * CH + a) * L.raw_row), &qmap, base, a0 + a,
                            bar);
            }
        }
    };

    if (warp == 0) {
        produce(0, 0);
        if (args.nchunks > 1) produce(1, 1);
    }

    // Per-thread pixels: column lx, rows ly0 + j * kYStride.
    const int lx = (warp % C::kWX) * 8 + (lane & 7);
    const int ly0 = (warp / C::kWX) * 4 + (lane >> 3);
    const float lxf = (float)lx;
    float lyf[C::kPPT];
    float acc[C::kPPT];
#pragma unroll
    for (int j = 0; j < C::kPPT; ++j) {
        lyf[j] = (float)(ly0 + j * C::kYStride);
        acc[j] = 0.0f;
    }

    for (int cc = 0; cc < args.nchunks; ++cc) {
        const int s = cc & 1;
        const uint32_t parity = (uint32_t)((cc >> 1) & 1);
        const int na = min(CH, args.A - cc * CH);
        const bool ok = mbar_wait_bounded(bar0 + 8u * s, parity);
        if (ok) {
            const unsigned char *raw_s = base_ptr + L.raw + s * CH * L.raw_row;
            for (int idx = tid; idx < na * wt; idx += NT) {
                const int a = idx / wt;
                const int k = idx - a * wt;
                const float *r = reinterpret_cast<const float *>(raw_s + a * L.raw_row);
                const float q0 = r[k];
                const float b = r[k + 1] - q0;
                reinterpret_cast<float2 *>(base_ptr + L.tab + a * L.tab_row)[k] =
                    make_float2(fmaf(0.5f - (float)k, b, q0), b);
            }
            if (tid < na) cur[tid] = prm[s * CH + tid];
        }
        if (__syncthreads_or(!ok)) {
            // A TMA load did not land within the limit: record it, give the
            // copies in flight a bounded chance to finish, and leave.
            if (tid == 0) {
                *reinterpret_cast<volatile int *>(args.status) = FBP_ERR_TIMEOUT;
                mbar_wait_bounded(bar0 + 8u * s, parity);
                if (cc + 1 < args.nchunks)
                    mbar_wait_bounded(bar0 + 8u * (s ^ 1), (uint32_t)(((cc + 1) >> 1) & 1));
            }
            __syncthreads();
            return;
        }
        if (warp == 0 && cc + 2 < args.nchunks) produce(cc + 2, s);

        const uint32_t tab_off = pad + (uint32_t)L.tab - (kMagicBits << 3);
#pragma unroll 2
        for (int a = 0; a < na; ++a) {
            const float4 p = cur[a];
            const uint32_t cb = tab_off + (uint32_t)(a * L.tab_row);
            const float xc = fmaf(lxf, p.x, p.z);
#pragma unroll
            for (int j = 0; j < C::kPPT; ++j) {
                const float v = fmaf(lyf[j], p.y, xc);
                const float t = __fadd_rn(v, kMagic);
                const uint32_t o = (__float_as_uint(t) << 3) + cb;
                const float2 ab = *reinterpret_cast<const float2 *>(smem + o);
                acc[j] += fmaf(v, ab.y, ab.x);
            }
        }
        __syncthreads();
    }

    const int col = col0 + lx;
#pragma unroll
    for (int j = 0; j < C::kPPT; ++j) {
        const int row = row0 + ly0 + j * C::kYStride;
        if (row < args.n && col < args.n)
            args.image[(size_t)row * args.n + col] = acc[j] * args.scale;
    }
}

constexpr int kTX = kBpTileX, kTY = kBpTileY, kNT = 256, kCH = kBpChunk;

}  // namespace

cudaError_t launch_backproject_f32(const Plan &p, const CUtensorMap &qmap, float *image,
                                   cudaStream_t s)
{
    BpArgs a;
    a.trig64 = p.d_trig64;
    a.image = image;
    a.status = p.d_status;
    a.n = p.n;
    a.A = p.A;
    a.wraw = p.bp.wraw;
    a.nchunks = (p.A + kCH - 1) / kCH;
    a.scale = p.scale32;
    a.half_n = 0.5 * (double)(p.n - 1);
    a.half_d = 0.5 * (double)(p.D - 1);
    const BpSmem L = BpSmem::make(a.wraw, kCH);
    auto kern = bp_f32_kernel<kTX, kTY, kNT, kCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    dim3 grid((p.n + kTX - 1) / kTX, (p.n + kTY - 1) / kTY);
    kern<<<grid, kNT, L.total, s>>>(qmap, a);
    return cudaGetLastError();
}

}  // namespace fbp
