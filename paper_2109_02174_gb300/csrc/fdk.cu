// FDK cone-beam reconstruction (Feldkamp, Davis & Kress 1984): the 3D
// extension the paper names as its future work (section "Conclusion"), built
// on the 2D path's filter.  Geometry (the paper fixes none): the source
// circles the z axis at radius R, at (R cos b, R sin b, 0); projections live on
// a virtual flat detector through the axis with u along (-sin b, cos b, 0) and
// v along z, P[a][i][j] at u_j = (j - (nu-1)/2) du, v_i = (i - (nv-1)/2) dv;
// voxel (ix, iy, iz) of f[nz][ny][nx] has centre
// (ix - (nx-1)/2, iy - (ny-1)/2, iz - (nz-1)/2).
//
//   1. weight and filter: every detector row (A nv rows of nu bins) goes
//      through the FFT ramp filter, its values multiplied on load by the
//      cosine weight R / sqrt(R^2 + u^2 + v^2) (a plan table), and leaves as
//      (mid, slope) pairs along u;
//   2. per (tile, angle) parameters, computed once per plan in FP64: the
//      projection of the tile centre, u_c = R t_c / U_c and v_c = R z_c / U_c
//      (s_c = x_c cos b + y_c sin b, t_c = -x_c sin b + y_c cos b,
//      U_c = R - s_c), and the detector window the tile's eight corners span
//      (a perspective projection maps the box into the hull of their images),
//      stored as the window's first pair and row plus the centre's offset from
//      them;
//   3. backprojection, gather-only and deterministic: one CTA per
//      16 x 16 x 16 voxel tile.  A producer warp brings each angle's window of
//      filtered pairs into shared memory with one 3D TMA load (rows outside
//      the detector arrive as zeros) into a ring of stages; 256 consumer
//      threads, one per (x, y) column, run down their 16 voxels.  A voxel at
//      (dx, dy, dz) from the centre projects to
//          u - u_c = R (dt U_c + t_c ds) / (U U_c),  v - v_c = R (dz U_c + z_c ds) / (U U_c)
//      (ds = dx cos b + dy sin b, dt = -dx sin b + dy cos b, U = U_c - ds), small
//      offsets, so FP32 keeps the detector position to about 1e-6 bins; the u
//      sample and the weight (R/U)^2 are formed once per column and angle,
//      each voxel reads two rows of pairs (bilinear; voxels taken two at a time
//      in packed f32x2 arithmetic), and angles are summed in order; the sum is
//      scaled by pi / A (a full turn).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fbp_internal.h"
#include "ptx.cuh"
#include "waithook.cuh"

namespace fbp {

cudaError_t launch_filter_fft(const Plan &p, const float *sino, int ld, void *q, cudaStream_t s);

namespace {

constexpr int kT = 16;                 // tile edge (voxels)
constexpr int kConsumers = kT * kT;    // one thread per (x, y) column
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kThreads = kConsumers + 32;  // + the TMA producer warp
constexpr int kStages = 2;
constexpr size_t kSmemBudget = 200 * 1024;
constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23: x + kMagic holds round(x) in its low bits
constexpr int kMagicLow = 0x4B400000;

__device__ __forceinline__ float2 lds_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

struct FdkPrm {
    float c, s, uc, tc;  // cos b, sin b, U_c, t_c
    float kuo, kvo;      // centre's bin and row coordinate, relative to the window
    int p0, r0;          // window's first pair (even) and first row
};

struct FdkPlan {
    int A, nv, nu, nx, ny, nz;
    double R, du, dv;
    int tiles_x, tiles_y, tiles_z;
    int wu, wv;          // window: pairs (even) and rows of one angle's box
    int ch;              // angles per shared-memory stage
    size_t box_bytes;    // one angle's box in shared memory (128-byte multiple)
    fbp_plan_t filt;     // FFT filter plan over the A nv rows
    float *d_wt;         // [nv][nu] cosine weights
    double2 *d_trig;     // (cos b, sin b)
    FdkPrm *d_prm;       // [tiles][A]
    int device;
};

struct FdkArgs {
    int A, nv, nu, nx, ny, nz, pitch2, tiles_x, tiles_y, tiles_z;
    int wu, wv, ch, box_bytes;
    float Ru, Rv, R;  // R / du, R / dv, R
    double R64, du, dv;
    float scale;      // pi / A
    int *status;
};

__device__ __forceinline__ double ku_of(const FdkArgs &g, double x, double y, double cb,
                                        double sb)
{
    const double t = -x * sb + y * cb, U = g.R64 - (x * cb + y * sb);
    return g.R64 * t / U / g.du + 0.5 * (g.nu - 1);
}

__device__ __forceinline__ double kv_of(const FdkArgs &g, double x, double y, double z,
                                        double cb, double sb)
{
    const double U = g.R64 - (x * cb + y * sb);
    return g.R64 * z / U / g.dv + 0.5 * (g.nv - 1);
}

// Parameters of every (tile, angle) and the largest window any needs
// (ext[0]: pairs, ext[1]: rows).
__global__ void __launch_bounds__(256)
    fdk_params_kernel(const double2 *__restrict__ trig, FdkPrm *__restrict__ prm, FdkArgs g,
                      int *ext)
{
    const long ntile = (long)g.tiles_x * g.tiles_y * g.tiles_z;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntile * g.A) return;
    const long tile = idx / g.A;
    const int a = (int)(idx - tile * g.A);
    const int tx = (int)(tile % g.tiles_x);
    const int ty = (int)((tile / g.tiles_x) % g.tiles_y);
    const int tz = (int)(tile / ((long)g.tiles_x * g.tiles_y));
    const double h = 0.5 * (kT - 1);
    const double xc = (double)(tx * kT) + h - 0.5 * (g.nx - 1);
    const double yc = (double)(ty * kT) + h - 0.5 * (g.ny - 1);
    const double zc = (double)(tz * kT) + h - 0.5 * (g.nz - 1);
    const double2 cs = trig[a];
    double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
    for (int k = 0; k < 8; ++k) {
        const double x = xc + ((k & 1) ? h : -h), y = yc + ((k & 2) ? h : -h);
        const double z = zc + ((k & 4) ? h : -h);
        const double ku = ku_of(g, x, y, cs.x, cs.y), kv = kv_of(g, x, y, z, cs.x, cs.y);
        umin = fmin(umin, ku);
        umax = fmax(umax, ku);
        vmin = fmin(vmin, kv);
        vmax = fmax(vmax, kv);
    }
    // bins floor(umin) .. floor(umax) use pairs floor(umin)+1 .. floor(umax)+1; one
    // pair of margin each side, first pair even (16-byte TMA coordinate)
    const int p0 = (int)floor(umin) & ~1;
    const int p_last = (int)floor(umax) + 2;
    // rows floor(vmin) .. floor(vmax)+1, one row of margin each side
    const int r0 = (int)floor(vmin) - 1;
    const int r_last = (int)floor(vmax) + 2;
    atomicMax(&ext[0], p_last - p0 + 1);
    atomicMax(&ext[1], r_last - r0 + 1);
    const double sc = xc * cs.x + yc * cs.y;
    const double tc = -xc * cs.y + yc * cs.x;
    const double Uc = g.R64 - sc;
    FdkPrm P;
    P.c = (float)cs.x;
    P.s = (float)cs.y;
    P.uc = (float)Uc;
    P.tc = (float)tc;
    P.kuo = (float)(ku_of(g, xc, yc, cs.x, cs.y) - (double)(p0 - 1));  // bin (p0-1) <-> window pair 0
    P.kvo = (float)(kv_of(g, xc, yc, zc, cs.x, cs.y) - (double)r0);
    P.p0 = p0;
    P.r0 = r0;
    prm[idx] = P;
}

__global__ void __launch_bounds__(kThreads, 2)
    fdk_backproject_kernel(const __grid_constant__ CUtensorMap qmap,
                           const FdkPrm *__restrict__ prm, float *__restrict__ vol,
                           const FdkArgs g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t base = (smem_addr(smem) + 127u) & ~127u;
    unsigned char *bp = smem + (base - smem_addr(smem));
    const uint32_t full0 = base + (uint32_t)(kStages * g.ch * g.box_bytes);
    const uint32_t empty0 = full0 + 8u * kStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, kConsumerWarps);
        }
        fence_proxy_async_smem();
    }
    __syncthreads();
    const int tile = blockIdx.x;
    const FdkPrm *pt = prm + (size_t)tile * g.A;
    const int nch = (g.A + g.ch - 1) / g.ch;
    const uint32_t box_payload = (uint32_t)(g.wv * 2 * g.wu * 4);
    const WaitHook hook = g_wait_hook;
    const unsigned long long lim = wait_limit_ns(hook);
    const int shrink = hook.shrink;
    (void)shrink;

    if (warp == kConsumerWarps) {
        // ---------------------------------------------------- TMA producer
        for (int c = 0; c < nch; ++c) {
            const int s = c % kStages;
            const uint32_t use = (uint32_t)(c / kStages);
            bool ok = true;
            if (use > 0) ok = mbar_wait_bounded(empty0 + 8u * s, (use - 1) & 1u, lim);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    *reinterpret_cast<volatile int *>(g.status) = FBP_ERR_TIMEOUT;
                    // the loads already issued (each stage's latest phase) land first
                    for (int j = (c > kStages ? c - kStages : 0); j < c; ++j)
                        (void)mbar_wait_bounded(full0 + 8u * (j % kStages),
                                                (uint32_t)(j / kStages) & 1u, lim);
                }
                __syncwarp();
                return;
            }
            const int a0 = c * g.ch;
            const int na = min(g.ch, g.A - a0);
            if (lane == 0) mbar_arrive_expect_tx(full0 + 8u * s, (uint32_t)na * box_payload);
            __syncwarp();
            if (lane < na) {
                const FdkPrm P = pt[a0 + lane];
                tma_load_3d(base + (uint32_t)((s * g.ch + lane) * g.box_bytes), &qmap, 2 * P.p0,
                            P.r0, a0 + lane, full0 + 8u * s);
            }
        }
        return;
    }

    // -------------------------------------------------------- consumers
    const int tx = tile % g.tiles_x;
    const int ty = (tile / g.tiles_x) % g.tiles_y;
    const int tz = tile / (g.tiles_x * g.tiles_y);
    // a warp covers 8 x 4 columns (a half-warp 8 x 2), so a half-warp's
    // detector bins span about 8 pairs and fewer of its 8-byte loads meet in a
    // bank (16 x 2 columns per warp: 4.30 ms for the bench's reconstruction,
    // 8 x 4: 4.13 ms)
    const int cx = (warp & 1) * 8 + (lane & 7);
    const int cy = (warp >> 1) * 4 + (lane >> 3);
    const float dx = (float)cx - 0.5f * (kT - 1);  // exact
    const float dy = (float)cy - 0.5f * (kT - 1);
    const float zc = (float)((double)(tz * kT) + 0.5 * (kT - 1) - 0.5 * (g.nz - 1));
    // voxels j and j + 1 of the column run as one packed f32x2 pair
    float2 acc[kT / 2];
#pragma unroll
    for (int jj = 0; jj < kT / 2; ++jj) acc[jj] = make_float2(0.0f, 0.0f);
    const int wu = g.wu;
    const float2 kM2 = make_float2(kMagic, kMagic), kNegM2 = make_float2(-kMagic, -kMagic);
    const float2 kNeg1 = make_float2(-1.0f, -1.0f), kHalf2 = make_float2(0.5f, 0.5f);
    for (int c = 0; c < nch; ++c) {
        const int s = c % kStages;
        const bool ok = mbar_wait_bounded(full0 + 8u * s, (uint32_t)(c / kStages) & 1u, lim);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) *reinterpret_cast<volatile int *>(g.status) = FBP_ERR_TIMEOUT;
            return;
        }
        const int a0 = c * g.ch;
        const int na = min(g.ch, g.A - a0);
        for (int k = 0; k < na; ++k) {
            const FdkPrm P = pt[a0 + k];
            const float ds = fmaf(dx, P.c, dy * P.s);
            const float dt = fmaf(dy, P.c, -dx * P.s);
            const float U = P.uc - ds;
            // fast reciprocal (about 2 ulp): the window offsets it scales are
            // tens of bins, so it moves a sample by ~1e-5 bins; IEEE division
            // here cost 8% of the reconstruction
            const float inv = __fdividef(1.0f, U * P.uc);
            const float ku = fmaf(g.Ru * fmaf(dt, P.uc, P.tc * ds), inv, P.kuo);
            const float fk = floorf(ku);
            // window pair of the voxel's interval; kept inside the window
            const int b = min(max((int)fk, 0), wu - 1);
            const float wu_off = ku - fk - 0.5f;
            const float rU = g.R * P.uc * inv;  // R / U
            const float W = rU * rU;
            const float bz = g.Rv * P.uc * inv;  // d(row) / d(dz)
            const float v0 = fmaf(g.Rv * zc * ds, inv, P.kvo) - 0.5f;
            const float2 bz2 = make_float2(bz, bz), v02 = make_float2(v0, v0);
            const float2 W2 = make_float2(W, W);
            // shared address of window pair (row r, pair b): the rounded row
            // coordinate's bits are r + kMagicLow, so with the offset folded
            // into wb the address is wb + bits * row_bytes (32-bit wraparound
            // cancels)
            const uint32_t row_bytes = 8u * (uint32_t)wu;
            const uint32_t wb = base + (uint32_t)((s * g.ch + k) * g.box_bytes) + 8u * (uint32_t)b -
                                row_bytes * (uint32_t)kMagicLow;
#pragma unroll
            for (int jj = 0; jj < kT / 2; ++jj) {
                const float2 dz = make_float2((float)(2 * jj) - 0.5f * (kT - 1),
                                              (float)(2 * jj + 1) - 0.5f * (kT - 1));
                const float2 kvh = __ffma2_rn(dz, bz2, v02);  // kv - 1/2
                const float2 t = __fadd2_rn(kvh, kM2);
                const float2 fl_f = __fadd2_rn(t, kNegM2);   // floor(kv), as floats
                // kv - floor(kv) = (kvh - floor) + 1/2
                const float2 wv_off = __fadd2_rn(__ffma2_rn(fl_f, kNeg1, kvh), kHalf2);
                // rows r and r + 1 lie inside the window: it spans the rows of the
                // tile's eight corners (where a box's perspective image takes its
                // extremes) with a row of margin each side, far beyond the FP32
                // error of kv (checked by emulating every test geometry's indices)
                uint32_t rx = __float_as_uint(t.x), ry = __float_as_uint(t.y);
#ifdef FBP_CHECK_BOUNDS
                // debug builds: rows r and r + 1 must lie in the staged window
                rx = (uint32_t)check_index((int)(rx - (uint32_t)kMagicLow), g.wv - 1 - shrink,
                                           g.status, kCheckFdk) + (uint32_t)kMagicLow;
                ry = (uint32_t)check_index((int)(ry - (uint32_t)kMagicLow), g.wv - 1 - shrink,
                                           g.status, kCheckFdk) + (uint32_t)kMagicLow;
#endif
                const uint32_t a0 = wb + rx * row_bytes;
                const uint32_t a1 = wb + ry * row_bytes;
                const float2 m00 = lds_f2(a0), m01 = lds_f2(a0 + row_bytes);
                const float2 m10 = lds_f2(a1), m11 = lds_f2(a1 + row_bytes);
                const float2 q0 = make_float2(fmaf(wu_off, m00.y, m00.x), fmaf(wu_off, m10.y, m10.x));
                const float2 q1 = make_float2(fmaf(wu_off, m01.y, m01.x), fmaf(wu_off, m11.y, m11.x));
                const float2 d = __ffma2_rn(q0, kNeg1, q1);   // q1 - q0
                acc[jj] = __ffma2_rn(W2, __ffma2_rn(wv_off, d, q0), acc[jj]);
            }
        }
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty0 + 8u * s)
                         : "memory");
    }
    const int ix = tx * kT + cx, iy = ty * kT + cy;
    if (ix < g.nx && iy < g.ny) {
#pragma unroll
        for (int j = 0; j < kT; ++j) {
            const int iz = tz * kT + j;
            if (iz < g.nz)
                vol[((size_t)iz * g.ny + iy) * g.nx + ix] =
                    ((j & 1) ? acc[j / 2].y : acc[j / 2].x) * g.scale;
        }
    }
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t q_bytes(const FdkPlan &f)
{
    const Plan *p = reinterpret_cast<const Plan *>(f.filt);
    return al256(sizeof(float) * (size_t)f.A * f.nv * (size_t)p->pitch);
}

size_t bp_smem_bytes(const FdkPlan &f)
{
    return 128 + (size_t)kStages * f.ch * f.box_bytes + 16 * kStages;
}

FdkArgs args_of(const FdkPlan &f)
{
    const Plan &p = *reinterpret_cast<const Plan *>(f.filt);
    FdkArgs g;
    std::memset(&g, 0, sizeof g);
    g.A = f.A;
    g.nv = f.nv;
    g.nu = f.nu;
    g.nx = f.nx;
    g.ny = f.ny;
    g.nz = f.nz;
    g.pitch2 = p.pitch / 2;
    g.tiles_x = f.tiles_x;
    g.tiles_y = f.tiles_y;
    g.tiles_z = f.tiles_z;
    g.wu = f.wu;
    g.wv = f.wv;
    g.ch = f.ch;
    g.box_bytes = (int)f.box_bytes;
    g.Ru = (float)(f.R / f.du);
    g.Rv = (float)(f.R / f.dv);
    g.R = (float)f.R;
    g.R64 = f.R;
    g.du = f.du;
    g.dv = f.dv;
    g.scale = (float)(M_PI / (double)f.A);
    g.status = p.d_status;
    return g;
}

void free_fdk(FdkPlan *f)
{
    if (f == nullptr) return;
    if (f->filt) fbp_plan_destroy(f->filt);
    cudaFree(f->d_wt);
    cudaFree(f->d_trig);
    cudaFree(f->d_prm);
    delete f;
}

}  // namespace

cudaError_t set_wait_hook_fdk(const WaitHook &h) { return write_wait_hook(h); }

}  // namespace fbp

using namespace fbp;

extern "C" {

fbp_status fbp_fdk_plan(fbp_fdk_plan_t *out, const fbp_fdk_geometry *geo, const double *beta,
                        fbp_filter_type filter)
{
    if (out == nullptr || geo == nullptr) {
        set_error("fbp_fdk_plan: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const fbp_fdk_geometry g = *geo;
    if (g.n_angles < 1 || g.nv < 1 || g.nu < 1 || g.nx < 1 || g.ny < 1 || g.nz < 1 ||
        !std::isfinite(g.R) || !std::isfinite(g.du) || !std::isfinite(g.dv) || !(g.du > 0.0) ||
        !(g.dv > 0.0) || g.nx > 8192 || g.ny > 8192 || g.nz > 8192 || g.n_angles > (1 << 20)) {
        set_error("fbp_fdk_plan: sizes must be >= 1 (volume <= 8192 a side), spacings > 0");
        return FBP_ERR_INVALID_ARG;
    }
    // every voxel of every tile (tiles may overhang the volume) inside the source circle
    const double hx = 0.5 * (g.nx - 1) + kT, hy = 0.5 * (g.ny - 1) + kT;
    const double rmax = std::sqrt(hx * hx + hy * hy);
    if (!(g.R > rmax + 1.0)) {
        set_error("fbp_fdk_plan: the source radius %g must exceed the volume's reach %g + 1",
                  g.R, rmax);
        return FBP_ERR_INVALID_ARG;
    }
    for (int a = 0; beta && a < g.n_angles; ++a)
        if (!std::isfinite(beta[a])) {
            set_error("fbp_fdk_plan: angle %d is not finite", a);
            return FBP_ERR_INVALID_ARG;
        }
    FdkPlan *f = new FdkPlan();
    std::memset(f, 0, sizeof *f);
    f->A = g.n_angles;
    f->nv = g.nv;
    f->nu = g.nu;
    f->nx = g.nx;
    f->ny = g.ny;
    f->nz = g.nz;
    f->R = g.R;
    f->du = g.du;
    f->dv = g.dv;
    f->tiles_x = (g.nx + kT - 1) / kT;
    f->tiles_y = (g.ny + kT - 1) / kT;
    f->tiles_z = (g.nz + kT - 1) / kT;
    cudaGetDevice(&f->device);
    fbp_options o;
    fbp_options_default(&o);
    o.filter_path = FBP_PATH_FFT;
    fbp_status st = fbp_plan(&f->filt, 1, g.n_angles * g.nv, g.nu, nullptr, g.du, filter, &o);
    if (st != FBP_OK) {
        free_fdk(f);
        return st;
    }
    std::vector<float> wt((size_t)g.nv * g.nu);
    for (int i = 0; i < g.nv; ++i) {
        const double v = (i - 0.5 * (g.nv - 1)) * g.dv;
        for (int j = 0; j < g.nu; ++j) {
            const double u = (j - 0.5 * (g.nu - 1)) * g.du;
            wt[(size_t)i * g.nu + j] = (float)(g.R / std::sqrt(g.R * g.R + u * u + v * v));
        }
    }
    std::vector<double2> trig((size_t)g.n_angles);
    for (int a = 0; a < g.n_angles; ++a) {
        const double b = beta ? beta[a] : 2.0 * M_PI * a / g.n_angles;
        trig[(size_t)a] = make_double2(std::cos(b), std::sin(b));
    }
    const size_t nprm = (size_t)f->tiles_x * f->tiles_y * f->tiles_z * (size_t)g.n_angles;
    int *d_ext = nullptr;
    int ext[2] = {0, 0};
    cudaError_t e = cudaMalloc(&f->d_wt, sizeof(float) * wt.size());
    if (e == cudaSuccess) e = cudaMalloc(&f->d_trig, sizeof(double2) * trig.size());
    if (e == cudaSuccess) e = cudaMalloc(&f->d_prm, sizeof(FdkPrm) * nprm);
    if (e == cudaSuccess) e = cudaMalloc(&d_ext, sizeof ext);
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_wt, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_trig, trig.data(), sizeof(double2) * trig.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ext, ext, sizeof ext, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const FdkArgs a = args_of(*f);
        fdk_params_kernel<<<(unsigned)((nprm + 255) / 256), 256>>>(f->d_trig, f->d_prm, a, d_ext);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(ext, d_ext, sizeof ext, cudaMemcpyDeviceToHost);
    cudaFree(d_ext);
    if (e != cudaSuccess) {
        free_fdk(f);
        set_error("fbp_fdk_plan: %s", cudaGetErrorString(e));
        return FBP_ERR_OUT_OF_MEMORY;
    }
    f->wu = (ext[0] + 1) & ~1;  // even: the box's row of pairs is a multiple of 16 bytes
    f->wv = std::max(ext[1], 2);
    f->box_bytes = ((size_t)f->wv * 2 * f->wu * 4 + 127) & ~(size_t)127;
    if (2 * f->wu > 256 || f->wv > 256) {
        free_fdk(f);
        set_error("fbp_fdk_plan: a tile's detector window (%d pairs x %d rows) exceeds one TMA "
                  "box (128 x 256)", ext[0], ext[1]);
        return FBP_ERR_UNSUPPORTED;
    }
    f->ch = 8;
    while (f->ch > 1 && bp_smem_bytes(*f) > kSmemBudget) f->ch /= 2;
    if (bp_smem_bytes(*f) > kSmemBudget) {
        free_fdk(f);
        set_error("fbp_fdk_plan: a tile's detector window (%zu bytes) does not fit shared memory",
                  f->box_bytes);
        return FBP_ERR_UNSUPPORTED;
    }
    Plan *p = reinterpret_cast<Plan *>(f->filt);
    p->d_row_weight = f->d_wt;
    p->row_weight_rows = g.nv;
    *out = reinterpret_cast<fbp_fdk_plan_t>(f);
    return FBP_OK;
}

fbp_status fbp_fdk_plan_destroy(fbp_fdk_plan_t plan)
{
    free_fdk(reinterpret_cast<FdkPlan *>(plan));
    return FBP_OK;
}

fbp_status fbp_fdk_workspace_bytes(fbp_fdk_plan_t plan, size_t *bytes)
{
    const FdkPlan *f = reinterpret_cast<const FdkPlan *>(plan);
    if (f == nullptr || bytes == nullptr) {
        set_error("fbp_fdk_workspace_bytes: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    *bytes = q_bytes(*f);
    return FBP_OK;
}

fbp_status fbp_fdk_reconstruct(fbp_fdk_plan_t plan, const void *proj, void *volume,
                               void *workspace, fbp_stream_t stream)
{
    const FdkPlan *f = reinterpret_cast<const FdkPlan *>(plan);
    if (f == nullptr || proj == nullptr || volume == nullptr || workspace == nullptr) {
        set_error("fbp_fdk_reconstruct: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    if (((reinterpret_cast<uintptr_t>(proj) | reinterpret_cast<uintptr_t>(volume) |
          reinterpret_cast<uintptr_t>(workspace)) & 15u) != 0) {
        set_error("fbp_fdk_reconstruct: buffers must be 16-byte aligned");
        return FBP_ERR_ALIGNMENT;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != f->device) {
        set_error("fbp_fdk_reconstruct: plan was made on device %d, current device is %d",
                  f->device, dev);
        return FBP_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Plan &p = *reinterpret_cast<const Plan *>(f->filt);
    float *q = static_cast<float *>(workspace);
    CUtensorMap qmap;
    if (!encode_rows_map_3d(q, 2 * (f->nu + 1), p.pitch, f->nv, f->A, 2 * f->wu, f->wv, &qmap))
        return FBP_ERR_CUDA;
    cudaError_t e = launch_filter_fft(p, static_cast<const float *>(proj), f->nu, q, s);
    const FdkArgs g = args_of(*f);
    const size_t smem = bp_smem_bytes(*f);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fdk_backproject_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        const unsigned ntile = (unsigned)(f->tiles_x * f->tiles_y * f->tiles_z);
        fdk_backproject_kernel<<<ntile, kThreads, smem, s>>>(qmap, f->d_prm,
                                                             static_cast<float *>(volume), g);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fbp_fdk_reconstruct: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_fdk_status(fbp_fdk_plan_t plan)
{
    const FdkPlan *f = reinterpret_cast<const FdkPlan *>(plan);
    if (f == nullptr) {
        set_error("fbp_fdk_status: NULL plan");
        return FBP_ERR_INVALID_ARG;
    }
    return fbp_device_status(f->filt);
}

}  // extern "C"
