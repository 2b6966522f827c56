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
//   2. per (tile, angle) parameters, FP64: the projection of the tile centre,
//      u_c = R t_c / U_c and v_c = R z_c / U_c with s_c = x_c cos b + y_c sin b,
//      t_c = -x_c sin b + y_c cos b, U_c = R - s_c, kept as an integer detector
//      base plus a small float offset;
//   3. backprojection, gather-only and deterministic: one CTA per 16 x 16 x 16
//      voxel tile, one thread per (x, y) column running down its 16 voxels.  A
//      voxel at (dx, dy, dz) from the centre projects to
//          u - u_c = R (dt U_c + t_c ds) / (U U_c),  v - v_c = R (dz U_c + z_c ds) / (U U_c)
//      (ds = dx cos b + dy sin b, dt = -dx sin b + dy cos b, U = U_c - ds), all
//      small offsets, so FP32 keeps the detector position to about 1e-6 bins;
//      the u sample and the weight (R/U)^2 are formed once per column and
//      angle, then each voxel reads two rows of pairs (bilinear) and adds in
//      angle order; the sum is scaled by pi / A (a full turn).
#include <cmath>
#include <cstring>
#include <vector>

#include "fbp_internal.h"

namespace fbp {

cudaError_t launch_filter_fft(const Plan &p, const float *sino, int ld, void *q, cudaStream_t s);

namespace {

constexpr int kT = 16;  // tile edge (voxels)

struct FdkPlan {
    int A, nv, nu, nx, ny, nz;
    double R, du, dv;
    int tiles_x, tiles_y, tiles_z;
    fbp_plan_t filt;   // FFT filter plan over the A nv rows
    float *d_wt;       // [nv][nu] cosine weights
    double2 *d_trig;   // (cos b, sin b)
    int device;
};

struct FdkPrm {
    float c, s, uc, tc;  // cos b, sin b, U_c, t_c
    float kuo, kvo;      // centre's detector column / row minus the integer bases
    int kub, kvb;        // integer bases (bin index, row index)
};

struct FdkArgs {
    int A, nv, nu, nx, ny, nz, pitch2, tiles_x, tiles_y, tiles_z;
    float Ru, Rv, R;  // R / du, R / dv, R
    double R64, du, dv;
    float scale;      // pi / A
};

__global__ void __launch_bounds__(256)
    fdk_params_kernel(const double2 *__restrict__ trig, FdkPrm *__restrict__ prm, FdkArgs g)
{
    const long ntile = (long)g.tiles_x * g.tiles_y * g.tiles_z;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntile * g.A) return;
    const long tile = idx / g.A;
    const int a = (int)(idx - tile * g.A);
    const int tx = (int)(tile % g.tiles_x);
    const int ty = (int)((tile / g.tiles_x) % g.tiles_y);
    const int tz = (int)(tile / ((long)g.tiles_x * g.tiles_y));
    const double xc = (double)(tx * kT) + 0.5 * (kT - 1) - 0.5 * (g.nx - 1);
    const double yc = (double)(ty * kT) + 0.5 * (kT - 1) - 0.5 * (g.ny - 1);
    const double zc = (double)(tz * kT) + 0.5 * (kT - 1) - 0.5 * (g.nz - 1);
    const double2 cs = trig[a];
    const double sc = xc * cs.x + yc * cs.y;
    const double tc = -xc * cs.y + yc * cs.x;
    const double Uc = g.R64 - sc;
    const double ku = g.R64 * tc / Uc / g.du + 0.5 * (g.nu - 1);
    const double kv = g.R64 * zc / Uc / g.dv + 0.5 * (g.nv - 1);
    const double fu = floor(ku), fv = floor(kv);
    FdkPrm P;
    P.c = (float)cs.x;
    P.s = (float)cs.y;
    P.uc = (float)Uc;
    P.tc = (float)tc;
    P.kuo = (float)(ku - fu);
    P.kvo = (float)(kv - fv);
    P.kub = (int)fu;
    P.kvb = (int)fv;
    prm[idx] = P;
}

// Pair (mid, slope) of bin `bin` of one detector row, interpolated at offset w
// in [-1/2, 1/2) from the bin's interval centre; zero outside the detector.
__device__ __forceinline__ float sample(const float2 *__restrict__ row, int pair, int npairs,
                                        float w)
{
    if (pair < 0 || pair >= npairs) return 0.0f;
    const float2 m = __ldg(&row[pair]);
    return fmaf(w, m.y, m.x);
}

__global__ void __launch_bounds__(kT * kT)
    fdk_backproject_kernel(const float2 *__restrict__ q, const FdkPrm *__restrict__ prm,
                           float *__restrict__ vol, FdkArgs g)
{
    const int tile = blockIdx.x;
    const int tx = tile % g.tiles_x;
    const int ty = (tile / g.tiles_x) % g.tiles_y;
    const int tz = tile / (g.tiles_x * g.tiles_y);
    const int cx = threadIdx.x % kT, cy = threadIdx.x / kT;
    const float dx = (float)cx - 0.5f * (kT - 1);  // exact
    const float dy = (float)cy - 0.5f * (kT - 1);
    const float zc = (float)((double)(tz * kT) + 0.5 * (kT - 1) - 0.5 * (g.nz - 1));
    float acc[kT];
#pragma unroll
    for (int j = 0; j < kT; ++j) acc[j] = 0.0f;
    const FdkPrm *pt = prm + (size_t)tile * g.A;
    const size_t plane = (size_t)g.nv * g.pitch2;
    for (int a = 0; a < g.A; ++a) {
        const FdkPrm P = pt[a];
        const float ds = fmaf(dx, P.c, dy * P.s);
        const float dt = fmaf(dy, P.c, -dx * P.s);
        const float U = P.uc - ds;
        const float inv = 1.0f / (U * P.uc);
        const float ku = fmaf(g.Ru * fmaf(dt, P.uc, P.tc * ds), inv, P.kuo);
        const float fk = floorf(ku);
        const int pair = P.kub + (int)fk + 1;  // pair of the interval [bin, bin + 1]
        const float wu = ku - fk - 0.5f;
        const float rU = g.R * P.uc * inv;     // R / U
        const float W = rU * rU;
        const float bz = g.Rv * P.uc * inv;    // d(row) / d(dz)
        const float v0 = fmaf(g.Rv * zc * ds, inv, P.kvo);
        const float2 *qa = q + (size_t)a * plane;
#pragma unroll
        for (int j = 0; j < kT; ++j) {
            const float kv = fmaf((float)j - 0.5f * (kT - 1), bz, v0);
            const float fv = floorf(kv);
            const int i = P.kvb + (int)fv;
            const float wv = kv - fv;
            const float r0 = (i >= 0 && i < g.nv)
                                 ? sample(qa + (size_t)i * g.pitch2, pair, g.pitch2, wu)
                                 : 0.0f;
            const float r1 = (i + 1 >= 0 && i + 1 < g.nv)
                                 ? sample(qa + (size_t)(i + 1) * g.pitch2, pair, g.pitch2, wu)
                                 : 0.0f;
            acc[j] = fmaf(W, fmaf(wv, r1 - r0, r0), acc[j]);
        }
    }
    const int ix = tx * kT + cx, iy = ty * kT + cy;
    if (ix < g.nx && iy < g.ny) {
#pragma unroll
        for (int j = 0; j < kT; ++j) {
            const int iz = tz * kT + j;
            if (iz < g.nz) vol[((size_t)iz * g.ny + iy) * g.nx + ix] = acc[j] * g.scale;
        }
    }
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t q_bytes(const FdkPlan &f)
{
    const Plan *p = reinterpret_cast<const Plan *>(f.filt);
    return al256(sizeof(float) * (size_t)f.A * f.nv * (size_t)p->pitch);
}

size_t prm_bytes(const FdkPlan &f)
{
    return al256(sizeof(FdkPrm) * (size_t)f.tiles_x * f.tiles_y * f.tiles_z * (size_t)f.A);
}

void free_fdk(FdkPlan *f)
{
    if (f == nullptr) return;
    if (f->filt) fbp_plan_destroy(f->filt);
    cudaFree(f->d_wt);
    cudaFree(f->d_trig);
    delete f;
}

}  // namespace
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
        !(g.dv > 0.0) || g.nx > 8192 || g.ny > 8192 || g.nz > 8192) {
        set_error("fbp_fdk_plan: sizes must be >= 1 (volume <= 8192 a side), spacings > 0");
        return FBP_ERR_INVALID_ARG;
    }
    const double rmax = std::sqrt(0.25 * (g.nx - 1.0) * (g.nx - 1.0) +
                                  0.25 * (g.ny - 1.0) * (g.ny - 1.0));
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
    cudaError_t e = cudaMalloc(&f->d_wt, sizeof(float) * wt.size());
    if (e == cudaSuccess) e = cudaMalloc(&f->d_trig, sizeof(double2) * trig.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_wt, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_trig, trig.data(), sizeof(double2) * trig.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_fdk(f);
        set_error("fbp_fdk_plan: %s", cudaGetErrorString(e));
        return FBP_ERR_OUT_OF_MEMORY;
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
    *bytes = q_bytes(*f) + prm_bytes(*f);
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
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Plan &p = *reinterpret_cast<const Plan *>(f->filt);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    float *q = reinterpret_cast<float *>(ws);
    FdkPrm *prm = reinterpret_cast<FdkPrm *>(ws + q_bytes(*f));
    cudaError_t e = launch_filter_fft(p, static_cast<const float *>(proj), f->nu, q, s);
    FdkArgs g;
    g.A = f->A;
    g.nv = f->nv;
    g.nu = f->nu;
    g.nx = f->nx;
    g.ny = f->ny;
    g.nz = f->nz;
    g.pitch2 = p.pitch / 2;
    g.tiles_x = f->tiles_x;
    g.tiles_y = f->tiles_y;
    g.tiles_z = f->tiles_z;
    g.Ru = (float)(f->R / f->du);
    g.Rv = (float)(f->R / f->dv);
    g.R = (float)f->R;
    g.R64 = f->R;
    g.du = f->du;
    g.dv = f->dv;
    g.scale = (float)(M_PI / (double)f->A);
    const long ntile = (long)f->tiles_x * f->tiles_y * f->tiles_z;
    if (e == cudaSuccess) {
        const long work = ntile * f->A;
        fdk_params_kernel<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(f->d_trig, prm, g);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        fdk_backproject_kernel<<<(unsigned)ntile, kT * kT, 0, s>>>(
            reinterpret_cast<const float2 *>(q), prm, static_cast<float *>(volume), g);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fbp_fdk_reconstruct: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

}  // extern "C"
