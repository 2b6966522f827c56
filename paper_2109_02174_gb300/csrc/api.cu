// C ABI of libfbp (include/fbp.h): argument checks, plan tables, dispatch.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "backproject.cuh"
#include "fbp_internal.h"
#include "filter_tc.cuh"
#include "ptx.cuh"

namespace fbp {

namespace {
thread_local std::string g_err;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fbp_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return FBP_ERR_CUDA;
}

// Common checks of every compute call: plan, device, pointers, alignment.
fbp_status check_call(const Plan *p, const char *fn, std::initializer_list<const void *> ptrs)
{
    if (p == nullptr) {
        set_error("%s: plan is NULL", fn);
        return FBP_ERR_INVALID_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
        set_error("%s: plan was made on device %d, current device is %d", fn, p->device, dev);
        return FBP_ERR_INVALID_ARG;
    }
    for (const void *q : ptrs) {
        if (q == nullptr) {
            set_error("%s: NULL buffer", fn);
            return FBP_ERR_INVALID_ARG;
        }
        if (!aligned16(q)) {
            set_error("%s: buffer %p is not 16-byte aligned", fn, q);
            return FBP_ERR_ALIGNMENT;
        }
    }
    return FBP_OK;
}

int round_up(int v, int m) { return ((v + m - 1) / m) * m; }

}  // namespace

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

bool encode_pairs_map(const Plan &p, const void *q, CUtensorMap *out)
{
    EncodeTiledFn enc = encode_fn();
    if (enc == nullptr) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    const int es = q_elem_bytes(p);
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * (p.D + 1)), (cuuint64_t)p.A};
    const cuuint64_t strides[1] = {(cuuint64_t)p.pitch * (cuuint64_t)es};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * p.bp_wp), 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt =
        es == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(out, dt, 2, const_cast<void *>(q), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return false;
    }
    return true;
}

bool encode_rows_map_3d(const void *q, int row_floats, int pitch, int rows, int planes,
                        int box_x, int box_y, CUtensorMap *out)
{
    EncodeTiledFn enc = encode_fn();
    if (enc == nullptr) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)row_floats, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4u, (cuuint64_t)pitch * 4u * (cuuint64_t)rows};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(q), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (3D rows) failed (%d)", (int)r);
        return false;
    }
    return true;
}

int tiles_of(const Plan &p)
{
    const int tx = 8 * p.bp_wx, ty = 32 * p.bp_wy;
    return ((p.n + tx - 1) / tx) * ((p.n + ty - 1) / ty);
}

// Backprojection work items of one slice: tiles, or tile pairs.
int items_of(const Plan &p) { return p.bp_point_pairs ? tiles_of(p) / 2 : tiles_of(p); }

BpSlice slice_desc(const Plan &p, float *image)
{
    BpSlice s;
    std::memset(&s, 0, sizeof s);
    s.trig64 = p.d_trig64;
    s.image = image;
    s.n = p.n;
    s.A = p.A;
    s.wp = p.bp_wp;
    s.tiles_x = (p.n + 8 * p.bp_wx - 1) / (8 * p.bp_wx);
    s.tiles = tiles_of(p);
    s.scale = p.scale32;
    s.half_n = 0.5 * (double)(p.n - 1);
    s.half_d = 0.5 * (double)(p.D - 1);
    return s;
}


BpConfig bp_config(const Plan &p)
{
    BpConfig c;
    c.wx = p.bp_wx;
    c.wy = p.bp_wy;
    c.chunk = p.bp_chunk;
    c.group = 1;
    c.half_pairs = p.q_storage == FBP_F16;
    c.kahan = p.accumulate == FBP_ACC_KAHAN;
    c.point_pairs = p.bp_point_pairs != 0;
    return c;
}

cudaError_t backproject_slice(const Plan &p, const void *q, float *image, cudaStream_t s)
{
    BpLaunch<1> L;
    std::memset(&L, 0, sizeof L);
    if (!encode_pairs_map(p, q, &L.maps[0])) return cudaErrorInvalidValue;
    L.slices[0] = slice_desc(p, image);
    L.n_slices = 1;
    L.n_items = items_of(p);
    L.tile_end[0] = L.n_items;
    L.wp_max = p.bp_wp;
    L.status = p.d_status;
    return launch_backproject(L, bp_config(p), s);
}

// Detector window (pairs) a tile of tx x ty pixels needs per angle: the tile's
// detector coordinates span ext = max_i (tx-1)|c_i| + (ty-1)|s_i| bins; the
// window starts one bin below floor(umin), aligned down to `align` pairs, and
// must hold the pair of round(u - base - 1/2) <= ext + align + 1.
int window_pairs(const std::vector<double2> &trig, int tx, int ty, int align)
{
    double ext = 0.0;
    for (const double2 &cs : trig)
        ext = std::fmax(ext, (tx - 1) * std::fabs(cs.x) + (ty - 1) * std::fabs(cs.y));
    const int wp = (int)std::ceil(ext + 1e-6) + align + 2;
    return ((wp + align - 1) / align) * align;
}


fbp_status take_device_status(int *d_status, const char *fn)
{
    int v[kStatusWords] = {0, 0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(v, d_status, sizeof v, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof v);
    if (e != cudaSuccess) {
        set_error("%s: %s", fn, cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    if (v[0] == FBP_ERR_BOUNDS) {
        set_error("device status %d: index check of a debug build: %s kernel index %d outside "
                  "[0, %d)", v[0], v[1] == 2 ? "FDK" : "backprojection", v[2], v[3]);
        return FBP_ERR_BOUNDS;
    }
    if (v[0] != 0) {
        set_error("device status %d: a bounded device wait ran out", v[0]);
        return (fbp_status)v[0];
    }
    return FBP_OK;
}

}  // namespace fbp

using namespace fbp;

namespace {

void free_plan(Plan *p)
{
    if (p == nullptr) return;
    if (p->tc) {
        cudaFree(p->tc->d_hi);
        cudaFree(p->tc->d_lo);
        delete p->tc;
    }
    cudaFree(p->d_trig64);
    cudaFree(p->d_taps32);
    cudaFree(p->d_taps64);
    cudaFree(p->d_fft_tw);
    cudaFree(p->d_fft_h);
    cudaFree(p->d_fft_tw64);
    cudaFree(p->d_trig_fx);
    cudaFree(p->d_fft_h64);
    cudaFree(p->d_status);
    delete p;
}

// Spatial taps tau*h(m), m = -(D-1)..D-1 (Kak & Slaney band-limited ramp kernels).
void make_taps(int kind, int D, double tau, std::vector<double> &out)
{
    out.assign((size_t)(2 * D - 1), 0.0);
    const double pi2 = M_PI * M_PI;
    for (int m = -(D - 1); m <= D - 1; ++m) {
        double h;
        if (kind == FBP_FILTER_RAM_LAK)
            h = (m == 0) ? 1.0 / (4.0 * tau * tau)
                         : ((m & 1) ? -1.0 / (pi2 * (double)m * (double)m * tau * tau) : 0.0);
        else if (kind == FBP_FILTER_SHEPP_LOGAN)
            h = 2.0 / (pi2 * tau * tau * (1.0 - 4.0 * (double)m * (double)m));
        else
            h = (m == 0) ? 1.0 / tau : 0.0;
        out[(size_t)(m + D - 1)] = tau * h;
    }
}

// T[n][k] = tau h(n - k), split into tf32 hi (round to nearest, ties away) and
// the remainder rounded the same way, rows n < D with stride kpad; plus their
// TMA maps.
bool make_tc_tables(const Plan &p, const std::vector<double> &taps, TcTables *t)
{
    const int D = p.D;
    t->kpad = round_up(D, 4);
    const size_t count = (size_t)D * (size_t)t->kpad;
    std::vector<float> hi(count, 0.0f), lo(count, 0.0f);
    for (int n = 0; n < D; ++n) {
        for (int k = 0; k < D; ++k) {
            const double v = taps[(size_t)(n - k + D - 1)];
            const float f = (float)v;
            uint32_t b;
            std::memcpy(&b, &f, 4);
            b = (b + 0x1000u) & 0xFFFFE000u;
            float h;
            std::memcpy(&h, &b, 4);
            hi[(size_t)n * t->kpad + k] = h;
            // the remainder, itself rounded to tf32 (to nearest, ties away)
            const float r = (float)(v - (double)h);
            uint32_t rb;
            std::memcpy(&rb, &r, 4);
            rb = (rb + 0x1000u) & 0xFFFFE000u;
            float rl;
            std::memcpy(&rl, &rb, 4);
            lo[(size_t)n * t->kpad + k] = rl;
        }
    }
    if (cudaMalloc(&t->d_hi, sizeof(float) * count) != cudaSuccess ||
        cudaMalloc(&t->d_lo, sizeof(float) * count) != cudaSuccess) {
        set_error("fbp_plan: cudaMalloc of the Toeplitz tables failed");
        return false;
    }
    if (cudaMemcpy(t->d_hi, hi.data(), sizeof(float) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(t->d_lo, lo.data(), sizeof(float) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        set_error("fbp_plan: upload of the Toeplitz tables failed");
        return false;
    }
    EncodeTiledFn enc = encode_fn();
    if (enc == nullptr) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)D};
    const cuuint64_t strides[1] = {(cuuint64_t)t->kpad * 4u};
    const cuuint32_t box[2] = {32u, 128u};
    const cuuint32_t estr[2] = {1u, 1u};
    for (int w = 0; w < 2; ++w) {
        CUresult r = enc(w ? &t->t_lo : &t->t_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         w ? t->d_lo : t->d_hi, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled (Toeplitz tables) failed (%d)", (int)r);
            return false;
        }
    }
    return true;
}

}  // namespace

extern "C" {

fbp_status fbp_options_default(fbp_options *opt)
{
    if (opt == nullptr) {
        set_error("fbp_options_default: NULL");
        return FBP_ERR_INVALID_ARG;
    }
    std::memset(opt, 0, sizeof *opt);
    opt->dtype = FBP_F32;
    opt->q_storage = FBP_F32;
    opt->accumulate = FBP_ACC_PLAIN;
    opt->filter_path = FBP_PATH_AUTO;
    return FBP_OK;
}

fbp_status fbp_plan(fbp_plan_t *out, int n_pix, int n_angles, int n_det, const double *angles,
                    double det_spacing, fbp_filter_type filter, const fbp_options *opt)
{
    if (out == nullptr) {
        set_error("fbp_plan: out is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n_pix < 1 || n_pix > 16384 || n_angles < 1 || n_angles > (1 << 24) || n_det < 1 ||
        n_det > 65535) {
        set_error("fbp_plan: sizes out of range (n_pix %d, n_angles %d, n_det %d)", n_pix,
                  n_angles, n_det);
        return FBP_ERR_INVALID_ARG;
    }
    if (!(det_spacing > 0.0) || !std::isfinite(det_spacing)) {
        set_error("fbp_plan: det_spacing must be finite and > 0");
        return FBP_ERR_INVALID_ARG;
    }
    if (filter != FBP_FILTER_RAM_LAK && filter != FBP_FILTER_SHEPP_LOGAN &&
        filter != FBP_FILTER_NONE) {
        set_error("fbp_plan: unknown filter %d", (int)filter);
        return FBP_ERR_INVALID_ARG;
    }
    fbp_options o;
    fbp_options_default(&o);
    if (opt != nullptr) o = *opt;
    if (o.dtype != FBP_F32 && o.dtype != FBP_F64) {
        set_error("fbp_plan: dtype %d not built", o.dtype);
        return FBP_ERR_UNSUPPORTED;
    }
    if (!std::isfinite(o.i0) || o.i0 < 0.0) {
        set_error("fbp_plan: i0 must be 0 (line integrals) or a positive incident intensity");
        return FBP_ERR_INVALID_ARG;
    }
    if (o.dtype == FBP_F64) {
        // The FP64 path: an FFT or direct filter and a per-pixel backprojection.
        if (o.q_storage != FBP_F32 || o.accumulate != FBP_ACC_PLAIN ||
            o.filter_path == FBP_PATH_TOEPLITZ_TC) {
            set_error("fbp_plan: FP64 plans take the default q_storage/accumulate and the "
                      "FFT or direct filter");
            return FBP_ERR_UNSUPPORTED;
        }
    }
    if ((o.q_storage != FBP_F32 && o.q_storage != FBP_F16) ||
        (o.accumulate != FBP_ACC_PLAIN && o.accumulate != FBP_ACC_KAHAN)) {
        set_error("fbp_plan: q_storage %d / accumulate %d not built", o.q_storage, o.accumulate);
        return FBP_ERR_UNSUPPORTED;
    }
    if (o.filter_path != FBP_PATH_AUTO && o.filter_path != FBP_PATH_DIRECT &&
        o.filter_path != FBP_PATH_FFT && o.filter_path != FBP_PATH_TOEPLITZ_TC) {
        set_error("fbp_plan: filter path %d not built", o.filter_path);
        return FBP_ERR_UNSUPPORTED;
    }
    if (o.filter_path == FBP_PATH_TOEPLITZ_TC &&
        (o.dtype != FBP_F32 || o.q_storage != FBP_F32)) {
        set_error("fbp_plan: the tensor-core filter writes FP32 pairs of FP32 plans");
        return FBP_ERR_UNSUPPORTED;
    }
    // FFT length: any power of two >= 2*n_det - 1 gives the linear convolution.
    int fft_len = o.fft_len;
    if (fft_len == 0) {
        fft_len = 16;
        while (fft_len < 2 * n_det - 1) fft_len <<= 1;
    } else if (fft_len < 2 * n_det - 1 || (fft_len & (fft_len - 1)) != 0) {
        set_error("fbp_plan: fft_len %d must be a power of two >= 2*n_det-1 = %d", fft_len,
                  2 * n_det - 1);
        return FBP_ERR_INVALID_ARG;
    }
    const int max_fft = o.dtype == FBP_F64 ? kMaxFftLen64 : kMaxFftLen;
    const bool fft_ok = fft_len <= max_fft;
    int path = o.filter_path;
    if (path == FBP_PATH_AUTO) path = fft_ok ? FBP_PATH_FFT : FBP_PATH_DIRECT;
    if (path == FBP_PATH_FFT && !fft_ok) {
        set_error("fbp_plan: FFT length %d exceeds %d", fft_len, max_fft);
        return FBP_ERR_UNSUPPORTED;
    }
    if (path == FBP_PATH_DIRECT &&
        (o.dtype == FBP_F64 ? filter_direct_f64_smem_bytes(n_det)
                            : filter_direct_smem_bytes(n_det)) > 200 * 1024) {
        set_error("fbp_plan: n_det %d too large for the direct filter", n_det);
        return FBP_ERR_UNSUPPORTED;
    }
    std::vector<double> theta((size_t)n_angles);
    for (int i = 0; i < n_angles; ++i) {
        theta[(size_t)i] = angles ? angles[i] : (double)i * (M_PI / (double)n_angles);
        if (!std::isfinite(theta[(size_t)i])) {
            set_error("fbp_plan: angle %d is not finite", i);
            return FBP_ERR_INVALID_ARG;
        }
    }

    Plan *p = new Plan();
    std::memset(p, 0, sizeof *p);
    p->n = n_pix;
    p->A = n_angles;
    p->D = n_det;
    p->pitch = round_up(2 * (n_det + 1), 8);
    p->filter = (int)filter;
    p->dtype = o.dtype;
    p->q_storage = o.q_storage;
    p->accumulate = o.accumulate;
    p->filter_path = path;
    p->fft_len = (path == FBP_PATH_FFT) ? fft_len : 0;
    p->tau = det_spacing;
    p->i0 = o.i0;
    p->i0f = (float)o.i0;
    p->ln_i0f = o.i0 > 0.0 ? (float)std::log(o.i0) : 0.0f;
    p->scale64 = M_PI / (double)n_angles;
    p->scale32 = (float)p->scale64;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        set_error("fbp_plan: no CUDA device");
        return FBP_ERR_CUDA;
    }

    std::vector<double2> trig((size_t)n_angles);
    for (int i = 0; i < n_angles; ++i)
        trig[(size_t)i] = make_double2(std::cos(theta[(size_t)i]) / det_spacing,
                                       std::sin(theta[(size_t)i]) / det_spacing);
    // Backprojection tile: the largest of 32x64, 32x32, 8x32 pixels whose
    // detector window fits one TMA box (256 elements = 128 pairs) and that
    // cuts the image into at least one tile per two SMs (else the smallest
    // that fits), unless the options name one of them or ask (-1) for the
    // largest that fits (for batches and serving waves, where several slices
    // fill the SMs and the largest tile costs least per pixel).  A tile alone on an SM
    // runs up to twice as fast as two sharing one, so a single slice loses
    // nothing while at most half the SMs idle, and smaller tiles cost more per
    // pixel (8x32 about 1.7x 32x64 on a full GPU).  One slice, microseconds,
    // 32x64 / 32x32 / 8x32: 256^2 x 180: 31.4 / 29.3 / 27.4; 256^2 x 720:
    // 77.4 / 65.2 / 61.1; 384^2 x 360: 49.8 / 43.7 / 48.8; 512^2 x 720:
    // 79.5 / 82.6 / 134.8; 1024^2 x 1440: 482 / 504 / 832.
    const int align = (o.q_storage == FBP_F16) ? 4 : 2;
    const int shapes[3][2] = {{4, 2}, {4, 1}, {1, 1}};
    int sms = 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const bool largest = o.tile_x < 0 || o.tile_y < 0;
    int pick = -1;
    for (int k = 0; k < 3; ++k) {
        const int tx = 8 * shapes[k][0], ty = 32 * shapes[k][1];
        if (!largest && (o.tile_x || o.tile_y) && (o.tile_x != tx || o.tile_y != ty)) continue;
        if (window_pairs(trig, tx, ty, align) > 128) continue;
        pick = k;
        if (largest) break;
        const long tiles = (long)((n_pix + tx - 1) / tx) * (long)((n_pix + ty - 1) / ty);
        if (2 * tiles >= (long)sms) break;
    }
    if (pick < 0 && o.dtype == FBP_F64) pick = 0;  // the FP64 path has no tiles
    // Point-symmetric tile pairs (see below) on the automatic tile: the
    // tiling must map onto itself under the reflection through the image
    // centre (n a multiple of both tile sides, the grid not odd in both
    // directions) and the sum be plain.  Auto (option 0) takes them, on 32 x 32
    // tiles, for a slice of at least 7/4 tiles of 32 x 64 per SM; one slice,
    // microseconds, without / with pairs: 512^2 x 720 at 32 x 32: 72.3 / 84.6;
    // 768^2 x 1440 at 32 x 64: 240 / 214, at 32 x 32: 249 / 216;
    // 1024^2 x 1440: 469 / 418, 484 / 425; 1536^2 x 1024: 664 / 591,
    // 687 / 570; 2048^2 x 2048: 2293 / 2040, 2380 / 1934.  FP16 pairs keep
    // 32 x 64 with point pairs where that tiling allows them (2048^2 x 2048,
    // backprojection alone: 1.868 ms on 32 x 64, 1.982 on 32 x 32; FP32 pairs
    // 2.039 and 1.932).
    auto pairs_fit = [&](int tx, int ty) {
        const int gx = n_pix / tx, gy = n_pix / ty;
        return o.dtype == FBP_F32 &&
               (o.accumulate == FBP_ACC_PLAIN || o.q_storage != FBP_F16) && n_pix % tx == 0 &&
               n_pix % ty == 0 && !((gx & 1) && (gy & 1));
    };
    const long tiles_big = (long)((n_pix + 31) / 32) * (long)((n_pix + 63) / 64);
    const bool pairs_auto = o.point_pairs == 0 && 4 * tiles_big >= 7L * sms;
    if (pick >= 0 && !largest && !o.tile_x && !o.tile_y && o.point_pairs >= 0 &&
        (pairs_auto || o.point_pairs > 0)) {
        const bool keep_wide = o.q_storage == FBP_F16 && pick == 0 && pairs_fit(32, 64);
        if (!keep_wide && pairs_fit(32, 32) && window_pairs(trig, 32, 32, align) <= 128)
            pick = 1;  // 32 x 32
    }
    if (pick < 0) {
        delete p;
        set_error("fbp_plan: no backprojection tile fits the detector window (det_spacing %.3g, "
                  "tile %dx%d requested)", det_spacing, o.tile_x, o.tile_y);
        return FBP_ERR_UNSUPPORTED;
    }
    p->bp_wx = shapes[pick][0];
    p->bp_wy = shapes[pick][1];
    p->bp_wp = window_pairs(trig, 8 * p->bp_wx, 32 * p->bp_wy, align);
    if (o.angle_chunk != 0 && o.angle_chunk != 8 && o.angle_chunk != 16 && o.angle_chunk != 32) {
        delete p;
        set_error("fbp_plan: angle_chunk %d is not 8, 16 or 32", o.angle_chunk);
        return FBP_ERR_INVALID_ARG;
    }
    // 32 angles per stage unless set: the tuner's choice in 29 of 30 tunings of
    // the 15 shapes of the uneven 64-slice batch (each for its own count and for
    // a batch of 64); one stage barrier per 32 angles
    p->bp_chunk = o.angle_chunk ? o.angle_chunk : 32;
    // Point-symmetric tile pairs: explicit (option 1) wherever the tiling
    // allows; automatic only with the automatic tile (tuned, batch and serving
    // plans name their tile and keep single-tile items unless asked).
    if (o.point_pairs < -1 || o.point_pairs > 1) {
        delete p;
        set_error("fbp_plan: point_pairs %d is not -1, 0 or 1", o.point_pairs);
        return FBP_ERR_INVALID_ARG;
    }
    {
        const bool can = pairs_fit(8 * p->bp_wx, 32 * p->bp_wy);
        const bool want = o.point_pairs > 0 ||
                          (pairs_auto && !largest && !o.tile_x && !o.tile_y);
        p->bp_point_pairs = (can && want) ? 1 : 0;
    }

    std::vector<double> taps;
    make_taps((int)filter, n_det, det_spacing, taps);
    std::vector<float> taps32(taps.size());
    for (size_t m = 0; m < taps.size(); ++m) taps32[m] = (float)taps[m];

    cudaError_t e = cudaMalloc(&p->d_trig64, sizeof(double2) * trig.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_taps32, sizeof(float) * taps32.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_taps64, sizeof(double) * taps.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int) * kStatusWords);
    if (e != cudaSuccess) {
        free_plan(p);
        set_error("fbp_plan: cudaMalloc: %s", cudaGetErrorString(e));
        return FBP_ERR_OUT_OF_MEMORY;
    }
    e = cudaMemcpy(p->d_trig64, trig.data(), sizeof(double2) * trig.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_taps32, taps32.data(), sizeof(float) * taps32.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->dtype == FBP_F64) {
        // Fixed-point detector coordinate of the FP64 backprojection: S fraction
        // bits, as many as keep |u| 2^S (with a margin of a partial block of
        // pixels beyond the image) below 2^62, at most 48.
        double cmax = 0.0, smax = 0.0;
        for (const double2 &t : trig) {
            cmax = std::max(cmax, std::fabs(t.x));
            smax = std::max(smax, std::fabs(t.y));
        }
        const double half = 0.5 * (double)(n_pix - 1) + 16.0;
        const double bound = half * (cmax + smax) + 0.5 * (double)(n_det - 1) + 1.0;
        int b = 0;
        while (std::ldexp(1.0, b) <= bound) ++b;
        p->fx_shift = std::min(48, 62 - b);
        if (p->fx_shift < 24) {
            free_plan(p);
            set_error("fbp_plan: detector coordinates up to %.3g bins are beyond the FP64 "
                      "path's fixed-point range", bound);
            return FBP_ERR_UNSUPPORTED;
        }
        const double unit = std::ldexp(1.0, p->fx_shift - 1);
        std::vector<longlong2> fx(trig.size());
        for (size_t i = 0; i < trig.size(); ++i)
            fx[i] = make_longlong2(std::llround(trig[i].x * unit), std::llround(trig[i].y * unit));
        p->half_d_fx = std::llround(0.5 * (double)(n_det - 1) * std::ldexp(1.0, p->fx_shift));
        e = cudaMalloc(&p->d_trig_fx, sizeof(longlong2) * fx.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_trig_fx, fx.data(), sizeof(longlong2) * fx.size(),
                           cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_taps64, taps.data(), sizeof(double) * taps.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->filter_path == FBP_PATH_FFT) {
        const int N = p->fft_len;
        std::vector<double> ct((size_t)N), st((size_t)N);
        for (int t = 0; t < N; ++t) {
            const double a = 2.0 * M_PI * (double)t / (double)N;
            ct[(size_t)t] = std::cos(a);
            st[(size_t)t] = std::sin(a);
        }
        // H[f] = sum_m tau h(m) e^{-2 pi i f m / N} = tau h(0) + 2 sum_{m>0} tau h(m) cos(2 pi f m / N)
        std::vector<double> hs((size_t)N);
        for (int f = 0; f < N; ++f) {
            double acc = taps[(size_t)(n_det - 1)];
            for (int m = 1; m < n_det; ++m)
                acc += 2.0 * taps[(size_t)(n_det - 1 + m)] * ct[(size_t)(((long)f * m) % N)];
            hs[(size_t)f] = acc / (double)N;
        }
        if (p->dtype == FBP_F64) {
            std::vector<double2> tw((size_t)N);
            for (int t = 0; t < N; ++t) tw[(size_t)t] = make_double2(ct[(size_t)t], -st[(size_t)t]);
            e = cudaMalloc(&p->d_fft_tw64, sizeof(double2) * (size_t)N);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_fft_h64, sizeof(double) * (size_t)N);
            if (e == cudaSuccess)
                e = cudaMemcpy(p->d_fft_tw64, tw.data(), sizeof(double2) * (size_t)N,
                               cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(p->d_fft_h64, hs.data(), sizeof(double) * (size_t)N,
                               cudaMemcpyHostToDevice);
        } else {
            // twiddles and spectrum stored twice over (one copy per transform of a
            // packed pair): tw[t] = (c, c, s, s), h[f] = (H, H)
            std::vector<float4> tw((size_t)N);
            std::vector<float2> h2((size_t)N);
            for (int t = 0; t < N; ++t) {
                const float c = (float)ct[(size_t)t], sn = (float)-st[(size_t)t];
                tw[(size_t)t] = make_float4(c, c, sn, sn);
                const float hv = (float)hs[(size_t)t];
                h2[(size_t)t] = make_float2(hv, hv);
            }
            e = cudaMalloc(&p->d_fft_tw, sizeof(float4) * (size_t)N);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_fft_h, sizeof(float2) * (size_t)N);
            if (e == cudaSuccess)
                e = cudaMemcpy(p->d_fft_tw, tw.data(), sizeof(float4) * (size_t)N,
                               cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(p->d_fft_h, h2.data(), sizeof(float2) * (size_t)N,
                               cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess && p->filter_path == FBP_PATH_TOEPLITZ_TC) {
        p->tc = new TcTables();
        std::memset(p->tc, 0, sizeof(TcTables));
        e = make_tc_tables(*p, taps, p->tc) ? cudaSuccess : cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int) * kStatusWords);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "fbp_plan: table upload");
    }
    // Load (CUDA loads modules lazily) the kernels of the plan's single-slice
    // path now, so that fbp_filter, fbp_backproject, fbp_reconstruct and
    // fbp_reconstruct_static load no code and allocate nothing when called.
    if (p->dtype == FBP_F64) {
        e = prepare_fp64(*p);
    } else {
        if (p->filter_path == FBP_PATH_FFT) e = prepare_filter_fft(*p);
        else if (p->filter_path == FBP_PATH_TOEPLITZ_TC) e = prepare_filter_tc(*p);
        else e = prepare_filter_direct(*p);
        if (e == cudaSuccess) e = prepare_backproject(*p);
    }
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "fbp_plan: kernel preparation");
    }
    static_scratch_setup(p->device);
    *out = reinterpret_cast<fbp_plan_t>(p);
    return FBP_OK;
}

fbp_status fbp_plan_destroy(fbp_plan_t plan)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (p == nullptr) return FBP_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return FBP_OK;
}

fbp_status fbp_workspace_bytes(fbp_plan_t plan, size_t *bytes)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (p == nullptr || bytes == nullptr) {
        set_error("fbp_workspace_bytes: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    *bytes = (size_t)p->A * (size_t)p->pitch * (size_t)q_elem_bytes(*p);
    return FBP_OK;
}

fbp_status fbp_plan_query(fbp_plan_t plan, int *q_pitch, int *fft_len, int *filter_path)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (p == nullptr) {
        set_error("fbp_plan_query: plan is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    if (q_pitch) *q_pitch = p->pitch;
    if (fft_len) *fft_len = p->fft_len;
    if (filter_path) *filter_path = p->filter_path;
    return FBP_OK;
}

fbp_status fbp_filter(fbp_plan_t plan, const void *sino, int ld_sino, void *filtered,
                      fbp_stream_t stream)
{
    NvtxRange range("fbp_filter");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    fbp_status st = check_call(p, "fbp_filter", {sino, filtered});
    if (st != FBP_OK) return st;
    if (ld_sino < p->D) {
        set_error("fbp_filter: ld_sino %d < n_det %d", ld_sino, p->D);
        return FBP_ERR_INVALID_ARG;
    }
    cudaError_t e;
    if (p->dtype == FBP_F64 && p->filter_path == FBP_PATH_FFT)
        e = launch_filter_fft_f64(*p, static_cast<const double *>(sino), ld_sino,
                                  static_cast<double *>(filtered), stream);
    else if (p->dtype == FBP_F64)
        e = launch_filter_direct_f64(*p, static_cast<const double *>(sino), ld_sino,
                                     static_cast<double *>(filtered), stream);
    else if (p->filter_path == FBP_PATH_FFT)
        e = launch_filter_fft(*p, static_cast<const float *>(sino), ld_sino, filtered, stream);
    else if (p->filter_path == FBP_PATH_TOEPLITZ_TC)
        e = launch_filter_tc(*p, static_cast<const float *>(sino), ld_sino,
                             static_cast<float *>(filtered), stream);
    else
        e = launch_filter_direct(*p, static_cast<const float *>(sino), ld_sino, filtered, stream);
    return e == cudaSuccess ? FBP_OK : cuda_fail(e, "fbp_filter");
}

fbp_status fbp_backproject(fbp_plan_t plan, const void *filtered, void *image,
                           fbp_stream_t stream)
{
    NvtxRange range("fbp_backproject");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    fbp_status st = check_call(p, "fbp_backproject", {filtered, image});
    if (st != FBP_OK) return st;
    if (p->dtype == FBP_F64) {
        cudaError_t e = launch_backproject_f64(*p, static_cast<const double *>(filtered),
                                               static_cast<double *>(image), stream);
        return e == cudaSuccess ? FBP_OK : cuda_fail(e, "fbp_backproject");
    }
    cudaError_t e = backproject_slice(*p, filtered, static_cast<float *>(image), stream);
    if (e == cudaErrorInvalidValue) return FBP_ERR_CUDA;  // tensor map encoding (message set)
    return e == cudaSuccess ? FBP_OK : cuda_fail(e, "fbp_backproject");
}

fbp_status fbp_reconstruct(fbp_plan_t plan, const void *sino, int ld_sino, void *image,
                           void *workspace, fbp_stream_t stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    fbp_status st = check_call(p, "fbp_reconstruct", {sino, image, workspace});
    if (st != FBP_OK) return st;
    st = fbp_filter(plan, sino, ld_sino, workspace, stream);
    if (st != FBP_OK) return st;
    return fbp_backproject(plan, workspace, image, stream);
}

fbp_status radon_forward(fbp_plan_t plan, const void *image, void *sino, fbp_stream_t stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    fbp_status st = check_call(p, "radon_forward", {image, sino});
    if (st != FBP_OK) return st;
    if (p->dtype != FBP_F32) {
        set_error("radon_forward: FP32 plans only");
        return FBP_ERR_UNSUPPORTED;
    }
    cudaError_t e = launch_radon_forward_f32(*p, static_cast<const float *>(image),
                                             static_cast<float *>(sino), stream);
    return e == cudaSuccess ? FBP_OK : cuda_fail(e, "radon_forward");
}

fbp_status fbp_device_status(fbp_plan_t plan)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    fbp_status st = check_call(p, "fbp_device_status", {});
    if (st != FBP_OK) return st;
    return take_device_status(p->d_status, "fbp_device_status");
}

const char *fbp_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// Host copies of the wait settings per device (written whole to every
// translation unit's device copy on each change).
constexpr int kHookDevices = 64;
std::mutex g_hook_mu;
fbp::WaitHook g_hooks[kHookDevices];

fbp_status push_hook(const char *fn, int dev)
{
    cudaError_t e = set_wait_hook_backproject(g_hooks[dev]);
    if (e == cudaSuccess) e = set_wait_hook_filter_tc(g_hooks[dev]);
    if (e == cudaSuccess) e = set_wait_hook_fdk(g_hooks[dev]);
    return e == cudaSuccess ? FBP_OK : cuda_fail(e, fn);
}

fbp_status hook_device(const char *fn, int *dev)
{
    if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= kHookDevices) {
        set_error("%s: no usable current CUDA device", fn);
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

}  // namespace

extern "C" {

fbp_status fbp_set_wait_limit(double seconds)
{
    if (!std::isfinite(seconds) || seconds < 0.0 || (seconds > 0.0 && seconds < 1e-6) ||
        seconds > 3600.0) {
        set_error("fbp_set_wait_limit: %g s is not 0 (default) or in [1e-6, 3600]", seconds);
        return FBP_ERR_INVALID_ARG;
    }
    int dev = -1;
    fbp_status st = hook_device("fbp_set_wait_limit", &dev);
    if (st != FBP_OK) return st;
    std::lock_guard<std::mutex> lock(g_hook_mu);
    g_hooks[dev].limit_ns = (unsigned long long)std::llround(seconds * 1e9);
    return push_hook("fbp_set_wait_limit", dev);
}

fbp_status fbp_test_withhold_arrival(int kernel, int stage)
{
    if (kernel != FBP_TEST_WITHHOLD_NONE && kernel != FBP_TEST_WITHHOLD_BACKPROJECT &&
        kernel != FBP_TEST_WITHHOLD_FILTER_TC) {
        set_error("fbp_test_withhold_arrival: unknown kernel kind %d", kernel);
        return FBP_ERR_INVALID_ARG;
    }
    if (kernel != FBP_TEST_WITHHOLD_NONE && stage < 0) {
        set_error("fbp_test_withhold_arrival: stage %d < 0", stage);
        return FBP_ERR_INVALID_ARG;
    }
    int dev = -1;
    fbp_status st = hook_device("fbp_test_withhold_arrival", &dev);
    if (st != FBP_OK) return st;
    std::lock_guard<std::mutex> lock(g_hook_mu);
    g_hooks[dev].kind = kernel == FBP_TEST_WITHHOLD_BACKPROJECT ? kWithholdBackproject
                        : kernel == FBP_TEST_WITHHOLD_FILTER_TC ? kWithholdFilterTc
                                                                : kWithholdNone;
    g_hooks[dev].stage = kernel == FBP_TEST_WITHHOLD_NONE ? -1 : stage;
    return push_hook("fbp_test_withhold_arrival", dev);
}

fbp_status fbp_test_shrink_window(int pairs)
{
    if (pairs < 0 || pairs > 4096) {
        set_error("fbp_test_shrink_window: %d is not in [0, 4096]", pairs);
        return FBP_ERR_INVALID_ARG;
    }
    int dev = -1;
    fbp_status st = hook_device("fbp_test_shrink_window", &dev);
    if (st != FBP_OK) return st;
    std::lock_guard<std::mutex> lock(g_hook_mu);
    g_hooks[dev].shrink = pairs;
    return push_hook("fbp_test_shrink_window", dev);
}

}  // extern "C"
