// Image quality on the device: PSNR (Eq. 3) and SSIM (Eq. 4) of an image
// against a reference, the measures the paper compares its CPU and GPU
// reconstructions with.  The paper leaves PSNR's MAX and SSIM's constants and
// window open; this library takes MAX = max |reference| and the window and
// constants of Wang, Bovik, Sheikh & Simoncelli (2004): an 11 x 11 Gaussian
// window of standard deviation 1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2, the
// image SSIM being the mean over every window inside the image; L is the
// dynamic range (the reference's max - min unless the caller gives one).
//
// Four launches, all deterministic (every sum in a fixed order):
//   1. stats: grid-stride over the pixels; per block the FP64 sum of squared
//      differences (each difference of two floats formed exactly in FP64),
//      max |reference|, min and max of the reference;
//   2. consts: one thread turns the block results into L, C1, C2;
//   3. ssim: one CTA per 16 x 16 block of window positions; the (16+10)^2
//      patch's five FP64 maps x, y, x^2 + y^2, d = x - y and d^2 (products
//      and the difference of two floats are exact in FP64) are formed once
//      per pixel in shared memory; the Gaussian is separable
//      (w[a][b] = g[a] g[b]), so a horizontal then a vertical pass give their
//      local means.  Per window the
//      SSIM is formed through its distance from 1, which needs no
//      cancellation of large terms:
//        1 - l  = (E[d])^2 / (mu_x^2 + mu_y^2 + C1)            (l: luminance)
//        1 - cs = Var(d) / (sigma_x^2 + sigma_y^2 + C2)         (cs: the rest)
//        1 - SSIM = (1 - l) + (1 - cs) - (1 - l)(1 - cs)  (one fraction),
//      with Var(d) = E[d^2] - (E[d])^2 = sigma_x^2 + sigma_y^2 - 2 sigma_xy
//      (clamped at 0); so a pair of near-identical images keeps 1 - SSIM to
//      the precision of the differences, and SSIM never exceeds 1.  The CTA's
//      sum of (1 - SSIM) values in FP64;
//   4. finish: one CTA sums the partial results in order and writes
//      out[0] = PSNR (dB), out[1] = 1 - mean(1 - SSIM).
#include <cmath>
#include <cstring>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kWin = 11;           // SSIM window side
constexpr int kHalo = kWin - 1;    // extra rows/columns a tile reads
constexpr int kTile = 16;          // window positions per CTA side
constexpr int kPatch = kTile + kHalo;
constexpr int kStatBlocks = 256;   // CTAs of the stats pass
constexpr int kThreads = 256;

struct Gauss {
    double g[kWin];  // normalised 1-D Gaussian, sigma 1.5
};

// Scratch layout (offsets in bytes, each part 256-byte aligned).
struct QLayout {
    size_t se, maxabs, ymin, ymax, consts, ssim, total;
    int tiles_x, tiles_y;
};

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

QLayout q_layout(int rows, int cols)
{
    QLayout L;
    L.tiles_y = rows >= kWin ? (rows - kHalo + kTile - 1) / kTile : 0;
    L.tiles_x = cols >= kWin ? (cols - kHalo + kTile - 1) / kTile : 0;
    size_t o = 0;
    L.se = o;
    o = al(o + sizeof(double) * kStatBlocks);
    L.maxabs = o;
    o = al(o + sizeof(float) * kStatBlocks);
    L.ymin = o;
    o = al(o + sizeof(float) * kStatBlocks);
    L.ymax = o;
    o = al(o + sizeof(float) * kStatBlocks);
    L.consts = o;  // L, C1, C2 (double)
    o = al(o + sizeof(double) * 4);
    L.ssim = o;
    o = al(o + sizeof(double) * (size_t)(L.tiles_x > 0 ? L.tiles_x * L.tiles_y : 1));
    L.total = o;
    return L;
}

// Fixed-order tree reduction of one value per thread (blockDim = kThreads).
template <typename T, typename Op>
__device__ T block_reduce(T v, T *sh, Op op)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = op(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads)
    quality_stats_kernel(const float *__restrict__ x, const float *__restrict__ y, int rows,
                         int cols, int ld, unsigned char *scratch, QLayout L)
{
    __shared__ double shd[kThreads];
    __shared__ float shf[kThreads];
    const long n = (long)rows * cols;
    double se = 0.0;
    float mx = 0.0f, lo = INFINITY, hi = -INFINITY;
    for (long k = (long)blockIdx.x * kThreads + threadIdx.x; k < n;
         k += (long)gridDim.x * kThreads) {
        const long r = k / cols, c = k - r * cols;
        const float a = x[r * ld + c], b = y[r * ld + c];
        const double d = (double)a - (double)b;  // exact
        se += d * d;
        mx = fmaxf(mx, fabsf(b));
        lo = fminf(lo, b);
        hi = fmaxf(hi, b);
    }
    se = block_reduce(se, shd, [](double u, double v) { return u + v; });
    mx = block_reduce(mx, shf, [](float u, float v) { return fmaxf(u, v); });
    lo = block_reduce(lo, shf, [](float u, float v) { return fminf(u, v); });
    hi = block_reduce(hi, shf, [](float u, float v) { return fmaxf(u, v); });
    if (threadIdx.x == 0) {
        reinterpret_cast<double *>(scratch + L.se)[blockIdx.x] = se;
        reinterpret_cast<float *>(scratch + L.maxabs)[blockIdx.x] = mx;
        reinterpret_cast<float *>(scratch + L.ymin)[blockIdx.x] = lo;
        reinterpret_cast<float *>(scratch + L.ymax)[blockIdx.x] = hi;
    }
}

__global__ void quality_consts_kernel(unsigned char *scratch, QLayout L, double range)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!(range > 0.0)) {
        float lo = INFINITY, hi = -INFINITY;
        for (int b = 0; b < kStatBlocks; ++b) {
            lo = fminf(lo, reinterpret_cast<const float *>(scratch + L.ymin)[b]);
            hi = fmaxf(hi, reinterpret_cast<const float *>(scratch + L.ymax)[b]);
        }
        range = (double)hi - (double)lo;
    }
    double *c = reinterpret_cast<double *>(scratch + L.consts);
    c[0] = range;
    c[1] = (0.01 * range) * (0.01 * range);
    c[2] = (0.03 * range) * (0.03 * range);
}

__global__ void __launch_bounds__(kThreads)
    quality_ssim_kernel(const float *__restrict__ x, const float *__restrict__ y, int rows,
                        int cols, int ld, unsigned char *scratch, QLayout L, Gauss G)
{
    // the patch's five maps, each formed once per pixel in FP64: x, y,
    // x^2 + y^2, d = x - y, d^2 (the difference and products of two floats
    // are exact in FP64)
    __shared__ double mp[5][kPatch][kPatch + 1];
    // horizontal pass results: [map][patch row][tile column]
    __shared__ double hz[5][kPatch][kTile + 1];
    __shared__ double shd[kThreads];
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    for (int t = threadIdx.x; t < kPatch * kPatch; t += kThreads) {
        const int r = t / kPatch, c = t - r * kPatch;
        const int gr = i0 + r, gc = j0 + c;
        const bool in = gr < rows && gc < cols;
        const double a = in ? (double)x[(long)gr * ld + gc] : 0.0;
        const double v = in ? (double)y[(long)gr * ld + gc] : 0.0;
        const double d = a - v;  // exact
        mp[0][r][c] = a;
        mp[1][r][c] = v;
        mp[2][r][c] = fma(a, a, v * v);
        mp[3][r][c] = d;
        mp[4][r][c] = d * d;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPatch * kTile; t += kThreads) {
        const int r = t / kTile, c = t - r * kTile;
        double sx = 0.0, sy = 0.0, s2 = 0.0, sd = 0.0, sdd = 0.0;
#pragma unroll
        for (int b = 0; b < kWin; ++b) {
            const double w = G.g[b];
            sx = fma(w, mp[0][r][c + b], sx);
            sy = fma(w, mp[1][r][c + b], sy);
            s2 = fma(w, mp[2][r][c + b], s2);
            sd = fma(w, mp[3][r][c + b], sd);
            sdd = fma(w, mp[4][r][c + b], sdd);
        }
        hz[0][r][c] = sx;
        hz[1][r][c] = sy;
        hz[2][r][c] = s2;
        hz[3][r][c] = sd;
        hz[4][r][c] = sdd;
    }
    __syncthreads();
    const double *cst = reinterpret_cast<const double *>(scratch + L.consts);
    const double c1 = cst[1], c2 = cst[2];
    double acc = 0.0;
    for (int t = threadIdx.x; t < kTile * kTile; t += kThreads) {
        const int r = t / kTile, c = t - r * kTile;
        if (i0 + r + kWin > rows || j0 + c + kWin > cols) continue;  // window leaves the image
        double mx = 0.0, my = 0.0, e2 = 0.0, md = 0.0, edd = 0.0;
#pragma unroll
        for (int a = 0; a < kWin; ++a) {
            const double w = G.g[a];
            mx = fma(w, hz[0][r + a][c], mx);
            my = fma(w, hz[1][r + a][c], my);
            e2 = fma(w, hz[2][r + a][c], e2);
            md = fma(w, hz[3][r + a][c], md);
            edd = fma(w, hz[4][r + a][c], edd);
        }
        const double m2 = fma(mx, mx, my * my);
        const double vsum = e2 - m2;                      // sigma_x^2 + sigma_y^2
        const double vd = fmax(fma(-md, md, edd), 0.0);   // Var(x - y)
        // 1 - SSIM = (1 - l) + (1 - cs) - (1 - l)(1 - cs) with 1 - l = a / b and
        // 1 - cs = c / e, as one fraction (one division): every term of the
        // numerator is >= 0 but a c, which is below each of the others
        const double a = md * md, b = m2 + c1, e = vsum + c2;
        acc += (fma(a, e, vd * b) - a * vd) / (b * e);   // 1 - SSIM of this window
    }
    acc = block_reduce(acc, shd, [](double u, double v) { return u + v; });
    if (threadIdx.x == 0)
        reinterpret_cast<double *>(scratch + L.ssim)[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads)
    quality_finish_kernel(const unsigned char *scratch, QLayout L, int rows, int cols,
                          double *out)
{
    __shared__ double shd[kThreads];
    __shared__ float shf[kThreads];
    double se = 0.0;
    float mx = 0.0f;
    for (int b = threadIdx.x; b < kStatBlocks; b += kThreads) {
        se += reinterpret_cast<const double *>(scratch + L.se)[b];
        mx = fmaxf(mx, reinterpret_cast<const float *>(scratch + L.maxabs)[b]);
    }
    se = block_reduce(se, shd, [](double u, double v) { return u + v; });
    mx = block_reduce(mx, shf, [](float u, float v) { return fmaxf(u, v); });
    const int nt = L.tiles_x * L.tiles_y;
    double s = 0.0;
    for (int b = threadIdx.x; b < nt; b += kThreads)
        s += reinterpret_cast<const double *>(scratch + L.ssim)[b];
    s = block_reduce(s, shd, [](double u, double v) { return u + v; });
    if (threadIdx.x == 0) {
        const double mse = se / ((double)rows * (double)cols);
        out[0] = mse > 0.0 ? 20.0 * log10((double)mx / sqrt(mse)) : (double)INFINITY;
        const double windows = (double)(rows - kHalo) * (double)(cols - kHalo);
        out[1] = nt > 0 ? 1.0 - s / windows : (double)NAN;
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace fbp

using namespace fbp;

extern "C" {

fbp_status fbp_quality_scratch_bytes(int rows, int cols, size_t *bytes)
{
    if (bytes == nullptr || rows < 1 || cols < 1) {
        set_error("fbp_quality_scratch_bytes: rows and cols must be >= 1, bytes not NULL");
        return FBP_ERR_INVALID_ARG;
    }
    *bytes = q_layout(rows, cols).total;
    return FBP_OK;
}

fbp_status fbp_quality(const void *image, const void *reference, int rows, int cols, int ld,
                       double dynamic_range, void *scratch, size_t scratch_bytes, double *out,
                       fbp_stream_t stream)
{
    if (image == nullptr || reference == nullptr || scratch == nullptr || out == nullptr ||
        rows < 1 || cols < 1 || ld < cols || !std::isfinite(dynamic_range)) {
        set_error("fbp_quality: NULL buffer, rows/cols < 1, ld < cols or non-finite range");
        return FBP_ERR_INVALID_ARG;
    }
    if (!aligned16(image) || !aligned16(reference) || !aligned16(scratch) || !aligned16(out)) {
        set_error("fbp_quality: buffers must be 16-byte aligned");
        return FBP_ERR_ALIGNMENT;
    }
    const QLayout L = q_layout(rows, cols);
    if (scratch_bytes < L.total) {
        set_error("fbp_quality: scratch of %zu bytes, %zu needed", scratch_bytes, L.total);
        return FBP_ERR_INVALID_ARG;
    }
    Gauss G;
    double g[kWin], gs = 0.0;
    for (int a = 0; a < kWin; ++a) {
        const double d = (double)(a - kWin / 2);
        g[a] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        gs += g[a];
    }
    for (int a = 0; a < kWin; ++a) G.g[a] = g[a] / gs;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float *x = static_cast<const float *>(image);
    const float *y = static_cast<const float *>(reference);
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    quality_stats_kernel<<<kStatBlocks, kThreads, 0, s>>>(x, y, rows, cols, ld, sc, L);
    quality_consts_kernel<<<1, 32, 0, s>>>(sc, L, dynamic_range);
    if (L.tiles_x > 0 && L.tiles_y > 0)
        quality_ssim_kernel<<<dim3(L.tiles_x, L.tiles_y), kThreads, 0, s>>>(x, y, rows, cols, ld,
                                                                           sc, L, G);
    quality_finish_kernel<<<1, kThreads, 0, s>>>(sc, L, rows, cols, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("fbp_quality: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

}  // extern "C"
