// FP64 variant of the whole path, for the paper's float-vs-double comparison
// (section "Results and discussion", double data type).  Same operator as the
// FP32 path: the ramp-filter convolution (the text after Eq. 2) written as
// (mid, slope) pairs of doubles, then Eq. 2 per pixel with linear
// interpolation, angles summed in order.  Plain CUDA-core code: GB300's FP64
// rate is a small fraction of its FP32 rate, so the kernels count FP64
// operations: the filter goes through an FP64 FFT (about 80 operations per
// bin instead of the direct convolution's 2 D), and the backprojection keeps
// the detector coordinate in 64-bit fixed point on the integer pipes and
// spends two FP64 operations per update (lerp, sum).  FP64 pairs are
// (a_k, d_k) = (2 Q[k] - Q[k+1], Q[k+1] - Q[k]) for bins k = -1 .. D-1, so
// the interpolant on [k, k+1] at fraction f is the single FMA a_k + (1 + f) d_k.
#include "fbp_internal.h"
#include "lambert.cuh"

namespace fbp {
namespace {

__global__ void __launch_bounds__(256)
    filter_direct_f64_kernel(const double *__restrict__ sino, int ld,
                             const double *__restrict__ taps, double *__restrict__ q, int D,
                             int pitch, double i0)
{
    extern __shared__ double smd[];
    double *st = smd;                // taps tau*h(m), index m + D - 1
    double *sp = smd + (2 * D - 1);  // the row
    double *sq = sp + D;             // sq[k + 1] = Q[k], sq[0] = sq[D + 1] = 0
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < 2 * D - 1; t += blockDim.x) st[t] = taps[t];
    for (int t = threadIdx.x; t < D; t += blockDim.x)
        sp[t] = line_integral(sino[(size_t)i * ld + t], i0);
    if (threadIdx.x == 0) {
        sq[0] = 0.0;
        sq[D + 1] = 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        const double *hk = st + k + D - 1;
        double acc = 0.0;
        for (int j = 0; j < D; ++j) acc = fma(hk[-j], sp[j], acc);
        sq[k + 1] = acc;
    }
    __syncthreads();
    double2 *row = reinterpret_cast<double2 *>(q + (size_t)i * pitch);
    for (int p = threadIdx.x; p < pitch / 2; p += blockDim.x) {
        if (p <= D)
            row[p] = make_double2(2.0 * sq[p] - sq[p + 1], sq[p + 1] - sq[p]);
        else
            row[p] = make_double2(0.0, 0.0);
    }
}

// FFT route: one CTA per pair of rows, the two rows as the real and imaginary
// parts of one N-point complex sequence (N a power of two >= 2D-1, so the
// circular convolution is the linear one on [0, D)), transformed in shared
// memory by a radix-4 Stockham FFT (one radix-2 pass first when log2 N is odd),
// multiplied by the real, even spectrum of the circular taps (divided by N)
// and transformed back: the real part is row a's filtered row, the imaginary
// part row b's.
constexpr int kFft64Threads = 256;

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dmul(double2 a, double2 w)
{
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}

// Stockham passes x -> y -> x ... over N = 2^L points (natural order in and
// out); tw[t] = exp(-2 pi i t / N), conjugated for the inverse.  Returns the
// buffer that holds the result.
template <bool INV>
__device__ double2 *fft64(double2 *x, double2 *y, const double2 *__restrict__ tw, int N, int L)
{
    int Ns = 1;
    if (L & 1) {  // radix-2 pass with Ns = 1: no twiddles
        for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
            const double2 v0 = x[j], v1 = x[j + N / 2];
            y[2 * j] = dadd(v0, v1);
            y[2 * j + 1] = dsub(v0, v1);
        }
        __syncthreads();
        double2 *t = x; x = y; y = t;
        Ns = 2;
    }
    for (; Ns < N; Ns <<= 2) {
        const int st = N / (4 * Ns);
        for (int j = threadIdx.x; j < N / 4; j += blockDim.x) {
            const int k = j & (Ns - 1);
            double2 w1 = __ldg(&tw[k * st]), w2 = __ldg(&tw[2 * k * st]), w3 = __ldg(&tw[3 * k * st]);
            if (INV) {
                w1.y = -w1.y;
                w2.y = -w2.y;
                w3.y = -w3.y;
            }
            const double2 v0 = x[j];
            const double2 v1 = dmul(x[j + N / 4], w1);
            const double2 v2 = dmul(x[j + N / 2], w2);
            const double2 v3 = dmul(x[j + 3 * (N / 4)], w3);
            const double2 a0 = dadd(v0, v2), a1 = dsub(v0, v2), a2 = dadd(v1, v3);
            const double2 d = dsub(v1, v3);
            const double2 a3 = INV ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);  // +-i d
            const int idx = ((j - k) << 2) + k;
            y[idx] = dadd(a0, a2);
            y[idx + Ns] = dadd(a1, a3);
            y[idx + 2 * Ns] = dsub(a0, a2);
            y[idx + 3 * Ns] = dsub(a1, a3);
        }
        __syncthreads();
        double2 *t = x; x = y; y = t;
    }
    return x;
}

__global__ void __launch_bounds__(kFft64Threads)
    filter_fft_f64_kernel(const double *__restrict__ sino, int ld,
                          const double2 *__restrict__ tw, const double *__restrict__ hs,
                          double *__restrict__ q, int A, int D, int N, int L, int pitch,
                          double i0)
{
    extern __shared__ double2 sz[];
    double2 *x = sz, *y = sz + N;
    const int ra = 2 * blockIdx.x, rb = ra + 1;
    const bool has_b = rb < A;
    const double *pa = sino + (size_t)ra * ld;
    const double *pb = sino + (size_t)(has_b ? rb : ra) * ld;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double a = 0.0, b = 0.0;
        if (j < D) {
            a = line_integral(pa[j], i0);
            if (has_b) b = line_integral(pb[j], i0);
        }
        x[j] = make_double2(a, b);
    }
    __syncthreads();
    double2 *z = fft64<false>(x, y, tw, N, L);
    double2 *o = (z == x) ? y : x;
    for (int f = threadIdx.x; f < N; f += blockDim.x) {
        const double h = __ldg(&hs[f]);
        z[f] = make_double2(z[f].x * h, z[f].y * h);
    }
    __syncthreads();
    z = fft64<true>(z, o, tw, N, L);
    // z[k] = (Q_a[k], Q_b[k]); pair p = (2 Q[p-1] - Q[p], Q[p] - Q[p-1]), Q
    // zero outside [0, D); pairs past D are zero
    double2 *qa = reinterpret_cast<double2 *>(q + (size_t)ra * pitch);
    double2 *qb = reinterpret_cast<double2 *>(q + (size_t)rb * pitch);
    for (int p = threadIdx.x; p < pitch / 2; p += blockDim.x) {
        double2 ma = make_double2(0.0, 0.0), mb = ma;
        if (p <= D) {
            const double2 lo = p > 0 ? z[p - 1] : make_double2(0.0, 0.0);
            const double2 hi = p < D ? z[p] : make_double2(0.0, 0.0);
            ma = make_double2(2.0 * lo.x - hi.x, hi.x - lo.x);
            mb = make_double2(2.0 * lo.y - hi.y, hi.y - lo.y);
        }
        qa[p] = ma;
        if (has_b) qb[p] = mb;
    }
}

// Backprojection: 16 x 16 pixels per 64-thread block, one thread per 4 pixels
// of a column (rows r0 + 4 j), the pairs read through the cache (every row of
// pairs serves the whole image).  Small blocks keep the FP64 work even across
// the SMs (a 512^2 image is 1024 blocks).  The detector coordinate
//     u = (X2 cos + Y2 sin) / (2 tau) + (D - 1) / 2,  X2 = 2c - (n-1), Y2 = 2r - (n-1)
// is a 64-bit integer in units of 2^-S (cos/tau and sin/tau in units of
// 2^-(S-1) from a plan table), so the next pixel's coordinate is an integer
// addition, floor(u) a shift, and 1 + (u - floor(u)) a double assembled from
// the fraction's bits: the FP64 pipe, about two operations per clock per SM
// on GB300, does only the interpolating FMA and the sum.
constexpr int kBp64Rows = 4;
constexpr int kBp64Threads = 16 * 16 / kBp64Rows;

__global__ void __launch_bounds__(kBp64Threads)
    backproject_f64_kernel(const double *__restrict__ q, int pitch,
                           const longlong2 *__restrict__ trig_fx, double *__restrict__ image,
                           int n, int A, int D, long long half_d_fx, int S, double scale)
{
    const int c = blockIdx.x * 16 + (threadIdx.x & 15);
    const int r0 = blockIdx.y * 16 + (threadIdx.x >> 4);
    const long long X2 = 2LL * c - (n - 1);
    const long long Y2 = 2LL * r0 - (n - 1);
    const unsigned long long frac_mask = (1ULL << S) - 1ULL;
    const int to_mantissa = 52 - S;
    constexpr unsigned long long kOne = 0x3FF0000000000000ULL;  // 1.0
    double acc[kBp64Rows];
#pragma unroll
    for (int j = 0; j < kBp64Rows; ++j) acc[j] = 0.0;
    for (int i = 0; i < A; ++i) {
        const longlong2 cs = __ldg(&trig_fx[i]);
        const double2 *row = reinterpret_cast<const double2 *>(q + (size_t)i * pitch);
        const long long du = (long long)(2 * (16 / kBp64Rows)) * cs.y;
        long long u = X2 * cs.x + Y2 * cs.y + half_d_fx;
#pragma unroll
        for (int j = 0; j < kBp64Rows; ++j) {
            if (j > 0) u += du;
            const int p = (int)(u >> S) + 1;  // pair of bin floor(u)
            const double f1 = __longlong_as_double(
                (long long)(kOne | (((unsigned long long)u & frac_mask) << to_mantissa)));
            if ((unsigned)p <= (unsigned)D) {
                const double2 ad = __ldg(&row[p]);
                acc[j] += fma(f1, ad.y, ad.x);
            }
        }
    }
    if (c < n) {
#pragma unroll
        for (int j = 0; j < kBp64Rows; ++j) {
            const int r = r0 + (16 / kBp64Rows) * j;
            if (r < n) image[(size_t)r * n + c] = acc[j] * scale;
        }
    }
}

}  // namespace

size_t filter_direct_f64_smem_bytes(int D) { return sizeof(double) * (size_t)(4 * D + 1); }

cudaError_t launch_filter_direct_f64(const Plan &p, const double *sino, int ld, double *q,
                                     cudaStream_t s)
{
    const size_t smem = filter_direct_f64_smem_bytes(p.D);
    cudaError_t e = cudaFuncSetAttribute(filter_direct_f64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_direct_f64_kernel<<<p.A, 256, smem, s>>>(sino, ld, p.d_taps64, q, p.D, p.pitch,
                                                     p.i0);
    return cudaGetLastError();
}

size_t filter_fft_f64_smem_bytes(int N) { return 2 * sizeof(double2) * (size_t)N; }

cudaError_t launch_filter_fft_f64(const Plan &p, const double *sino, int ld, double *q,
                                  cudaStream_t s)
{
    const int N = p.fft_len;
    int L = 0;
    while ((1 << L) < N) ++L;
    const size_t smem = filter_fft_f64_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(filter_fft_f64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_fft_f64_kernel<<<(p.A + 1) / 2, kFft64Threads, smem, s>>>(
        sino, ld, p.d_fft_tw64, p.d_fft_h64, q, p.A, p.D, N, L, p.pitch, p.i0);
    return cudaGetLastError();
}

cudaError_t prepare_fp64(const Plan &p)
{
    cudaError_t e;
    if (p.filter_path == FBP_PATH_FFT)
        e = cudaFuncSetAttribute(filter_fft_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)filter_fft_f64_smem_bytes(p.fft_len));
    else
        e = cudaFuncSetAttribute(filter_direct_f64_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)filter_direct_f64_smem_bytes(p.D));
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, backproject_f64_kernel);
    return e;
}

cudaError_t launch_backproject_f64(const Plan &p, const double *q, double *image, cudaStream_t s)
{
    dim3 grid((p.n + 15) / 16, (p.n + 15) / 16);
    backproject_f64_kernel<<<grid, kBp64Threads, 0, s>>>(q, p.pitch, p.d_trig_fx, image, p.n,
                                                          p.A, p.D, p.half_d_fx, p.fx_shift,
                                                          p.scale64);
    return cudaGetLastError();
}

}  // namespace fbp
