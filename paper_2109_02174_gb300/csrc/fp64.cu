// FP64 variant of the whole path, for the paper's float-vs-double comparison
// (section "Results and discussion", double data type).  Same operator as the
// FP32 path: the direct ramp-filter convolution (the text after Eq. 2) written
// as (mid, slope) pairs of doubles, then Eq. 2 per pixel with linear
// interpolation, angles summed in order.  Plain CUDA-core code: GB300's FP64
// rate is a small fraction of its FP32 rate, so this path is for accuracy, not
// throughput.
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
            row[p] = make_double2((sq[p] + sq[p + 1]) * 0.5, sq[p + 1] - sq[p]);
        else
            row[p] = make_double2(0.0, 0.0);
    }
}

// One thread per pixel; pairs are read through the cache (each row of pairs is
// reused by every pixel of the image).
__global__ void __launch_bounds__(256)
    backproject_f64_kernel(const double *__restrict__ q, int pitch,
                           const double2 *__restrict__ trig, double *__restrict__ image, int n,
                           int A, int D, double half_n, double half_d, double scale)
{
    const int c = blockIdx.x * 16 + (threadIdx.x & 15);
    const int r = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (r >= n || c >= n) return;
    const double x = (double)c - half_n;
    const double y = (double)r - half_n;
    double acc = 0.0;
    for (int i = 0; i < A; ++i) {
        const double2 cs = __ldg(&trig[i]);
        const double u = x * cs.x + y * cs.y + half_d;
        const double fk = floor(u);
        const int p = (int)fk + 1;  // pair of bin floor(u)
        if (p >= 0 && p <= D) {
            const double2 ms = __ldg(reinterpret_cast<const double2 *>(q + (size_t)i * pitch) + p);
            acc += fma(u - fk - 0.5, ms.y, ms.x);
        }
    }
    image[(size_t)r * n + c] = acc * scale;
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

cudaError_t launch_backproject_f64(const Plan &p, const double *q, double *image, cudaStream_t s)
{
    dim3 grid((p.n + 15) / 16, (p.n + 15) / 16);
    backproject_f64_kernel<<<grid, 256, 0, s>>>(q, p.pitch, p.d_trig64, image, p.n, p.A, p.D,
                                                0.5 * (double)(p.n - 1), 0.5 * (double)(p.D - 1),
                                                p.scale64);
    return cudaGetLastError();
}

}  // namespace fbp
