// Ramp filter Q = P * H (the convolution stated after Eq. 2), direct route:
//   Q[i][k] = sum_{j=0}^{n_det-1} (tau h)(k - j) * P[i][j],   k < n_det
//   Q[i][k] = 0                                               n_det <= k < pitch
// One CTA per sinogram row; the row and the 2*n_det-1 taps sit in shared
// memory; each thread owns output bins k, k + blockDim, ... and sums j in
// increasing order (deterministic).
#include "fbp_internal.h"

namespace fbp {
namespace {

__global__ void __launch_bounds__(256)
    filter_direct_f32_kernel(const float *__restrict__ sino, int ld,
                             const float *__restrict__ taps, float *__restrict__ q, int D,
                             int pitch)
{
    extern __shared__ float sm[];
    float *st = sm;               // taps, index m + D - 1
    float *sp = sm + (2 * D - 1); // the row
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < 2 * D - 1; t += blockDim.x) st[t] = taps[t];
    for (int t = threadIdx.x; t < D; t += blockDim.x) sp[t] = sino[(size_t)i * ld + t];
    __syncthreads();
    for (int k = threadIdx.x; k < pitch; k += blockDim.x) {
        float acc = 0.0f;
        if (k < D) {
            const float *hk = st + k + D - 1;
            for (int j = 0; j < D; ++j) acc = fmaf(hk[-j], sp[j], acc);
        }
        q[(size_t)i * pitch + k] = acc;
    }
}

}  // namespace

size_t filter_direct_smem_bytes(int D) { return sizeof(float) * (size_t)(3 * D - 1); }

cudaError_t launch_filter_direct_f32(const Plan &p, const float *sino, int ld, float *q,
                                     cudaStream_t s)
{
    const size_t smem = filter_direct_smem_bytes(p.D);
    cudaError_t e = cudaFuncSetAttribute(filter_direct_f32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_direct_f32_kernel<<<p.A, 256, smem, s>>>(sino, ld, p.d_taps32, q, p.D, p.pitch);
    return cudaGetLastError();
}

}  // namespace fbp
