// Ramp filter Q = P * H (the convolution stated after Eq. 2), direct route:
//   Q[i][k] = sum_{j=0}^{n_det-1} (tau h)(k - j) * P[i][j],   0 <= k < n_det
// One CTA per sinogram row; the row and the 2*n_det-1 taps sit in shared
// memory; each thread owns output bins k, k + blockDim, ... and sums j in
// increasing order (deterministic).  The row is then written as (mid, slope)
// pairs (pairs.cuh).  Intensity input is converted on load (lambert.cuh).
#include "fbp_internal.h"
#include "lambert.cuh"
#include "pairs.cuh"

namespace fbp {
namespace {

template <typename OutT>
__global__ void __launch_bounds__(256)
    filter_direct_kernel(const float *__restrict__ sino, int ld, const float *__restrict__ taps,
                         OutT *__restrict__ q, int D, int pitch, float i0, float ln_i0)
{
    extern __shared__ float sm[];
    float *st = sm;                // taps, index m + D - 1
    float *sp = sm + (2 * D - 1);  // the row
    float *sq = sp + D;            // sq[k + 1] = Q[k], sq[0] = sq[D + 1] = 0
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < 2 * D - 1; t += blockDim.x) st[t] = taps[t];
    for (int t = threadIdx.x; t < D; t += blockDim.x)
        sp[t] = line_integral(sino[(size_t)i * ld + t], i0, ln_i0);
    if (threadIdx.x == 0) {
        sq[0] = 0.0f;
        sq[D + 1] = 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        const float *hk = st + k + D - 1;
        float acc = 0.0f;
        for (int j = 0; j < D; ++j) acc = fmaf(hk[-j], sp[j], acc);
        sq[k + 1] = acc;
    }
    __syncthreads();
    OutT *row = q + (size_t)i * pitch;
    for (int p = threadIdx.x; p < pitch / 2; p += blockDim.x) {
        if (p <= D)
            store_pair(row, p, sq[p], sq[p + 1]);
        else
            store_pair(row, p, 0.0f, 0.0f);
    }
}

template <typename OutT>
cudaError_t launch(const Plan &p, const float *sino, int ld, OutT *q, cudaStream_t s)
{
    const size_t smem = filter_direct_smem_bytes(p.D);
    cudaError_t e = cudaFuncSetAttribute(filter_direct_kernel<OutT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_direct_kernel<OutT><<<p.A, 256, smem, s>>>(sino, ld, p.d_taps32, q, p.D, p.pitch,
                                                       p.i0f, p.ln_i0f);
    return cudaGetLastError();
}

}  // namespace

size_t filter_direct_smem_bytes(int D) { return sizeof(float) * (size_t)(4 * D + 1); }

cudaError_t prepare_filter_direct(const Plan &p)
{
    const int smem = (int)filter_direct_smem_bytes(p.D);
    if (p.q_storage == FBP_F16)
        return cudaFuncSetAttribute(filter_direct_kernel<__half>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaFuncSetAttribute(filter_direct_kernel<float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_filter_direct(const Plan &p, const float *sino, int ld, void *q,
                                 cudaStream_t s)
{
    if (p.q_storage == FBP_F16) return launch(p, sino, ld, static_cast<__half *>(q), s);
    return launch(p, sino, ld, static_cast<float *>(q), s);
}

}  // namespace fbp
