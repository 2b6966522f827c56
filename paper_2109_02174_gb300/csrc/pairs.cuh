// Writing the filtered sinogram in interpolation-ready form: for every bin
// k = -1 .. n_det-1 the pair (mid_k, slope_k) = ((Q[k] + Q[k+1]) / 2, Q[k+1] - Q[k]),
// Q zero outside [0, n_det); pair p (= k + 1) sits at elements 2p, 2p+1 of the
// row; pairs n_det+1 .. pitch/2-1 are zero.
#pragma once

#include <cuda_fp16.h>

namespace fbp {

__device__ __forceinline__ void store_pair(float *row, int p, float q0, float q1)
{
    reinterpret_cast<float2 *>(row)[p] = make_float2((q0 + q1) * 0.5f, q1 - q0);
}

__device__ __forceinline__ void store_pair(__half *row, int p, float q0, float q1)
{
    reinterpret_cast<__half2 *>(row)[p] = __floats2half2_rn((q0 + q1) * 0.5f, q1 - q0);
}

}  // namespace fbp
