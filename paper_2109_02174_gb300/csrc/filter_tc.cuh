// Plan tables of the tensor-core (Toeplitz) filter route (filter_tc.cu).
#pragma once

#include "fbp_internal.h"

namespace fbp {

// T[n][k] = tau h(n - k) split into tf32 hi and lo parts, [n_det][kpad] fp32
// each, with their TMA maps (box 32 x 128, 128-byte swizzle).
struct TcTables {
    CUtensorMap t_hi;
    CUtensorMap t_lo;
    float *d_hi;
    float *d_lo;
    int kpad;
};

size_t filter_tc_smem_bytes();
cudaError_t launch_filter_tc(const Plan &p, const float *sino, int ld, float *q, cudaStream_t s);

}  // namespace fbp
