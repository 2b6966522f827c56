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

constexpr int kTcMaxSlices = 64;  // slices of one plan per launch

size_t filter_tc_smem_bytes();
cudaError_t launch_filter_tc(const Plan &p, const float *sino, int ld, float *q, cudaStream_t s);
// Every slice of `n` that uses plan p in as few launches as possible.
cudaError_t launch_filter_tc_many(const Plan &p, const float *const *sinos, const int *lds,
                                  float *const *qs, int n, cudaStream_t s);

}  // namespace fbp
