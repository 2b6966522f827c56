// The per-translation-unit copy of the wait settings (WaitHook, ptx.cuh).
// Include once per .cu file whose kernels wait on mbarriers; the file exports
// a host function that writes its copy (declared in fbp_internal.h).
#pragma once

#include "ptx.cuh"

namespace fbp {
namespace {

__device__ WaitHook g_wait_hook;

// The wait limit a kernel uses, read when it starts.
__device__ __forceinline__ unsigned long long wait_limit_ns(const WaitHook &h)
{
    return h.limit_ns ? h.limit_ns : kWaitLimitNs;
}

// Stage whose arrival this CTA withholds (tests only), or -1.
__device__ __forceinline__ int withheld_stage(const WaitHook &h, int kind, bool first_cta)
{
    return (first_cta && h.kind == kind) ? h.stage : -1;
}

inline cudaError_t write_wait_hook(const WaitHook &h)
{
    return cudaMemcpyToSymbol(g_wait_hook, &h, sizeof h);
}

}  // namespace
}  // namespace fbp
