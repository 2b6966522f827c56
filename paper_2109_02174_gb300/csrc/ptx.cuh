// Inline-PTX helpers for sm_103a: shared-memory addresses, mbarriers, TMA
// tensor loads and bounded waits.  Every wait here gives up after a time
// limit and reports failure instead of spinning forever.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace fbp {

// Default limit of every device-side wait (ns of %globaltimer).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Run-time settings of the bounded waits (fbp_set_wait_limit and the
// test-only fbp_test_withhold_arrival).  Every translation unit with waiting
// kernels holds one copy as a device variable (waithook.cuh), which its kernels
// read when they start, so the settings also reach kernels of CUDA graphs
// captured before they changed.
enum : int { kWithholdNone = 0, kWithholdBackproject = 1, kWithholdFilterTc = 2 };
struct WaitHook {
    unsigned long long limit_ns;  // 0: kWaitLimitNs
    int kind;                     // kWithhold*: kernel kind whose first CTA withholds ...
    int stage;                    // ... the arrival of this stage (ring fill) of its pipeline
    int shrink;                   // index checks of FBP_CHECK_BOUNDS builds: window - shrink
};

// Index checks of debug builds (compiled with FBP_CHECK_BOUNDS): a kernel's
// index into its staged window outside [0, limit) is recorded in the launch's
// status words (code 8, kernel kind, index, limit; the first one only) and
// replaced by 0, so the access stays inside the window and nothing traps.
enum : int { kStatusBounds = 8, kCheckBackproject = 1, kCheckFdk = 2 };
__device__ __forceinline__ int check_index(int i, int limit, int *status, int kind)
{
    if (limit > 0 && (unsigned)i < (unsigned)limit) return i;
    if (atomicCAS(status, 0, kStatusBounds) == 0) {
        status[1] = kind;
        status[2] = i;
        status[3] = limit;
    }
    return 0;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make mbarrier initialisation and prior generic-proxy shared-memory accesses
// visible to the async proxy (TMA).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete; false once limit_ns
// have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// 2D tiled TMA load of one box into shared memory, completing on `bar`.
// x (innermost coordinate) must be a multiple of 16 bytes' worth of elements.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void prefetch_tensor_map(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(map))
                 : "memory");
}

}  // namespace fbp
