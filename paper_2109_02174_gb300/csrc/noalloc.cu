// fbp_reconstruct_static: fbp_reconstruct without a caller-supplied workspace
// and without any device allocation on the call path.
//
// Why it exists: some callers cannot allocate device memory when they want a
// reconstruction.  A scanner's acquisition loop that must keep a fixed
// per-slice deadline cannot absorb the device-wide synchronisation that
// cudaMalloc/cudaFree imply; an application whose device memory is owned by
// another allocator (a framework pool, or a hard budget that the rest of the
// process accounts for) may not make allocations of its own; and a plug-in
// that only receives device pointers from its host has no allocator at all.
// Such callers still own the sinogram and the image; the only scratch, the
// filtered sinogram, lives in a fixed array compiled into this library.
//
// The array below is a device symbol: every GPU that loads libfbp holds
// kStaticScratchBytes of it until the process exits.  Host code must never
// pass the symbol itself to a kernel (on the host it names a host-side shadow,
// not device memory); its device address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr size_t kStaticScratchBytes = FBP_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes % 256 == 0, "scratch size keeps 256-byte alignment");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
fbp_status static_scratch(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("fbp_reconstruct_static: device %d out of range", device);
        return FBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[device] == nullptr) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            set_error("fbp_reconstruct_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return FBP_ERR_CUDA;
        }
        g_scratch_ptr[device] = ptr;
    }
    *out = g_scratch_ptr[device];
    return FBP_OK;
}

}  // namespace
}  // namespace fbp

extern "C" fbp_status fbp_reconstruct_static(fbp_plan_t plan, const void *sino, int ld_sino,
                                             void *image, fbp_stream_t stream)
{
    using namespace fbp;
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (p == nullptr) {
        set_error("fbp_reconstruct_static: plan is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    size_t need = 0;
    fbp_status st = fbp_workspace_bytes(plan, &need);
    if (st != FBP_OK) return st;
    if (need > kStaticScratchBytes) {
        set_error("fbp_reconstruct_static: plan needs %zu bytes of scratch, the static array "
                  "holds %zu (use fbp_reconstruct with a workspace)",
                  need, kStaticScratchBytes);
        return FBP_ERR_BUDGET;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("fbp_reconstruct_static: no current CUDA device");
        return FBP_ERR_CUDA;
    }
    void *scratch = nullptr;
    st = static_scratch(dev, &scratch);
    if (st != FBP_OK) return st;
    // The filter writes every element of the filtered rows it covers (bins past
    // n_det as zeros), so nothing left in the array by an earlier call is read.
    st = fbp_filter(plan, sino, ld_sino, scratch, stream);
    if (st != FBP_OK) return st;
    return fbp_backproject(plan, scratch, image, stream);
}
