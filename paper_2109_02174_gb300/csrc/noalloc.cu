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
// The array below is a device symbol: every GPU that loads libfbp's module
// holding it keeps kStaticScratchBytes of it until the process exits.  Host
// code must never pass the symbol itself to a kernel (on the host it names a
// host-side shadow, not device memory); its device address comes from
// cudaGetSymbolAddress, called with the device current.  That call is the
// set-up: fbp_plan makes it for its device after building the plan (CUDA loads
// modules lazily, so this is also where the array becomes resident on that
// device), and fbp_reconstruct_static only reads the address it left.  Every
// plan refreshes the address, so a plan made after a cudaDeviceReset (which
// invalidates earlier plans) never hands out a stale one.
#include <mutex>
#include <string>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr size_t kStaticScratchBytes = FBP_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes % 256 == 0, "scratch size keeps 256-byte alignment");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};
std::string g_scratch_err[kMaxDevices];

// The scratch array's device address on `device` (current), as the last plan
// made on it found it.
fbp_status static_scratch(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("fbp_reconstruct_static: device %d out of range", device);
        return FBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[device] == nullptr) {
        set_error("fbp_reconstruct_static: no scratch address on device %d (%s)", device,
                  g_scratch_err[device].empty() ? "no plan was made on it"
                                                : g_scratch_err[device].c_str());
        return FBP_ERR_CUDA;
    }
    *out = g_scratch_ptr[device];
    return FBP_OK;
}

}  // namespace

void static_scratch_setup(int device)
{
    if (device < 0 || device >= kMaxDevices) return;
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (e != cudaSuccess || ptr == nullptr) {
        // fbp_reconstruct_static reports this; every other call is unaffected
        g_scratch_ptr[device] = nullptr;
        g_scratch_err[device] = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        (void)cudaGetLastError();
        return;
    }
    g_scratch_ptr[device] = ptr;
    g_scratch_err[device].clear();
}

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
