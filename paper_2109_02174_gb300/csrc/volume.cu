// A 3D volume from a stack of reconstructed 2D slices, by interpolation along
// z (section "Introduction": 3D CT images from the interpolation of a stack of
// 2D images; the paper gives no rule, linear interpolation is used):
//     plane m = (1 - t_m) S_k + t_m S_{k+1},  z_k <= zo_m <= z_{k+1},
//     t_m = (zo_m - z_k) / (z_{k+1} - z_k).
// The interval and weights of every plane are found on the host (FP64); the
// device streams two slices in and one plane out per voxel, an HBM-bound copy
// with 16-byte vector accesses when n^2 is a multiple of four.  One launch
// covers up to kVolPlanes planes (their table rides in the kernel parameters),
// so the call allocates nothing.
#include <vector>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kVolPlanes = 256;

struct VolPlane {
    const float *a;  // S_k
    const float *b;  // S_{k+1}
    float wa;        // 1 - t
    float wb;        // t
};

struct VolLaunch {
    VolPlane p[kVolPlanes];
    float *out;  // first plane of this launch
    long np;     // voxels per plane (n^2)
};

template <bool VEC4>
__global__ void __launch_bounds__(256) volume_kernel(const __grid_constant__ VolLaunch L)
{
    const VolPlane &P = L.p[blockIdx.y];
    float *o = L.out + (size_t)blockIdx.y * (size_t)L.np;
    const long stride = (long)gridDim.x * blockDim.x;
    if (VEC4) {
        const float4 *a = reinterpret_cast<const float4 *>(P.a);
        const float4 *b = reinterpret_cast<const float4 *>(P.b);
        float4 *o4 = reinterpret_cast<float4 *>(o);
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L.np / 4; i += stride) {
            const float4 u = __ldg(&a[i]), v = __ldg(&b[i]);
            o4[i] = make_float4(fmaf(P.wb, v.x, P.wa * u.x), fmaf(P.wb, v.y, P.wa * u.y),
                                fmaf(P.wb, v.z, P.wa * u.z), fmaf(P.wb, v.w, P.wa * u.w));
        }
    } else {
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L.np; i += stride)
            o[i] = fmaf(P.wb, __ldg(&P.b[i]), P.wa * __ldg(&P.a[i]));
    }
}

}  // namespace
}  // namespace fbp

using namespace fbp;

extern "C" {

fbp_status fbp_volume_from_slices(const void *const *slices, int n_slices, const double *z,
                                  int n_pix, const double *z_out, int n_planes, void *volume,
                                  fbp_stream_t stream)
{
    if (slices == nullptr || z == nullptr || z_out == nullptr || volume == nullptr ||
        n_slices < 1 || n_planes < 1 || n_pix < 1) {
        set_error("fbp_volume_from_slices: NULL argument or a count < 1");
        return FBP_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_slices; ++k) {
        if (slices[k] == nullptr || (reinterpret_cast<uintptr_t>(slices[k]) & 15u) != 0) {
            set_error("fbp_volume_from_slices: slice %d is NULL or not 16-byte aligned", k);
            return slices[k] ? FBP_ERR_ALIGNMENT : FBP_ERR_INVALID_ARG;
        }
        if (k > 0 && !(z[k] > z[k - 1])) {
            set_error("fbp_volume_from_slices: slice positions must increase strictly");
            return FBP_ERR_INVALID_ARG;
        }
    }
    if ((reinterpret_cast<uintptr_t>(volume) & 15u) != 0) {
        set_error("fbp_volume_from_slices: volume not 16-byte aligned");
        return FBP_ERR_ALIGNMENT;
    }
    const long np = (long)n_pix * n_pix;
    const bool vec4 = (np % 4) == 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<VolPlane> planes((size_t)n_planes);
    for (int m = 0; m < n_planes; ++m) {
        const double zm = z_out[m];
        if (!(zm >= z[0] && zm <= z[n_slices - 1])) {
            set_error("fbp_volume_from_slices: plane %d (z = %g) outside the stack", m, zm);
            return FBP_ERR_INVALID_ARG;
        }
        VolPlane &P = planes[(size_t)m];
        if (n_slices == 1) {
            P = {static_cast<const float *>(slices[0]), static_cast<const float *>(slices[0]),
                 1.0f, 0.0f};
            continue;
        }
        int k = 0;
        while (k + 1 < n_slices - 1 && zm > z[k + 1]) ++k;
        const double t = (zm - z[k]) / (z[k + 1] - z[k]);
        P = {static_cast<const float *>(slices[k]), static_cast<const float *>(slices[k + 1]),
             (float)(1.0 - t), (float)t};
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int m0 = 0; m0 < n_planes; m0 += kVolPlanes) {
        const int cnt = n_planes - m0 < kVolPlanes ? n_planes - m0 : kVolPlanes;
        VolLaunch L;
        for (int i = 0; i < cnt; ++i) L.p[i] = planes[(size_t)(m0 + i)];
        L.out = static_cast<float *>(volume) + (size_t)m0 * (size_t)np;
        L.np = np;
        const long work = vec4 ? np / 4 : np;
        long bx = (work + 255) / 256;
        const long cap = (long)(sms > 0 ? sms : 1) * 8 / cnt + 1;  // about 8 CTAs per SM in all
        if (bx > cap) bx = cap;
        if (bx < 1) bx = 1;
        const dim3 grid((unsigned)bx, (unsigned)cnt);
        if (vec4)
            volume_kernel<true><<<grid, 256, 0, s>>>(L);
        else
            volume_kernel<false><<<grid, 256, 0, s>>>(L);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("fbp_volume_from_slices: %s", cudaGetErrorString(e));
            return FBP_ERR_CUDA;
        }
    }
    return FBP_OK;
}

}  // extern "C"
