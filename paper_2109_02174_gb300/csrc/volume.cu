// A 3D volume from a stack of reconstructed 2D slices, by interpolation along
// z (section "Introduction": 3D CT images from the interpolation of a stack of
// 2D images; the paper gives no rule, linear interpolation is used):
//     plane m = (1 - t_m) S_k + t_m S_{k+1},  z_k <= zo_m <= z_{k+1},
//     t_m = (zo_m - z_k) / (z_{k+1} - z_k).
// The interval and weights of every plane are found on the host (FP64);
// consecutive planes in one interval form a group of up to kGroup planes, and
// the device streams the group's two slices in once and its planes out (16-byte
// vectors when n^2 is a multiple of four): an HBM-bound copy whose reads fall
// from two slices per plane to two per group.  One launch covers up to
// kVolGroups groups (their table rides in the kernel parameters), so the call
// allocates nothing.
#include <vector>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kGroup = 8;       // planes per group
constexpr int kVolGroups = 192;  // groups per launch

struct VolGroup {
    const float *a;  // S_k
    const float *b;  // S_{k+1}
    int m0;          // first plane of the group, counted from the launch's first plane
    int cnt;         // planes in the group, 1 .. kGroup
    float wa[kGroup];  // 1 - t
    float wb[kGroup];  // t
};

struct VolLaunch {
    VolGroup g[kVolGroups];
    float *out;  // first plane of this launch
    long np;     // voxels per plane (n^2)
};

template <bool VEC4>
__global__ void __launch_bounds__(256) volume_kernel(const __grid_constant__ VolLaunch L)
{
    const VolGroup &G = L.g[blockIdx.y];
    const long stride = (long)gridDim.x * blockDim.x;
    if (VEC4) {
        const float4 *a = reinterpret_cast<const float4 *>(G.a);
        const float4 *b = reinterpret_cast<const float4 *>(G.b);
        float4 *o4 = reinterpret_cast<float4 *>(L.out) + (size_t)G.m0 * (size_t)(L.np / 4);
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L.np / 4; i += stride) {
            const float4 u = __ldg(&a[i]), v = __ldg(&b[i]);
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                if (j < G.cnt) {
                    const float wa = G.wa[j], wb = G.wb[j];
                    o4[(size_t)j * (size_t)(L.np / 4) + i] =
                        make_float4(fmaf(wb, v.x, wa * u.x), fmaf(wb, v.y, wa * u.y),
                                    fmaf(wb, v.z, wa * u.z), fmaf(wb, v.w, wa * u.w));
                }
            }
        }
    } else {
        float *o = L.out + (size_t)G.m0 * (size_t)L.np;
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L.np; i += stride) {
            const float u = __ldg(&G.a[i]), v = __ldg(&G.b[i]);
#pragma unroll
            for (int j = 0; j < kGroup; ++j)
                if (j < G.cnt) o[(size_t)j * (size_t)L.np + i] = fmaf(G.wb[j], v, G.wa[j] * u);
        }
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
    // interval and weights of every plane, then groups of consecutive planes
    // that share an interval
    std::vector<int> kk((size_t)n_planes);
    std::vector<float> wa((size_t)n_planes), wb((size_t)n_planes);
    for (int m = 0; m < n_planes; ++m) {
        const double zm = z_out[m];
        if (!(zm >= z[0] && zm <= z[n_slices - 1])) {
            set_error("fbp_volume_from_slices: plane %d (z = %g) outside the stack", m, zm);
            return FBP_ERR_INVALID_ARG;
        }
        if (n_slices == 1) {
            kk[(size_t)m] = 0;
            wa[(size_t)m] = 1.0f;
            wb[(size_t)m] = 0.0f;
            continue;
        }
        int k = 0;
        while (k + 1 < n_slices - 1 && zm > z[k + 1]) ++k;
        const double t = (zm - z[k]) / (z[k + 1] - z[k]);
        kk[(size_t)m] = k;
        wa[(size_t)m] = (float)(1.0 - t);
        wb[(size_t)m] = (float)t;
    }
    std::vector<VolGroup> groups;
    for (int m = 0; m < n_planes;) {
        const int k = kk[(size_t)m];
        VolGroup G;
        G.a = static_cast<const float *>(slices[k]);
        G.b = static_cast<const float *>(slices[n_slices == 1 ? 0 : k + 1]);
        G.m0 = m;
        G.cnt = 0;
        while (m < n_planes && kk[(size_t)m] == k && G.cnt < kGroup) {
            G.wa[G.cnt] = wa[(size_t)m];
            G.wb[G.cnt] = wb[(size_t)m];
            ++G.cnt;
            ++m;
        }
        for (int j = G.cnt; j < kGroup; ++j) G.wa[j] = G.wb[j] = 0.0f;
        groups.push_back(G);
    }
    const int n_groups = (int)groups.size();
    for (int g0 = 0; g0 < n_groups; g0 += kVolGroups) {
        const int cnt = n_groups - g0 < kVolGroups ? n_groups - g0 : kVolGroups;
        VolLaunch L;
        const int m_first = groups[(size_t)g0].m0;
        for (int i = 0; i < cnt; ++i) {
            L.g[i] = groups[(size_t)(g0 + i)];
            L.g[i].m0 -= m_first;
        }
        L.out = static_cast<float *>(volume) + (size_t)m_first * (size_t)np;
        L.np = np;
        // one thread per vector (the loop only covers planes beyond 2^24
        // vectors): many short CTAs keep more stores in flight than a grid
        // of about 8 CTAs per SM looping over the plane (64 x 512^2 slices
        // to 253 planes: 54.9 us, 6.05 TB/s, against 63.1 us)
        const long work = vec4 ? np / 4 : np;
        long bx = (work + 255) / 256;
        if (bx > 65535) bx = 65535;
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
