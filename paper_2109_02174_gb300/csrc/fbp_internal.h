// Internal declarations shared by the translation units of libfbp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "fbp.h"

namespace fbp {

// Launch shape of the FP32 backprojection.  A work item is one tile of
// tile_x x tile_y pixels; its detector window per angle is `wraw` bins long
// (a multiple of 4, at most 256 = the TMA box limit).
constexpr int kBpTileX = 32;
constexpr int kBpTileY = 32;
constexpr int kBpChunk = 16;
constexpr int kMaxFftLen = 8192;  // two N-point complex buffers in shared memory

struct BpShape {
    int tile_x;
    int tile_y;
    int chunk;  // angles staged per shared-memory window
    int wraw;
};

struct Plan {
    int n;      // image side
    int A;      // angles
    int D;      // detector bins
    int pitch;  // row pitch (elements) of the filtered sinogram
    int filter;
    int dtype;
    int q_storage;
    int accumulate;
    int filter_path;
    int fft_len;
    double tau;
    int device;
    BpShape bp;
    float scale32;   // pi / A
    double scale64;  // pi / A
    // Device tables owned by the plan.
    double2 *d_trig64;  // (cos th_i, sin th_i) / tau
    float *d_taps32;    // tau * h(m), m = -(D-1) .. D-1
    double *d_taps64;   // same in FP64
    float2 *d_fft_tw;   // FFT route: exp(-2 pi i t / N), t < N
    float *d_fft_h;     // FFT route: DFT_N of the circular taps, times 1/N (real, even)
    int *d_status;      // device status word (0 = ok)
};

// Thread-local error message for fbp_last_error().
void set_error(const char *fmt, ...);

// Tensor map of a filtered sinogram [A][pitch] (4-byte elements), box {wraw, 1}.
bool encode_q_map(const Plan &p, const void *q, int wraw, CUtensorMap *out);

// Launchers (each returns the launch's cudaError_t).
cudaError_t launch_filter_direct_f32(const Plan &p, const float *sino, int ld, float *q,
                                     cudaStream_t s);
cudaError_t launch_filter_fft_f32(const Plan &p, const float *sino, int ld, float *q,
                                  cudaStream_t s);
size_t filter_fft_smem_bytes(int N);
size_t filter_direct_smem_bytes(int D);
cudaError_t launch_backproject_f32(const Plan &p, const CUtensorMap &qmap, float *image,
                                   cudaStream_t s);
cudaError_t launch_radon_forward_f32(const Plan &p, const float *image, float *sino,
                                     cudaStream_t s);

}  // namespace fbp
