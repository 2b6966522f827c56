// Internal declarations shared by the translation units of libfbp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "fbp.h"

namespace fbp {

// NVTX range over a host scope (the enqueue of a filter, a backprojection, a
// graph replay, a serving admission): visible in a profiler's timeline,
// inert otherwise (the header-only NVTX library does nothing until a tool
// attaches).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxFftLen = 8192;    // FP32 FFT route: two N-point complex buffers in shared memory
constexpr int kMaxFftLen64 = 4096;  // FP64 FFT route: two N-point double2 buffers (128 KB)
constexpr int kFftMaxSlices = 64; // slices per batched FFT launch

struct TcTables;  // tensor-core filter tables (filter_tc.cuh)

struct Plan {
    int n;      // image side
    int A;      // angles
    int D;      // detector bins
    int pitch;  // row pitch of the filtered sinogram, in elements of q_storage
    int filter;
    int dtype;
    int q_storage;
    int accumulate;
    int filter_path;
    int fft_len;
    double tau;
    int device;
    // Backprojection launch shape: tile (8 bp_wx) x (32 bp_wy) pixels and the
    // detector window per tile and angle, in (mid, slope) pairs.
    int bp_wx;
    int bp_wy;
    int bp_wp;
    int bp_chunk;  // angles per shared-memory stage (8, 16, 32)
    int bp_point_pairs;  // 1: work items are point-symmetric tile pairs (backproject.cu)
    double i0;       // > 0: the sinogram holds intensities, converted on load (Eq. 1)
    float i0f;
    float ln_i0f;    // ln(i0) (FP64, rounded)
    float scale32;   // pi / A
    double scale64;  // pi / A
    // Device tables owned by the plan.
    double2 *d_trig64;  // (cos th_i, sin th_i) / tau
    float *d_taps32;    // tau * h(m), m = -(D-1) .. D-1
    double *d_taps64;   // same in FP64
    float4 *d_fft_tw;   // FFT route: (c, c, s, s) with c + i s = exp(-2 pi i t / N), t < N
    float2 *d_fft_h;    // FFT route: (H, H), H = DFT_N of the circular taps / N (real, even)
    longlong2 *d_trig_fx;  // FP64 path: (cos, sin) / tau in units of 2^-(fx_shift-1)
    long long half_d_fx;   // FP64 path: (n_det - 1) / 2 in units of 2^-fx_shift
    int fx_shift;          // FP64 path: fraction bits of the fixed-point detector coordinate
    double2 *d_fft_tw64;  // FP64 FFT route: exp(-2 pi i t / N), t < N
    double *d_fft_h64;    // FP64 FFT route: H = DFT_N of the circular taps / N
    const float *d_row_weight;  // FFT route, optional: [row_weight_rows][D] factors applied to
    int row_weight_rows;        //   row r's values on load (row r uses table row r mod rows)
    int *d_status;      // device status word (0 = ok)
    TcTables *tc;       // Toeplitz route: T_hi / T_lo and their TMA maps
};

// Element size of the filtered sinogram.
inline int q_elem_bytes(const Plan &p)
{
    return p.dtype == FBP_F64 ? 8 : (p.q_storage == FBP_F16 ? 2 : 4);
}

// Thread-local error message for fbp_last_error().
void set_error(const char *fmt, ...);

// Tensor map over the filtered pairs of one slice: [A][2 (D+1)] elements of the
// q_storage type with row stride pitch, box {2 wp, 1}.
bool encode_pairs_map(const Plan &p, const void *q, CUtensorMap *out);

// Tensor map over `planes` x `rows` rows of `row_floats` floats (row stride
// `pitch` floats, a multiple of 4), box {box_x floats, box_y rows, 1}; outside
// the extents TMA fills zeros.
bool encode_rows_map_3d(const void *q, int row_floats, int pitch, int rows, int planes,
                        int box_x, int box_y, CUtensorMap *out);

// A second stream for enqueue_many: when given, the single-slice
// backprojection launches run on `side` (after `fork`, recorded on the main
// stream once the filters are enqueued) beside the two-slice launches, and the
// main stream waits for `join` at the end, so one launch's last work items
// and the other's overlap.
struct BpFork {
    cudaStream_t side;
    cudaEvent_t fork;
    cudaEvent_t join;
};

// Every slice's filter, then the persistent backprojection launches over all
// slices' tiles (batch.cu).  `sched`: n_sched work counters (two ints each,
// zero) for the backprojection launches in order; launches beyond them
// stride.  Launch-only: no allocation, no synchronisation.
cudaError_t enqueue_many(const Plan *const *plans, const fbp_batch_io *io, int n, int parts,
                         int *status, cudaStream_t s, int *sched, int n_sched,
                         const BpFork *fork = nullptr);

// Filter launchers: write the (mid, slope) pairs of every row (see fbp.h).
cudaError_t launch_filter_direct(const Plan &p, const float *sino, int ld, void *q,
                                 cudaStream_t s);
cudaError_t launch_filter_fft(const Plan &p, const float *sino, int ld, void *q, cudaStream_t s);
// The FFT-route slices among plans[0..n) in as few launches as possible
// (other slices are skipped).
cudaError_t launch_filter_fft_many(const Plan *const *plans, const float *const *sinos,
                                   const int *lds, void *const *qs, int n, cudaStream_t s);
size_t filter_fft_smem_bytes(int N);
size_t filter_direct_smem_bytes(int D);

// Backprojection of one slice with its plan's launch shape.
cudaError_t backproject_slice(const Plan &p, const void *q, float *image, cudaStream_t s);

// FP64 path (fp64.cu).
cudaError_t launch_filter_direct_f64(const Plan &p, const double *sino, int ld, double *q,
                                     cudaStream_t s);
cudaError_t launch_filter_fft_f64(const Plan &p, const double *sino, int ld, double *q,
                                  cudaStream_t s);
cudaError_t launch_backproject_f64(const Plan &p, const double *q, double *image, cudaStream_t s);
size_t filter_direct_f64_smem_bytes(int D);
size_t filter_fft_f64_smem_bytes(int N);

cudaError_t launch_radon_forward_f32(const Plan &p, const float *image, float *sino,
                                     cudaStream_t s);

// Writers of each translation unit's copy of the wait settings (WaitHook,
// ptx.cuh) on the current device.
struct WaitHook;
cudaError_t set_wait_hook_backproject(const WaitHook &h);
cudaError_t set_wait_hook_filter_tc(const WaitHook &h);
cudaError_t set_wait_hook_fdk(const WaitHook &h);

// Device status words of a plan or batch: [0] the status (0, FBP_ERR_TIMEOUT,
// or FBP_ERR_BOUNDS from the index checks of debug builds), [1..3] what an
// index check recorded (kernel kind, index, limit).
constexpr int kStatusWords = 4;
// Synchronise the device, read and clear the words, and turn them into a
// status and error message (fn names the caller).
fbp_status take_device_status(int *d_status, const char *fn);

// Kernel preparation at plan time (each loads, under CUDA's lazy module
// loading, the kernels the plan's single-slice path launches, and sets their
// shared-memory limits), so later calls load no code.
cudaError_t prepare_filter_fft(const Plan &p);
cudaError_t prepare_filter_direct(const Plan &p);
cudaError_t prepare_filter_tc(const Plan &p);
cudaError_t prepare_backproject(const Plan &p);
cudaError_t prepare_fp64(const Plan &p);

// Device address of fbp_reconstruct_static's scratch array on the current
// device, looked up at plan time (noalloc.cu).
void static_scratch_setup(int device);

}  // namespace fbp
