/*
 * fbp.h -- C ABI of libfbp: GPU filtered backprojection (FBP) for 2D
 * parallel-beam CT on NVIDIA GB300 (sm_103a).
 *
 * The method is the paper's Eq. 2 ("Performance evaluation in the
 * reconstruction of 2D images of computed tomography using massively parallel
 * programming CUDA", arXiv 2109.02174, section "Computed tomography"):
 *
 *     f(x,y) = (pi/A) * sum_{i=0}^{A-1} Q_i(x cos th_i + y sin th_i),
 *     Q_i    = P_i * H   (each sinogram row convolved with a ramp filter)
 *
 * Geometry (the paper fixes none of it; this library's convention):
 *   - image f is n_pix x n_pix, row-major f[r][c]; pixel centre
 *     x = c - (n_pix-1)/2, y = r - (n_pix-1)/2 (pixel size 1);
 *   - detector bin k of n_det has centre t_k = (k - (n_det-1)/2) * det_spacing;
 *   - Q_i is read at t by linear interpolation, zero outside [0, n_det);
 *   - the angular weight pi/A is applied (Eq. 2 as printed omits it).
 *
 * Conventions of every call:
 *   - Ownership: the caller owns every buffer passed in (device memory unless
 *     stated); the plan owns its own tables.  Nothing here frees caller memory.
 *   - Asynchrony: compute calls only enqueue work on `stream` and return; the
 *     result is ready when the stream is.  fbp_plan() synchronises once (table
 *     upload).  A NULL stream is the legacy default stream.
 *   - Errors: every call returns an fbp_status; fbp_last_error() gives a
 *     message for the calling thread.  Arguments are checked on the host
 *     before any launch.  A device-side timeout (a bounded wait that ran out)
 *     is recorded in the plan's status word: fbp_device_status() reads it.
 *   - Alignment: every device pointer must be 16-byte aligned, else
 *     FBP_ERR_ALIGNMENT.
 *   - Element type: float for FBP_F32 plans, double for FBP_F64 plans (the
 *     sinogram, the image and, unless q_storage says otherwise, the filtered
 *     sinogram).
 */
#ifndef FBP_H
#define FBP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque plan: geometry, filter, trig and filter tables, tuned launch shape. */
typedef struct fbp_plan_s *fbp_plan_t;

/* A CUDA stream (the same type as cudaStream_t). */
typedef struct CUstream_st *fbp_stream_t;

typedef enum {
    FBP_OK = 0,
    FBP_ERR_INVALID_ARG = 1,
    FBP_ERR_ALIGNMENT = 2,
    FBP_ERR_OUT_OF_MEMORY = 3,
    FBP_ERR_BUDGET = 4,
    FBP_ERR_CUDA = 5,
    FBP_ERR_TIMEOUT = 6,
    FBP_ERR_UNSUPPORTED = 7,
    /* Debug builds (compiled with FBP_CHECK_BOUNDS) only: a kernel computed an
     * index outside the detector window it staged in shared memory; the first
     * such index is recorded (fbp_last_error names the kernel, index and
     * limit) and the access is redirected inside the window. */
    FBP_ERR_BOUNDS = 8
} fbp_status;

/* The filter H of Q = P * H.  The paper does not name it; the band-limited
 * spatial ramp kernels of Kak & Slaney (ch. 3) are offered:
 *   Ram-Lak:     h(0) = 1/(4 tau^2), h(m even) = 0, h(m odd) = -1/(pi^2 m^2 tau^2)
 *   Shepp-Logan: h(m) = 2/(pi^2 tau^2 (1 - 4 m^2))
 *   none:        Q = P (plain backprojection)
 * and Q_i[k] = tau * sum_{j=0}^{n_det-1} h(k-j) P_i[j] (linear convolution). */
typedef enum {
    FBP_FILTER_RAM_LAK = 0,
    FBP_FILTER_SHEPP_LOGAN = 1,
    FBP_FILTER_NONE = 2
} fbp_filter_type;

/* Element types. */
enum { FBP_F32 = 0, FBP_F64 = 1, FBP_F16 = 2 };
/* Accumulation over angles: plain FP32 sum, or Kahan-compensated. */
enum { FBP_ACC_PLAIN = 0, FBP_ACC_KAHAN = 1 };
/* Filter route (all compute the same linear convolution). */
enum { FBP_PATH_AUTO = 0, FBP_PATH_TOEPLITZ_TC = 1, FBP_PATH_FFT = 2, FBP_PATH_DIRECT = 3 };

typedef struct {
    int dtype;        /* FBP_F32 (default) or FBP_F64 (float-vs-double comparison) */
    int q_storage;    /* FBP_F32 (default) or FBP_F16: element type of the filtered
                         sinogram's (mid, slope) pairs.  FP16 pairs round every stored
                         value to 2^-11 of itself and hold magnitudes below 65504 (the
                         filtered rows must fit); the backprojection feeds them, with an
                         FP16 interpolation weight, straight into FP32 sums (faster than
                         FP32 pairs; error stated, no bar) */
    int accumulate;   /* FBP_ACC_PLAIN (default) or FBP_ACC_KAHAN */
    int filter_path;  /* FBP_PATH_AUTO (default), _TOEPLITZ_TC, _FFT or _DIRECT.  AUTO
                         takes the FFT when its length fits (8192 FP32, 4096 FP64),
                         else the direct convolution; FP64 plans have no tensor-core
                         route */
    int fft_len;      /* 0 = auto (next power of two >= 2*n_det-1) */
    int tile_x;       /* pixel tile of one backprojection work item: 32x64, 32x32 or
                         8x32; 0 = auto for one slice (the largest whose detector
                         window fits and that leaves at most half the SMs idle);
                         -1 = the largest that fits (for batches and waves) */
    int tile_y;       /* 0 = auto, -1 = largest (with tile_x) */
    int angle_chunk;  /* angles staged per shared-memory window: 8, 16, 32; 0 = 32 */
    double i0;        /* 0 (default): the sinogram holds line integrals p.  > 0: it
                         holds measured intensities or photon counts I of rays with
                         incident intensity i0, and every filter route converts them
                         as it loads them, p = -ln(max(I, 1) / i0) (Eq. 1,
                         Lambert-Beer; one count is the floor).  Must be finite. */
    int point_pairs;  /* backprojection work items as pairs of tiles mirrored through
                         the image centre, a pixel and its partner computed from one
                         detector position (they sit at u and n_det - 1 - u): 0 = auto,
                         1 = on when the plan can, -1 = off.  A plan can when n_pix is
                         a multiple of both tile sides, the tile grid is not odd in
                         both directions, and the sum is plain (not Kahan).  Auto
                         applies to the automatic tile only (tile_x = tile_y = 0): it
                         takes pairs on 32 x 32 tiles when one slice has at least 7/4
                         tiles of 32 x 64 per SM (n_pix > 704 on 152 SMs).  The images
                         differ from those without pairs in the last bits only. */
} fbp_options;

/* Fill *opt with the defaults listed above. */
fbp_status fbp_options_default(fbp_options *opt);

/*
 * Create a plan on the current CUDA device.
 *   n_pix        image side, 1 .. 16384
 *   n_angles     projections, 1 .. 16777216 (2^24)
 *   n_det        detector bins per projection, 1 .. 65535
 *   angles       host array of n_angles radians (copied), or NULL for
 *                th_i = i*pi/n_angles
 *   det_spacing  bin width tau in pixel units, > 0
 *   filter       fbp_filter_type
 *   opt          NULL for defaults
 * Errors: FBP_ERR_INVALID_ARG (bad size, non-finite angle, tau <= 0),
 * FBP_ERR_UNSUPPORTED (option combination not built), FBP_ERR_OUT_OF_MEMORY,
 * FBP_ERR_CUDA.  On error *out is NULL.
 */
fbp_status fbp_plan(fbp_plan_t *out, int n_pix, int n_angles, int n_det,
                    const double *angles, double det_spacing,
                    fbp_filter_type filter, const fbp_options *opt);

/* Release the plan's device tables (synchronises the device). NULL is a no-op. */
fbp_status fbp_plan_destroy(fbp_plan_t plan);

/* Bytes of device workspace fbp_reconstruct() needs (the filtered sinogram). */
fbp_status fbp_workspace_bytes(fbp_plan_t plan, size_t *bytes);

/* Resolved choices: row pitch (elements) of the filtered sinogram, FFT length
 * (0 when the FFT route is not used) and filter route.  Any pointer may be NULL. */
fbp_status fbp_plan_query(fbp_plan_t plan, int *q_pitch, int *fft_len, int *filter_path);

/*
 * Ramp filter, Q = P * H (the text after Eq. 2), written in interpolation-ready
 * form for fbp_backproject.
 *   sino      device [n_angles][ld_sino] float, ld_sino >= n_det
 *   filtered  device [n_angles][q_pitch] of the q_storage type (float, or half for
 *             FBP_F16; double for FBP_F64 plans).  Row i holds, for every bin
 *             k = -1 .. n_det-1, a pair at elements 2(k+1) and 2(k+1)+1, with Q_i
 *             zero outside [0, n_det):
 *               FP32/FP16 plans: mid_k = (Q_i[k] + Q_i[k+1]) / 2,
 *                 slope_k = Q_i[k+1] - Q_i[k]  (the interpolant on [k, k+1] is
 *                 mid_k + (u - k - 1/2) slope_k);
 *               FP64 plans: a_k = 2 Q_i[k] - Q_i[k+1], d_k = Q_i[k+1] - Q_i[k]
 *                 (the interpolant is a_k + (1 + u - k) d_k);
 *             elements 2(n_det+1) .. q_pitch-1 are written as zero.
 */
fbp_status fbp_filter(fbp_plan_t plan, const void *sino, int ld_sino, void *filtered,
                      fbp_stream_t stream);

/*
 * Backprojection, Eq. 2: image[r][c] = (pi/A) sum_i lerp(Q_i, u_i(r,c)) with
 * u_i = (x cos th_i + y sin th_i)/tau + (n_det-1)/2, angles summed in order
 * i = 0..A-1 (deterministic: same bits every run).
 *   filtered  device [n_angles][q_pitch] pairs as written by fbp_filter
 *   image     device [n_pix][n_pix] float, written once
 */
fbp_status fbp_backproject(fbp_plan_t plan, const void *filtered, void *image,
                           fbp_stream_t stream);

/*
 * fbp_filter followed by fbp_backproject, the filtered sinogram kept in
 * `workspace` (device, >= fbp_workspace_bytes, 16-byte aligned).
 */
fbp_status fbp_reconstruct(fbp_plan_t plan, const void *sino, int ld_sino, void *image,
                           void *workspace, fbp_stream_t stream);

/*
 * Test-only discrete projector: the exact transpose of the unfiltered
 * backprojection without its pi/A factor,
 *   sino[i][k] = sum_{r,c} image[r][c] * max(0, 1 - |u_i(r,c) - k|),
 * (the projection of section "Computed tomography", Fig. 1).
 *   image  device [n_pix][n_pix] float (F32 plans only)
 *   sino   device [n_angles][n_det] float
 */
fbp_status radon_forward(fbp_plan_t plan, const void *image, void *sino, fbp_stream_t stream);

/* ------------------------------------------------------------------ batches
 * Many slices (any mix of sizes and plans) reconstructed by one captured CUDA
 * graph: every slice's ramp filter, then one persistent backprojection launch
 * per kernel configuration whose work list holds the pixel tiles of all its
 * slices, most angles first.  Each slice goes through the same arithmetic as
 * fbp_reconstruct with its plan, so its image is bit-identical to the one it
 * gets alone.  (The paper reconstructs one image at a time; batching is this
 * library's throughput form of the same Eq. 2.) */
typedef struct fbp_batch_s *fbp_batch_t;

typedef struct {
    const void *sino;  /* device [n_angles][ld_sino] float of that slice */
    int ld_sino;       /* >= n_det */
    void *image;       /* device [n_pix][n_pix] float */
    void *workspace;   /* device, >= fbp_workspace_bytes(plan), 16-byte aligned */
} fbp_batch_io;

/*
 * Build a batch of n (1..64) slices: plans[i] with buffers io[i].  The buffer
 * addresses are bound into the graph: refill the sinogram buffers and call
 * fbp_batch_launch again to reconstruct new data.  The plans and buffers must
 * outlive the batch.  Building allocates a small work list and records the
 * graph (no kernel runs); `stream` is unused and may be NULL.
 * Errors: FBP_ERR_INVALID_ARG, FBP_ERR_ALIGNMENT, FBP_ERR_UNSUPPORTED (FP64
 * plans), FBP_ERR_OUT_OF_MEMORY, FBP_ERR_CUDA.
 */
fbp_status fbp_batch_build(fbp_batch_t *out, const fbp_plan_t *plans, int n,
                           const fbp_batch_io *io, fbp_stream_t stream);

/*
 * The same multi-slice work enqueued directly on `stream` (no graph): every
 * slice's filter, then one persistent backprojection launch per kernel
 * configuration over all tiles.  For work lists that change call to call
 * (the serving loop); allocates nothing.  Images are bit-identical to
 * fbp_reconstruct per slice.  A device timeout is recorded in the status word
 * of plans[0].
 */
fbp_status fbp_reconstruct_many(const fbp_plan_t *plans, int n, const fbp_batch_io *io,
                                fbp_stream_t stream);

/* Parts of a batch graph (fbp_batch_build records both). */
enum { FBP_BATCH_FILTER = 1, FBP_BATCH_BACKPROJECT = 2 };

/* fbp_batch_build recording only the given parts (a bitwise OR of FBP_BATCH_*),
 * e.g. to time the backprojection launch alone over the same buffers. */
fbp_status fbp_batch_build_parts(fbp_batch_t *out, const fbp_plan_t *plans, int n,
                                 const fbp_batch_io *io, int parts, fbp_stream_t stream);

/* Enqueue the whole batch on `stream` (one graph launch).  A batch's launches
 * and fbp_batch_run_host calls share its buffers and the work counters of its
 * backprojection launches: the caller orders them (one stream, or events);
 * different batches may run concurrently. */
fbp_status fbp_batch_launch(fbp_batch_t batch, fbp_stream_t stream);

/* Number of kernel launches one fbp_batch_launch performs (the kernel nodes of
 * the batch's graph), written to *count.  Host-only; no device work.  The
 * paper has no counterpart (it reconstructs one image at a time). */
fbp_status fbp_batch_kernel_count(fbp_batch_t batch, int *count);

/*
 * The batch end to end from host memory: each slice's sinogram (host,
 * [n_angles][n_det] float, contiguous) is copied into the batch's device
 * sinogram buffer, the slice is reconstructed, and its image is copied back to
 * host_images[i] ([n_pix][n_pix] float).  The slices are processed in up to
 * six chunks, pipelined: the sinogram copies run on one internal stream, the
 * image copies on another, the compute alternately on `stream` and a third
 * internal stream, so that chunk c+1 comes in and chunk c-1 goes out while
 * chunk c computes, and consecutive chunks' kernels overlap.  One copy per slice
 * and direction; host buffers should be pinned for the copies to be asynchronous.
 * The work starts after what is already on `stream` and `stream` waits for the
 * last image copy, so synchronising `stream` (or an event recorded on it after
 * this call) makes every image readable.  Results equal those of
 * fbp_batch_launch bit for bit.  Returns after enqueueing.
 */
fbp_status fbp_batch_run_host(fbp_batch_t batch, const void *const *host_sinos,
                              void *const *host_images, fbp_stream_t stream);

/* Read and clear the batch's device status word (synchronises the device). */
fbp_status fbp_batch_status(fbp_batch_t batch);

/* Release the batch (synchronises the device).  NULL is a no-op. */
fbp_status fbp_batch_destroy(fbp_batch_t batch);

/* ------------------------------------------------------------------ serving
 * A request loop for slice reconstructions that arrive over time (the paper's
 * motivation, section "Introduction": a shorter wait for the exam result).
 * A worker thread admits queued requests in arrival order while a device
 * arena of hbm_budget_bytes can hold their sinogram, filtered pairs and image,
 * and launches admitted requests as waves (copies in, every slice's filter,
 * one persistent backprojection over all their tiles, copies out) on up to
 * n_streams streams at once, so requests that arrive while others run are
 * batched and overlap on the device (continuous batching).  The server's
 * plans take the largest backprojection tile that fits (tile_x = tile_y = -1),
 * and each request's image is bit-identical to fbp_reconstruct with such a
 * plan of its geometry.  Latency = submit to the end of its image copy. */
typedef struct fbp_server_s *fbp_server_t;

typedef struct {
    int n_pix, n_angles, n_det;
    double det_spacing;
    int filter;             /* fbp_filter_type */
    const float *host_sino; /* host [n_angles][n_det]; must stay valid until the request is done */
    float *host_image;      /* host [n_pix][n_pix]; written when done (pin both for async copies) */
} fbp_request;

typedef struct {
    long long submitted, completed, failed, admission_stalls, waves;
    int max_waves_in_flight;                /* > 1: waves overlapped on the device */
    double p50_ms, p99_ms, mean_ms, max_ms; /* latency of completed requests */
    double span_s;                          /* first submit to last completion */
    size_t bytes_in_use, peak_bytes, budget_bytes;
} fbp_server_stats;

/* Start a server on the current device: reserves hbm_budget_bytes (>= 1 MiB)
 * of device memory up front; max_wave 1..64 requests per wave; n_streams 1..16. */
fbp_status fbp_server_create(fbp_server_t *out, size_t hbm_budget_bytes, int max_wave,
                             int n_streams);
/* Create the plan of a geometry ahead of traffic (plan creation synchronises the device). */
fbp_status fbp_server_warm(fbp_server_t server, int n_pix, int n_angles, int n_det,
                           double det_spacing, int filter);
/* Queue a request; *id identifies it.  FBP_ERR_INVALID_ARG for a bad geometry or
 * NULL buffer, FBP_ERR_BUDGET if it alone exceeds the budget.  Never blocks on the GPU. */
fbp_status fbp_server_submit(fbp_server_t server, const fbp_request *req, long long *id);
/* Withdraw a request that is still queued (not yet admitted). */
fbp_status fbp_server_cancel(fbp_server_t server, long long id);
/* Block until the request is done; FBP_ERR_TIMEOUT after timeout_s seconds. */
fbp_status fbp_server_wait(fbp_server_t server, long long id, double timeout_s);
/* state: 0 queued, 1 admitted, 2 running, 3 done, 4 failed, 5 cancelled;
 * latency_ms: submit to completion, or -1 if not done.  Either may be NULL. */
fbp_status fbp_server_request_info(fbp_server_t server, long long id, int *state,
                                   double *latency_ms);
/* Block until nothing is queued or running; FBP_ERR_TIMEOUT after timeout_s. */
fbp_status fbp_server_drain(fbp_server_t server, double timeout_s);
fbp_status fbp_server_get_stats(fbp_server_t server, fbp_server_stats *out);
/* Stop the worker, wait for the streams, release plans and the arena. NULL is a no-op. */
fbp_status fbp_server_destroy(fbp_server_t server);

/* ------------------------------------------------------------------ tuning
 * Choice of the filter route (FFT, tensor-core Toeplitz, direct) and of the
 * backprojection launch shape (pixel tile, angles per shared-memory stage) for
 * one geometry, by timing every candidate on the device over `batch` slices.
 * Cached in memory per (GPU model, geometry, base options, batch); when the
 * environment variable FBP_TUNE_CACHE names a file, results are appended to it
 * and read back by later processes.  Plans made with the returned options give
 * the same bits alone, in batches and in the server. */
typedef struct {
    fbp_options options;   /* base options with filter_path, fft_len, tile_x, tile_y,
                              angle_chunk filled in */
    double filter_ms;      /* per slice, best route */
    double backproject_ms; /* per slice, best shape */
    int from_cache;
} fbp_tuning;

/* Tune the geometry (allocates test buffers for `batch` (1..64) slices while it
 * runs; synchronises the device).  base may be NULL (defaults); FP32 only.  A
 * filter_path other than FBP_PATH_AUTO, a tile (tile_x, tile_y) or an
 * angle_chunk set in base is kept, and only the rest is tuned. */
fbp_status fbp_autotune(int n_pix, int n_angles, int n_det, double det_spacing,
                        fbp_filter_type filter, const fbp_options *base, int batch,
                        fbp_tuning *out);

/* ------------------------------------------------------------------ quality
 * PSNR (Eq. 3) and SSIM (Eq. 4) of an image against a reference on the device:
 * the measures the paper compares its reconstructions with (section
 * "Benchmark").  The paper leaves PSNR's MAX and SSIM's window and constants
 * open; here
 *   PSNR = 20 log10(MAX / sqrt(MSE)), MAX = max |reference|, +inf when the
 *          images are identical;
 *   SSIM = mean over every 11 x 11 window inside the image of
 *          (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))
 *          with Gaussian window weights (sigma 1.5, normalised), C1 = (0.01 L)^2,
 *          C2 = (0.03 L)^2 (Wang, Bovik, Sheikh & Simoncelli 2004); L is
 *          dynamic_range, or the reference's max - min when dynamic_range <= 0;
 *          NaN when rows or cols < 11.  The local statistics are FP64 and each
 *          window's value is formed through its distance from 1 (from the
 *          local mean and variance of x - y), so near-identical images keep
 *          1 - SSIM to the precision of their differences and SSIM <= 1.
 * Every sum is taken in a fixed order: the results are the same bits every run. */

/* Device scratch fbp_quality needs for a rows x cols image, in *bytes. */
fbp_status fbp_quality_scratch_bytes(int rows, int cols, size_t *bytes);

/* image, reference: device [rows][ld] float (ld >= cols, 16-byte aligned);
 * scratch: device, >= fbp_quality_scratch_bytes; out: device, 2 doubles,
 * out[0] = PSNR in dB, out[1] = SSIM.  Asynchronous on `stream`; allocates
 * nothing.  FBP_ERR_INVALID_ARG for bad sizes, NULL buffers, a short scratch
 * or a non-finite dynamic_range; FBP_ERR_ALIGNMENT for unaligned buffers. */
fbp_status fbp_quality(const void *image, const void *reference, int rows, int cols, int ld,
                       double dynamic_range, void *scratch, size_t scratch_bytes, double *out,
                       fbp_stream_t stream);

/* ------------------------------------------------------------------ volume
 * A 3D volume from a stack of reconstructed 2D slices by interpolation along z
 * (section "Introduction": 3D CT images from the interpolation of a stack of
 * 2D images; the paper gives no rule, linear interpolation is used):
 *     plane m = (1 - t) S_k + t S_{k+1},  z[k] <= z_out[m] <= z[k+1],
 *     t = (z_out[m] - z[k]) / (z[k+1] - z[k]).
 * slices: host array of n_slices device pointers, each an [n_pix][n_pix]
 * float image (e.g. the images of a batch), 16-byte aligned; z: host,
 * n_slices strictly increasing positions; z_out: host, n_planes positions in
 * [z[0], z[n_slices-1]]; volume: device [n_planes][n_pix][n_pix] float,
 * 16-byte aligned.  Asynchronous on `stream`; allocates nothing.
 * FBP_ERR_INVALID_ARG for NULL/empty inputs, non-increasing z or a plane
 * outside the stack; FBP_ERR_ALIGNMENT for unaligned buffers. */
fbp_status fbp_volume_from_slices(const void *const *slices, int n_slices, const double *z,
                                  int n_pix, const double *z_out, int n_planes, void *volume,
                                  fbp_stream_t stream);

/* ------------------------------------------------------------------ FDK
 * Cone-beam 3D reconstruction by the algorithm of Feldkamp, Davis & Kress
 * (1984), the extension the paper names as its future work (section
 * "Conclusion").  The paper fixes no cone-beam geometry; this library's:
 *   - the source circles the z axis at radius R, at (R cos b, R sin b, 0) for
 *     projection angle b; a full turn (default b_a = 2 pi a / n_angles);
 *   - projections lie on a virtual flat detector through the axis, u along
 *     (-sin b, cos b, 0) and v along z: P[a][i][j] (float, device) at
 *     u_j = (j - (nu-1)/2) du, v_i = (i - (nv-1)/2) dv;
 *   - the volume f[nz][ny][nx] (float, device) has voxel size 1 and voxel
 *     (ix, iy, iz) at (ix - (nx-1)/2, iy - (ny-1)/2, iz - (nz-1)/2); every
 *     voxel must lie more than one unit inside the source circle.
 * Steps: cosine weight R / sqrt(R^2 + u^2 + v^2), ramp filter along u (the
 * filter of Q = P * H with spacing du), then for every voxel the sum over the
 * angles of (R/U)^2 Q(b, R t / U, R z / U) with U = R - (x cos b + y sin b),
 * t = -x sin b + y cos b, bilinear interpolation (zero outside the detector),
 * scaled by pi / n_angles.  As R grows this tends to Eq. 2 applied to each
 * detector row. */
typedef struct fbp_fdk_plan_s *fbp_fdk_plan_t;

typedef struct {
    int n_angles, nv, nu;  /* projections [n_angles][nv][nu] */
    double R;              /* source to rotation axis, in voxel units */
    double du, dv;         /* detector spacing on the virtual detector */
    int nx, ny, nz;        /* volume [nz][ny][nx], each side <= 8192 */
} fbp_fdk_geometry;

/* Plan a geometry (beta: host, n_angles radians, or NULL for a uniform full
 * turn).  FBP_ERR_INVALID_ARG for bad sizes or a volume reaching the source
 * circle; FBP_ERR_UNSUPPORTED beyond the FFT filter's reach (nu > 4096). */
fbp_status fbp_fdk_plan(fbp_fdk_plan_t *out, const fbp_fdk_geometry *geometry,
                        const double *beta, fbp_filter_type filter);
fbp_status fbp_fdk_plan_destroy(fbp_fdk_plan_t plan);
/* Device workspace a reconstruction needs (the filtered rows; the per-tile
 * tables belong to the plan). */
fbp_status fbp_fdk_workspace_bytes(fbp_fdk_plan_t plan, size_t *bytes);
/* proj: device [n_angles][nv][nu] float; volume: device [nz][ny][nx] float;
 * workspace: device, fbp_fdk_workspace_bytes; all 16-byte aligned.
 * Asynchronous on `stream`; deterministic (angles summed in order per voxel). */
fbp_status fbp_fdk_reconstruct(fbp_fdk_plan_t plan, const void *proj, void *volume,
                               void *workspace, fbp_stream_t stream);
/* Synchronise the device and read the plan's device status word (a bounded
 * wait that ran out reports FBP_ERR_TIMEOUT; the word is then cleared). */
fbp_status fbp_fdk_status(fbp_fdk_plan_t plan);

/* Capacity of the scratch array behind fbp_reconstruct_static (bytes). */
#define FBP_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/*
 * fbp_reconstruct for callers that cannot allocate device memory at the time
 * they reconstruct (an acquisition loop with a fixed per-slice deadline cannot
 * absorb the device-wide synchronisation of cudaMalloc/cudaFree; a host whose
 * device memory belongs to another allocator or budget may not allocate at
 * all).  The paper has no counterpart: it is a deployment convenience.
 *
 * Same result as fbp_reconstruct (same kernels, same bits); the filtered
 * sinogram goes to a 256-byte-aligned static device array of
 * FBP_STATIC_SCRATCH_BYTES compiled into the library instead of a caller
 * workspace.  The call makes no cudaMalloc, cudaFree or other allocating call,
 * and loads no code: fbp_plan, which the caller runs once beforehand, loads
 * the plan's kernels and looks up the array's device address on its device
 * (cudaGetSymbolAddress).  Under CUDA's lazy module loading (the default) the
 * array becomes resident on a device at that first fbp_plan, not when the
 * library is loaded, and stays until the process exits.  Each fbp_plan
 * refreshes the address, so plans made after a cudaDeviceReset use the new one.
 *   sino, ld_sino, image  as for fbp_reconstruct (device, caller-owned)
 * Errors: FBP_ERR_BUDGET when the plan's workspace (fbp_workspace_bytes)
 * exceeds FBP_STATIC_SCRATCH_BYTES; FBP_ERR_CUDA if the address could not be
 * looked up when the plan was made; otherwise as fbp_reconstruct.
 * Every call on a device shares the one array and it keeps the last call's
 * contents (nothing in it needs to start at zero: the filter writes every
 * element the backprojection reads), so calls whose GPU work overlaps -- on
 * different streams, or from different threads -- race on it; order them on
 * one stream or serialise them.
 */
fbp_status fbp_reconstruct_static(fbp_plan_t plan, const void *sino, int ld_sino, void *image,
                                  fbp_stream_t stream);

/* Read and clear the plan's device status word (synchronises the device):
 * FBP_OK, or FBP_ERR_TIMEOUT if a bounded device wait ran out since the last read. */
fbp_status fbp_device_status(fbp_plan_t plan);

/* ------------------------------------------------------------------ bounded waits
 * The pipelined kernels (backprojection, tensor-core filter, FDK
 * backprojection) wait on shared-memory barriers; every such wait gives up
 * after a limit, records FBP_ERR_TIMEOUT in the status word of the plan, batch
 * or FDK plan that launched it (fbp_device_status, fbp_batch_status,
 * fbp_fdk_status), and the kernel returns with nothing in flight, leaving the
 * CUDA context usable.  The paper has no counterpart: this is the library's
 * failure detection.  A batch whose status reports a timeout also has its
 * work counters reset by fbp_batch_status, so its next launch is complete. */

/* Set the wait limit, in seconds, for kernels that start after the call on the
 * current device (kernels of CUDA graphs read it when they run, so graphs
 * captured earlier follow it too).  0 restores the default of 2 s; otherwise
 * 1e-6 .. 3600.  Writes device memory (synchronous).  FBP_ERR_INVALID_ARG for
 * a value out of range, FBP_ERR_CUDA without a usable device. */
fbp_status fbp_set_wait_limit(double seconds);

/* TEST ONLY (fault injection without a GPU fault).  With kernel set, the first
 * CTA of every later launch of that kernel kind on the current device
 * withholds the arrival of one pipeline stage (`stage`: the CTA's stage fill
 * count, from 0) and issues no copy for it, so the waits on that stage run out
 * after the wait limit and the launch reports FBP_ERR_TIMEOUT; the image of
 * that launch is then incomplete.  FBP_TEST_WITHHOLD_NONE (stage ignored)
 * switches it off.  Read by kernels when they run, like the wait limit. */
enum {
    FBP_TEST_WITHHOLD_NONE = 0,
    FBP_TEST_WITHHOLD_BACKPROJECT = 1, /* persistent backprojection (single slice and batches) */
    FBP_TEST_WITHHOLD_FILTER_TC = 2    /* tensor-core Toeplitz filter (loader warps' arrival) */
};
fbp_status fbp_test_withhold_arrival(int kernel, int stage);

/* TEST ONLY.  In debug builds compiled with FBP_CHECK_BOUNDS, the index
 * checks of the backprojection and FDK kernels on the current device take
 * their limit as the staged window's width minus `pairs` (0 .. 4096), so a
 * test can make them fire (FBP_ERR_BOUNDS from the next status call); 0 is
 * the true width.  Stored but without effect in normal builds.  Read by
 * kernels when they run.  FBP_ERR_INVALID_ARG for a value out of range. */
fbp_status fbp_test_shrink_window(int pairs);

/* Message of the calling thread's last failed call ("" if none). */
const char *fbp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FBP_H */
