// Autotuner: picks, per geometry ("shape bucket"), the filter route and the
// backprojection launch shape (pixel tile, angles per shared-memory stage) by
// timing them on the device, and caches the choice per GPU model.  A route,
// tile or angle chunk fixed in the base options is kept (only the rest is
// tuned then).
//
// The two kernels are independent, so they are tuned separately: every
// available filter route (FFT, tensor-core Toeplitz, direct) on `batch` slices,
// then every tile x chunk candidate of the backprojection on `batch` slices
// (one persistent launch over all their tiles, as in a batch or a serving
// wave).  Data are zeros: neither kernel's work depends on the values.
// Results are kept in memory and, when FBP_TUNE_CACHE names a file, appended
// to it as one line per bucket and read back by later processes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fbp_internal.h"

using namespace fbp;

namespace {

std::mutex g_mu;
std::map<std::string, fbp_tuning> g_cache;
bool g_file_loaded = false;

std::string gpu_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s = prop.name;
    for (char &c : s)
        if (c == ' ' || c == '|') c = '_';
    return s;
}

std::string bucket_key(int n, int A, int D, double tau, int filter, const fbp_options &b,
                       int batch)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|%d|%d|%.9g|%d|%d|%d|%d|%d|%dx%dx%d|%d|pp%d",
             gpu_name().c_str(), n, A, D, tau, filter, b.dtype, b.q_storage, b.accumulate,
             b.filter_path, b.tile_x, b.tile_y, b.angle_chunk, batch, b.point_pairs);
    return buf;
}

void load_file()
{
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char *path = std::getenv("FBP_TUNE_CACHE");
    if (path == nullptr || *path == 0) return;
    FILE *f = std::fopen(path, "r");
    if (f == nullptr) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[300];
        fbp_tuning t;
        std::memset(&t, 0, sizeof t);
        if (std::sscanf(line, "%299s %d %d %d %d %d %lf %lf", key, &t.options.tile_x,
                        &t.options.tile_y, &t.options.angle_chunk, &t.options.filter_path,
                        &t.options.fft_len, &t.filter_ms, &t.backproject_ms) == 8)
            g_cache[key] = t;
    }
    std::fclose(f);
}

void save_line(const std::string &key, const fbp_tuning &t)
{
    const char *path = std::getenv("FBP_TUNE_CACHE");
    if (path == nullptr || *path == 0) return;
    FILE *f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f, "%s %d %d %d %d %d %.6f %.6f\n", key.c_str(), t.options.tile_x,
                 t.options.tile_y, t.options.angle_chunk, t.options.filter_path,
                 t.options.fft_len, t.filter_ms, t.backproject_ms);
    std::fclose(f);
}

// Median over `reps` timed runs of `batch` slices, in ms per slice.
double time_parts(const Plan *p, const std::vector<fbp_batch_io> &io, int parts, int reps,
                  cudaStream_t s)
{
    const int batch = (int)io.size();
    std::vector<const Plan *> ps((size_t)batch, p);
    // work counters as a batch has them (dynamic item hand-out)
    constexpr int kCounters = 16;
    int *sched = nullptr;
    if (cudaMalloc(&sched, sizeof(int) * 2 * kCounters) != cudaSuccess) return -1.0;
    if (cudaMemset(sched, 0, sizeof(int) * 2 * kCounters) != cudaSuccess ||
        enqueue_many(ps.data(), io.data(), batch, parts, p->d_status, s, sched, kCounters) !=
            cudaSuccess) {
        cudaFree(sched);
        return -1.0;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<double> ms;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        enqueue_many(ps.data(), io.data(), batch, parts, p->d_status, s, sched, kCounters);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        ms.push_back((double)t / batch);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sched);
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

}  // namespace

extern "C" {

fbp_status fbp_autotune(int n_pix, int n_angles, int n_det, double det_spacing,
                        fbp_filter_type filter, const fbp_options *base, int batch,
                        fbp_tuning *out)
{
    if (out == nullptr || batch < 1 || batch > 64) {
        set_error("fbp_autotune: out must not be NULL and batch must be 1..64");
        return FBP_ERR_INVALID_ARG;
    }
    fbp_options b;
    fbp_options_default(&b);
    if (base) b = *base;
    if (b.dtype != FBP_F32) {
        set_error("fbp_autotune: FP32 plans only (the FP64 path has one shape)");
        return FBP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    load_file();
    const std::string key = bucket_key(n_pix, n_angles, n_det, det_spacing, (int)filter, b, batch);
    auto hit = g_cache.find(key);
    if (hit != g_cache.end()) {
        *out = hit->second;
        out->options.dtype = b.dtype;
        out->options.q_storage = b.q_storage;
        out->options.accumulate = b.accumulate;
        out->options.point_pairs = b.point_pairs;
        out->options.i0 = b.i0;
        out->from_cache = 1;
        return FBP_OK;
    }

    // A probe plan fixes the buffer sizes (pitch) and validates the geometry.
    fbp_plan_t probe = nullptr;
    fbp_status st = fbp_plan(&probe, n_pix, n_angles, n_det, nullptr, det_spacing, filter, &b);
    if (st != FBP_OK) return st;
    size_t ws_bytes = 0;
    fbp_workspace_bytes(probe, &ws_bytes);
    fbp_plan_destroy(probe);

    const size_t sino_bytes = sizeof(float) * (size_t)n_angles * (size_t)n_det;
    const size_t img_bytes = sizeof(float) * (size_t)n_pix * (size_t)n_pix;
    const size_t per = ((sino_bytes + 255) & ~(size_t)255) + ((ws_bytes + 255) & ~(size_t)255) +
                       ((img_bytes + 255) & ~(size_t)255);
    char *mem = nullptr;
    if (cudaMalloc(&mem, per * (size_t)batch) != cudaSuccess) {
        set_error("fbp_autotune: cannot allocate %zu bytes of test buffers", per * (size_t)batch);
        return FBP_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(mem, 0, per * (size_t)batch);
    std::vector<fbp_batch_io> io((size_t)batch);
    for (int i = 0; i < batch; ++i) {
        char *m = mem + per * (size_t)i;
        io[(size_t)i].sino = m;
        io[(size_t)i].ld_sino = n_det;
        io[(size_t)i].workspace = m + ((sino_bytes + 255) & ~(size_t)255);
        io[(size_t)i].image = m + ((sino_bytes + 255) & ~(size_t)255) + ((ws_bytes + 255) & ~(size_t)255);
    }
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);

    fbp_tuning best;
    std::memset(&best, 0, sizeof best);
    best.filter_ms = 1e30;
    best.backproject_ms = 1e30;
    const int reps = 3;

    // 1. filter routes
    const int paths[3] = {FBP_PATH_FFT, FBP_PATH_TOEPLITZ_TC, FBP_PATH_DIRECT};
    for (int k = 0; k < 3; ++k) {
        if (b.filter_path != FBP_PATH_AUTO && paths[k] != b.filter_path) continue;
        if (paths[k] == FBP_PATH_TOEPLITZ_TC && b.q_storage != FBP_F32) continue;
        if (paths[k] == FBP_PATH_DIRECT && n_det > 2048) continue;  // O(n_det^2) per row
        fbp_options o = b;
        o.filter_path = paths[k];
        fbp_plan_t pl = nullptr;
        if (fbp_plan(&pl, n_pix, n_angles, n_det, nullptr, det_spacing, filter, &o) != FBP_OK)
            continue;
        const double t = time_parts(reinterpret_cast<const Plan *>(pl), io, FBP_BATCH_FILTER,
                                    reps, s);
        if (t >= 0 && t < best.filter_ms) {
            best.filter_ms = t;
            best.options.filter_path = paths[k];
            best.options.fft_len = reinterpret_cast<const Plan *>(pl)->fft_len;
        }
        fbp_plan_destroy(pl);
    }
    // 2. backprojection shapes
    const int tiles[3][2] = {{32, 64}, {32, 32}, {8, 32}};
    const int chunks[3] = {8, 16, 32};
    for (int ti = 0; ti < 3; ++ti) {
        if (b.tile_x > 0 && (b.tile_x != tiles[ti][0] || b.tile_y != tiles[ti][1])) continue;
        for (int ci = 0; ci < 3; ++ci) {
            if (b.angle_chunk > 0 && b.angle_chunk != chunks[ci]) continue;
            fbp_options o = b;
            o.filter_path = best.options.filter_path ? best.options.filter_path : FBP_PATH_AUTO;
            o.tile_x = tiles[ti][0];
            o.tile_y = tiles[ti][1];
            o.angle_chunk = chunks[ci];
            fbp_plan_t pl = nullptr;
            if (fbp_plan(&pl, n_pix, n_angles, n_det, nullptr, det_spacing, filter, &o) != FBP_OK)
                continue;  // window does not fit this tile
            const double t = time_parts(reinterpret_cast<const Plan *>(pl), io,
                                        FBP_BATCH_BACKPROJECT, reps, s);
            if (t >= 0 && t < best.backproject_ms) {
                best.backproject_ms = t;
                best.options.tile_x = tiles[ti][0];
                best.options.tile_y = tiles[ti][1];
                best.options.angle_chunk = chunks[ci];
            }
            fbp_plan_destroy(pl);
        }
    }
    cudaStreamDestroy(s);
    cudaFree(mem);
    if (best.backproject_ms >= 1e30 || best.filter_ms >= 1e30) {
        set_error("fbp_autotune: no candidate ran for this geometry");
        return FBP_ERR_UNSUPPORTED;
    }
    best.options.dtype = b.dtype;
    best.options.q_storage = b.q_storage;
    best.options.accumulate = b.accumulate;
    best.options.point_pairs = b.point_pairs;
    best.options.i0 = b.i0;
    best.from_cache = 0;
    g_cache[key] = best;
    save_line(key, best);
    *out = best;
    return FBP_OK;
}

}  // extern "C"
