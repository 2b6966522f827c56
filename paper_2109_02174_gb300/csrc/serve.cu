// Serving runtime: continuous batching of slice reconstructions.
//
// The paper's motivation is a shorter wait for the exam result (section
// "Introduction"); here requests (one slice each, any geometry) arrive while
// others are on the GPU.  A worker thread
//   1. retires finished waves (their completion time is stamped on the GPU's
//      stream by a host function) and returns their memory to the arena;
//   2. admits queued requests in arrival order while the device arena, sized
//      to the HBM budget, can hold their sinogram, filtered pairs and image;
//   3. launches admitted requests as a wave on the next free stream: host-to-
//      device copies, every slice's filter, one persistent backprojection
//      launch over all their tiles (fbp_reconstruct_many's path), device-to-
//      host copies of the images.
// Up to n_streams waves are in flight at once, so a new wave's copies and
// kernels overlap the ones still running.  Each slice goes through exactly
// the arithmetic fbp_reconstruct applies with a default plan of its geometry,
// so its image is bit-identical to the one it gets alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "fbp_internal.h"

using namespace fbp;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// First-fit allocator over one device allocation, coalescing on free.
class Arena {
  public:
    bool init(size_t bytes)
    {
        size_ = round256(bytes);
        if (cudaMalloc(&base_, size_) != cudaSuccess) return false;
        free_[0] = size_;
        return true;
    }
    void release()
    {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t next = it->first + bytes;
                free_.erase(it);
                if (rest) free_[next] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void free(size_t off, size_t bytes)
    {
        bytes = round256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *ptr(size_t off) const { return static_cast<char *>(base_) + off; }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum { ST_QUEUED = 0, ST_ADMITTED = 1, ST_RUNNING = 2, ST_DONE = 3, ST_FAILED = 4, ST_CANCELLED = 5 };

struct Req {
    long long id;
    fbp_request r;
    double t_submit = 0, t_done = 0;
    int state = ST_QUEUED;
    bool stalled = false;
    fbp_plan_t plan = nullptr;
    size_t off = 0, bytes = 0;
    size_t sino_off = 0, ws_off = 0, img_off = 0;
};

struct Wave {
    int stream = -1;
    std::vector<Req *> reqs;
    std::atomic<int> done{0};
    double t_done = 0;
    struct fbp_server_s *server = nullptr;
};

using GeomKey = std::tuple<int, int, int, double, int>;

constexpr int kServeCounters = 8;  // backprojection launches of one wave with a work counter

}  // namespace

struct fbp_server_s {
    int device = 0;
    int max_wave = 32;
    int n_streams = 2;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    int *d_sched = nullptr;  // work counters of the backprojection launches, per stream
    std::map<GeomKey, fbp_plan_t> plans;
    std::mutex mu;
    std::condition_variable cv_work;  // worker wake-up
    std::condition_variable cv_done;  // request completions
    std::deque<Req *> pending;        // submitted, not admitted
    std::deque<Req *> ready;          // admitted, not launched
    std::deque<Wave *> inflight;
    std::unordered_map<long long, Req *> reqs;
    long long next_id = 1;
    std::thread worker;
    bool stop = false;
    // statistics
    long long submitted = 0, completed = 0, failed = 0, stalls = 0, waves = 0;
    int max_inflight = 0;
    std::vector<double> latencies_ms;
    double t_first = 0, t_last = 0;
    std::string last_error;
};

namespace {

void CUDART_CB wave_done_cb(void *arg)
{
    Wave *w = static_cast<Wave *>(arg);
    w->t_done = now_s();
    w->done.store(1, std::memory_order_release);
    w->server->cv_work.notify_one();
}

size_t request_bytes(const fbp_request &r, const Plan &p, size_t *sino, size_t *ws, size_t *img)
{
    *sino = round256(sizeof(float) * (size_t)r.n_angles * (size_t)r.n_det);
    *ws = round256((size_t)p.A * (size_t)p.pitch * (size_t)q_elem_bytes(p));
    *img = round256(sizeof(float) * (size_t)r.n_pix * (size_t)r.n_pix);
    return *sino + *ws + *img;
}

// Plan of a geometry (created on first use; plan creation synchronises the device).
fbp_plan_t plan_for(fbp_server_s *s, const fbp_request &r)
{
    const GeomKey key(r.n_pix, r.n_angles, r.n_det, r.det_spacing, r.filter);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) return it->second;
    // The largest backprojection tile that fits (tile -1), not the one-slice
    // default: a wave holds several requests and makes one launch per tile
    // shape, and the largest tile costs least per pixel.
    fbp_options o;
    fbp_options_default(&o);
    o.tile_x = o.tile_y = -1;
    fbp_plan_t p = nullptr;
    if (fbp_plan(&p, r.n_pix, r.n_angles, r.n_det, nullptr, r.det_spacing,
                 (fbp_filter_type)r.filter, &o) != FBP_OK)
        return nullptr;
    s->plans[key] = p;
    return p;
}

void finish_wave(fbp_server_s *s, Wave *w, bool ok)
{
    for (Req *q : w->reqs) {
        q->state = ok ? ST_DONE : ST_FAILED;
        q->t_done = w->t_done;
        s->arena.free(q->off, q->bytes);
        if (ok) {
            ++s->completed;
            s->latencies_ms.push_back(1e3 * (q->t_done - q->t_submit));
            s->t_last = std::max(s->t_last, q->t_done);
        } else {
            ++s->failed;
        }
    }
    if (w->stream >= 0) s->stream_busy[(size_t)w->stream] = false;
    delete w;
}

// One wave on stream `si`: copies in, filters + one persistent backprojection, copies out.
bool launch_wave(fbp_server_s *s, Wave *w, int si)
{
    cudaStream_t st = s->streams[(size_t)si];
    w->stream = si;
    w->server = s;
    const int n = (int)w->reqs.size();
    std::vector<const Plan *> ps((size_t)n);
    std::vector<fbp_batch_io> io((size_t)n);
    for (int i = 0; i < n; ++i) {
        Req *q = w->reqs[(size_t)i];
        const Plan *p = reinterpret_cast<const Plan *>(q->plan);
        ps[(size_t)i] = p;
        io[(size_t)i].sino = s->arena.ptr(q->sino_off);
        io[(size_t)i].ld_sino = q->r.n_det;
        io[(size_t)i].image = s->arena.ptr(q->img_off);
        io[(size_t)i].workspace = s->arena.ptr(q->ws_off);
        if (cudaMemcpyAsync(s->arena.ptr(q->sino_off), q->r.host_sino,
                            sizeof(float) * (size_t)q->r.n_angles * (size_t)q->r.n_det,
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return false;
        q->state = ST_RUNNING;
    }
    // the stream's work counters start each wave at zero (a wave that gave up
    // may have left them elsewhere)
    int *sched = s->d_sched + 2 * kServeCounters * si;
    if (cudaMemsetAsync(sched, 0, sizeof(int) * 2 * kServeCounters, st) != cudaSuccess)
        return false;
    if (enqueue_many(ps.data(), io.data(), n, FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT,
                     ps[0]->d_status, st, sched, kServeCounters) != cudaSuccess)
        return false;
    for (int i = 0; i < n; ++i) {
        Req *q = w->reqs[(size_t)i];
        if (cudaMemcpyAsync(q->r.host_image, s->arena.ptr(q->img_off),
                            sizeof(float) * (size_t)q->r.n_pix * (size_t)q->r.n_pix,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return false;
    }
    return cudaLaunchHostFunc(st, wave_done_cb, w) == cudaSuccess;
}

void worker_main(fbp_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progressed = false;
        // 1. retire finished waves
        for (auto it = s->inflight.begin(); it != s->inflight.end();) {
            if ((*it)->done.load(std::memory_order_acquire)) {
                finish_wave(s, *it, true);
                it = s->inflight.erase(it);
                progressed = true;
            } else {
                ++it;
            }
        }
        if (progressed) s->cv_done.notify_all();
        // 2. admit in arrival order while the arena has room
        if (!s->pending.empty()) nvtxRangePushA("serving admission");
        const bool admitting = !s->pending.empty();
        while (!s->pending.empty()) {
            Req *q = s->pending.front();
            if (q->state == ST_CANCELLED) {
                s->pending.pop_front();
                continue;
            }
            size_t off = 0;
            if (!s->arena.alloc(q->bytes, &off)) {
                if (!q->stalled) {
                    q->stalled = true;
                    ++s->stalls;
                }
                break;
            }
            q->off = off;
            q->sino_off += off;
            q->ws_off += off;
            q->img_off += off;
            q->state = ST_ADMITTED;
            s->pending.pop_front();
            s->ready.push_back(q);
            progressed = true;
        }
        if (admitting) nvtxRangePop();
        // 3. launch waves on free streams
        while (!s->ready.empty()) {
            int si = -1;
            for (int k = 0; k < s->n_streams; ++k)
                if (!s->stream_busy[(size_t)k]) {
                    si = k;
                    break;
                }
            if (si < 0) break;
            Wave *w = new Wave();
            while (!s->ready.empty() && (int)w->reqs.size() < s->max_wave) {
                w->reqs.push_back(s->ready.front());
                s->ready.pop_front();
            }
            s->stream_busy[(size_t)si] = true;
            ++s->waves;
            bool launched;
            {
                NvtxRange range("serving wave launch");
                launched = launch_wave(s, w, si);
            }
            if (!launched) {
                s->last_error = cudaGetErrorString(cudaGetLastError());
                // work already enqueued may still touch the wave's memory
                cudaStreamSynchronize(s->streams[(size_t)si]);
                w->t_done = now_s();
                finish_wave(s, w, false);
                s->cv_done.notify_all();
            } else {
                s->inflight.push_back(w);
                s->max_inflight = std::max(s->max_inflight, (int)s->inflight.size());
            }
            progressed = true;
        }
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return (i + 1 < v.size()) ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

fbp_status fbp_server_create(fbp_server_t *out, size_t hbm_budget_bytes, int max_wave,
                             int n_streams)
{
    if (out == nullptr) {
        set_error("fbp_server_create: out is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (hbm_budget_bytes < (1u << 20) || max_wave < 1 || max_wave > 64 || n_streams < 1 ||
        n_streams > 16) {
        set_error("fbp_server_create: budget >= 1 MiB, max_wave 1..64, n_streams 1..16");
        return FBP_ERR_INVALID_ARG;
    }
    fbp_server_s *s = new fbp_server_s();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        set_error("fbp_server_create: no CUDA device");
        return FBP_ERR_CUDA;
    }
    s->max_wave = max_wave;
    s->n_streams = n_streams;
    if (!s->arena.init(hbm_budget_bytes)) {
        delete s;
        set_error("fbp_server_create: cannot reserve %zu bytes of device memory",
                  hbm_budget_bytes);
        return FBP_ERR_OUT_OF_MEMORY;
    }
    const size_t sched_bytes = sizeof(int) * 2 * kServeCounters * (size_t)n_streams;
    if (cudaMalloc(&s->d_sched, sched_bytes) != cudaSuccess ||
        cudaMemset(s->d_sched, 0, sched_bytes) != cudaSuccess) {
        s->arena.release();
        cudaFree(s->d_sched);
        delete s;
        set_error("fbp_server_create: cannot allocate the work counters");
        return FBP_ERR_OUT_OF_MEMORY;
    }
    for (int k = 0; k < n_streams; ++k) {
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        s->streams.push_back(st);
        s->stream_busy.push_back(false);
    }
    s->worker = std::thread(worker_main, s);
    *out = reinterpret_cast<fbp_server_t>(s);
    return FBP_OK;
}

fbp_status fbp_server_warm(fbp_server_t server, int n_pix, int n_angles, int n_det,
                           double det_spacing, int filter)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) {
        set_error("fbp_server_warm: server is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    fbp_request r;
    std::memset(&r, 0, sizeof r);
    r.n_pix = n_pix;
    r.n_angles = n_angles;
    r.n_det = n_det;
    r.det_spacing = det_spacing;
    r.filter = filter;
    std::lock_guard<std::mutex> lk(s->mu);
    return plan_for(s, r) ? FBP_OK : FBP_ERR_INVALID_ARG;
}

fbp_status fbp_server_submit(fbp_server_t server, const fbp_request *req, long long *id)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr || req == nullptr || id == nullptr) {
        set_error("fbp_server_submit: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    if (req->host_sino == nullptr || req->host_image == nullptr) {
        set_error("fbp_server_submit: NULL host buffer");
        return FBP_ERR_INVALID_ARG;
    }
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    fbp_plan_t p = plan_for(s, *req);
    if (p == nullptr) return FBP_ERR_INVALID_ARG;  // fbp_plan set the message
    const Plan &pl = *reinterpret_cast<const Plan *>(p);
    if (pl.dtype != FBP_F32) {
        set_error("fbp_server_submit: FP32 requests only");
        return FBP_ERR_UNSUPPORTED;
    }
    Req *q = new Req();
    q->r = *req;
    q->plan = p;
    size_t a, b, c;
    q->bytes = request_bytes(*req, pl, &a, &b, &c);
    q->sino_off = 0;
    q->ws_off = a;
    q->img_off = a + b;
    if (q->bytes > s->arena.size()) {
        delete q;
        set_error("fbp_server_submit: request needs %zu bytes, the budget is %zu", q->bytes,
                  s->arena.size());
        return FBP_ERR_BUDGET;
    }
    q->id = s->next_id++;
    q->t_submit = t;
    if (s->submitted == 0) s->t_first = t;
    ++s->submitted;
    s->reqs[q->id] = q;
    s->pending.push_back(q);
    *id = q->id;
    s->cv_work.notify_one();
    return FBP_OK;
}

fbp_status fbp_server_cancel(fbp_server_t server, long long id)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) {
        set_error("fbp_server_cancel: server is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_error("fbp_server_cancel: unknown request %lld", id);
        return FBP_ERR_INVALID_ARG;
    }
    if (it->second->state != ST_QUEUED) {
        set_error("fbp_server_cancel: request %lld is already admitted", id);
        return FBP_ERR_INVALID_ARG;
    }
    it->second->state = ST_CANCELLED;
    s->cv_done.notify_all();
    return FBP_OK;
}

fbp_status fbp_server_wait(fbp_server_t server, long long id, double timeout_s)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) {
        set_error("fbp_server_wait: server is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_error("fbp_server_wait: unknown request %lld", id);
        return FBP_ERR_INVALID_ARG;
    }
    Req *q = it->second;
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (q->state < ST_DONE) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && q->state < ST_DONE) {
            set_error("fbp_server_wait: request %lld not done after %.3f s", id, timeout_s);
            return FBP_ERR_TIMEOUT;
        }
    }
    if (q->state == ST_FAILED) {
        set_error("fbp_server_wait: request %lld failed (%s)", id, s->last_error.c_str());
        return FBP_ERR_CUDA;
    }
    if (q->state == ST_CANCELLED) {
        set_error("fbp_server_wait: request %lld was cancelled", id);
        return FBP_ERR_INVALID_ARG;
    }
    return FBP_OK;
}

fbp_status fbp_server_request_info(fbp_server_t server, long long id, int *state,
                                   double *latency_ms)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) {
        set_error("fbp_server_request_info: server is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_error("fbp_server_request_info: unknown request %lld", id);
        return FBP_ERR_INVALID_ARG;
    }
    if (state) *state = it->second->state;
    if (latency_ms)
        *latency_ms = it->second->state == ST_DONE
                          ? 1e3 * (it->second->t_done - it->second->t_submit)
                          : -1.0;
    return FBP_OK;
}

fbp_status fbp_server_drain(fbp_server_t server, double timeout_s)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) {
        set_error("fbp_server_drain: server is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    auto busy = [&]() {
        for (Req *q : s->pending)
            if (q->state != ST_CANCELLED) return true;
        return !s->ready.empty() || !s->inflight.empty();
    };
    while (busy()) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && busy()) {
            set_error("fbp_server_drain: work left after %.3f s", timeout_s);
            return FBP_ERR_TIMEOUT;
        }
    }
    return FBP_OK;
}

fbp_status fbp_server_get_stats(fbp_server_t server, fbp_server_stats *out)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr || out == nullptr) {
        set_error("fbp_server_get_stats: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->admission_stalls = s->stalls;
    out->waves = s->waves;
    out->max_waves_in_flight = s->max_inflight;
    out->p50_ms = percentile(s->latencies_ms, 0.50);
    out->p99_ms = percentile(s->latencies_ms, 0.99);
    double sum = 0, mx = 0;
    for (double v : s->latencies_ms) {
        sum += v;
        mx = std::max(mx, v);
    }
    out->mean_ms = s->latencies_ms.empty() ? 0.0 : sum / (double)s->latencies_ms.size();
    out->max_ms = mx;
    out->span_s = s->completed ? s->t_last - s->t_first : 0.0;
    out->bytes_in_use = s->arena.used();
    out->peak_bytes = s->arena.peak();
    out->budget_bytes = s->arena.size();
    return FBP_OK;
}

fbp_status fbp_server_destroy(fbp_server_t server)
{
    fbp_server_s *s = reinterpret_cast<fbp_server_s *>(server);
    if (s == nullptr) return FBP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (Wave *w : s->inflight) delete w;
    for (auto &kv : s->reqs) delete kv.second;
    for (auto &kv : s->plans) fbp_plan_destroy(kv.second);
    s->arena.release();
    cudaFree(s->d_sched);
    delete s;
    return FBP_OK;
}

}  // extern "C"
