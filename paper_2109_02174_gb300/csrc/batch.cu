// Batched reconstruction of many slices (possibly of different sizes) as one
// CUDA graph: each slice's ramp filter, then ONE persistent backprojection
// launch per kernel configuration whose work list holds the tiles of all
// slices, costliest first.  Every slice goes through the same arithmetic as
// fbp_reconstruct with its plan (same tile shape, same window, same angle
// order), so its image is bit-identical to the one it gets alone.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include "backproject.cuh"
#include "fbp_internal.h"
#include "filter_tc.cuh"

namespace fbp {
BpSlice slice_desc(const Plan &p, float *image);
int items_of(const Plan &p);
BpConfig bp_config(const Plan &p);
}  // namespace fbp

using namespace fbp;

// Chunks of a batch's slices that fbp_batch_run_host pipelines: while chunk c
// computes, chunk c+1's sinograms come in and chunk c-1's images go out, and
// consecutive chunks compute on alternate streams, so that a chunk's launches
// take the SMs the previous chunk's last work items leave idle.  Only the
// first chunk's copy in and the last chunk's copy out are not hidden, so the
// chunks taper at both ends: 1/32, 3/32, 3/8, 3/8, 3/32, 1/32 of the slices,
// on even slice counts (two slices of one plan share a backprojection work
// item), at least two slices each.  Each chunk's copy in (a sinogram copies in
// four times faster than it computes) hides behind the previous chunk's
// compute.  Measured on 64 slices of 512x512, 720 angles, 725 bins, end to
// end: 2/6/24/24/6/2 slices per chunk 21.3k slices/s; 2/14/32/14/2 20.8k;
// eight chunks 2/4/10/16/16/10/4/2 21.3k; 4/12/32/12/4 on one stream with
// static work items 20.0k.
constexpr int kRunHostChunks = 6;

// Slice index where chunk c begins (c = 0..chunks), for n slices.
int chunk_begin(int n, int chunks, int c)
{
    if (chunks == kRunHostChunks) {
        static const int at[kRunHostChunks + 1] = {0, 2, 8, 32, 56, 62, 64};  // 64ths
        if (c == 0) return 0;
        if (c == chunks) return n;
        int b = 2 * ((n * at[c] + 64) / 128);  // nearest even count
        if (b < 2 * c) b = 2 * c;
        if (b > n - 2 * (chunks - c)) b = n - 2 * (chunks - c);
        return b;
    }
    return (int)((long long)n * c / chunks);
}

// Work counters of the backprojection launches (dynamic item hand-out): one
// set per compute stream a batch uses, one counter per launch of a set.
constexpr int kSchedSets = 2;
constexpr int kSchedPerSet = 16;

struct fbp_batch_s {
    int device;
    int n;
    std::vector<const Plan *> plans;
    std::vector<fbp_batch_io> io;
    int *d_status;
    int *d_sched;  // [kSchedSets][kSchedPerSet][2], zero between launches
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long updates;
    int parts;
    // fbp_batch_run_host pipeline (created on first use): a stream for the
    // sinogram copies, one for the image copies, a second compute stream
    // beside the caller's, and the events that order them.
    cudaStream_t s_in;
    cudaStream_t s_out;
    cudaStream_t s_comp;
    cudaEvent_t ev_start;
    cudaEvent_t ev_out;
    cudaEvent_t ev_in[kRunHostChunks];
    cudaEvent_t ev_done[kRunHostChunks];
};

namespace {

void free_batch(fbp_batch_s *b)
{
    if (b == nullptr) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->s_in) cudaStreamDestroy(b->s_in);
    if (b->s_out) cudaStreamDestroy(b->s_out);
    if (b->s_comp) cudaStreamDestroy(b->s_comp);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    for (int c = 0; c < kRunHostChunks; ++c) {
        if (b->ev_in[c]) cudaEventDestroy(b->ev_in[c]);
        if (b->ev_done[c]) cudaEventDestroy(b->ev_done[c]);
    }
    cudaFree(b->d_status);
    cudaFree(b->d_sched);
    delete b;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace fbp {

// Every slice's filter, then one persistent backprojection launch per kernel
// configuration and item size over the tiles of all slices of that
// configuration (slices with the most angles first).  The k-th backprojection
// launch takes work counter k of `sched` and hands out its items dynamically;
// launches beyond the n_sched counters stride statically.
cudaError_t enqueue_many(const Plan *const *plans, const fbp_batch_io *io, int n, int parts,
                         int *status, cudaStream_t s, int *sched, int n_sched,
                         const BpFork *fork)
{
    if (parts & FBP_BATCH_FILTER) {
        // FFT-route slices: one launch over all their row pairs
        std::vector<const float *> sinos((size_t)n);
        std::vector<int> lds((size_t)n);
        std::vector<void *> qs((size_t)n);
        for (int i = 0; i < n; ++i) {
            sinos[(size_t)i] = static_cast<const float *>(io[i].sino);
            lds[(size_t)i] = io[i].ld_sino;
            qs[(size_t)i] = io[i].workspace;
        }
        cudaError_t e = launch_filter_fft_many(plans, sinos.data(), lds.data(), qs.data(), n, s);
        if (e != cudaSuccess) return e;
        // Toeplitz-route slices: one launch per plan (they share its T tables)
        std::map<const Plan *, std::vector<int>> by_plan;
        for (int i = 0; i < n; ++i)
            if (plans[i]->filter_path == FBP_PATH_TOEPLITZ_TC) by_plan[plans[i]].push_back(i);
        for (auto &kv : by_plan) {
            std::vector<const float *> ss;
            std::vector<int> ll;
            std::vector<float *> qq;
            for (int i : kv.second) {
                ss.push_back(sinos[(size_t)i]);
                ll.push_back(lds[(size_t)i]);
                qq.push_back(static_cast<float *>(qs[(size_t)i]));
            }
            e = launch_filter_tc_many(*kv.first, ss.data(), ll.data(), qq.data(),
                                      (int)ss.size(), s);
            if (e != cudaSuccess) return e;
        }
        for (int i = 0; i < n; ++i) {
            const Plan &p = *plans[i];
            if (p.filter_path != FBP_PATH_DIRECT) continue;
            e = launch_filter_direct(p, sinos[(size_t)i], lds[(size_t)i], qs[(size_t)i], s);
            if (e != cudaSuccess) return e;
        }
    }
    if (!(parts & FBP_BATCH_BACKPROJECT)) return cudaSuccess;
    std::map<std::tuple<int, int, int, int>, std::vector<int>> by_cfg;
    for (int i = 0; i < n; ++i) {
        const BpConfig c = bp_config(*plans[i]);
        by_cfg[std::make_tuple(c.wx, c.wy, (int)c.half_pairs,
                               (int)c.kahan + 2 * (int)c.point_pairs)].push_back(i);
    }
    std::unique_ptr<BpLaunch<kBpMaxSlices>> L(new BpLaunch<kBpMaxSlices>());
    int launches = 0;
    bool forked = false;
    if (fork != nullptr) {
        cudaError_t e = cudaEventRecord(fork->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->side, fork->fork, 0);
        if (e != cudaSuccess) return e;
        forked = true;
    }
    for (auto &kv : by_cfg) {
        std::vector<int> members = kv.second;
        std::stable_sort(members.begin(), members.end(),
                         [&](int a, int c) { return plans[a]->A > plans[c]->A; });
        const BpConfig cfg = bp_config(*plans[members[0]]);
        // Slices of one plan share every index computation: pair them into
        // two-slice items (not Kahan sums of FP16 pairs); the rest stay
        // single.  Plans with point-symmetric tile pairs share it within each
        // slice instead.
        const bool two = !(cfg.kahan && cfg.half_pairs) && !cfg.point_pairs;
        std::vector<std::pair<int, int>> pairs;
        std::vector<int> singles;
        if (two) {
            std::map<const Plan *, std::vector<int>> by_plan;
            for (int i : members) by_plan[plans[i]].push_back(i);
            std::vector<bool> paired((size_t)n, false);
            for (int i : members) {
                if (paired[(size_t)i]) continue;
                std::vector<int> &same = by_plan[plans[i]];
                int mate = -1;
                for (int j : same)
                    if (j != i && !paired[(size_t)j]) {
                        mate = j;
                        break;
                    }
                if (mate >= 0) {
                    paired[(size_t)i] = paired[(size_t)mate] = true;
                    pairs.push_back(std::make_pair(i, mate));
                } else {
                    singles.push_back(i);
                }
            }
        } else {
            singles = members;
        }
        // Work-list entries: (slice, partner or -1).  Pairing configurations
        // put the pairs and the odd slices out into one two-slice launch (a
        // single slice stages one row per angle there), most angles first;
        // the others launch single-slice items.
        std::vector<std::pair<int, int>> entries = pairs;
        for (int i : singles) entries.push_back(std::make_pair(i, -1));
        std::stable_sort(entries.begin(), entries.end(),
                         [&](const std::pair<int, int> &a, const std::pair<int, int> &c) {
                             return plans[a.first]->A > plans[c.first]->A;
                         });
        const int group = two ? 2 : 1;
        const int count = (int)entries.size();
        for (int b = 0; b < count; b += kBpMaxSlices) {
            const int cnt = std::min(kBpMaxSlices, count - b);
            std::memset(L.get(), 0, sizeof(*L));
            int acc = 0;
            for (int m = 0; m < cnt; ++m) {
                const int i = entries[(size_t)(b + m)].first;
                const int j = entries[(size_t)(b + m)].second;
                const Plan &p = *plans[i];
                if (!encode_pairs_map(p, io[i].workspace, &L->maps[group * m]))
                    return cudaErrorInvalidValue;
                L->slices[m] = slice_desc(p, static_cast<float *>(io[i].image));
                if (j >= 0) {
                    if (!encode_pairs_map(*plans[j], io[j].workspace, &L->maps[2 * m + 1]))
                        return cudaErrorInvalidValue;
                    L->slices[m].image2 = static_cast<float *>(io[j].image);
                }
                acc += items_of(p);
                L->tile_end[m] = acc;
                L->wp_max = std::max(L->wp_max, p.bp_wp);
            }
            L->n_slices = cnt;
            L->n_items = acc;
            L->status = status;
            L->sched = (sched != nullptr && launches < n_sched) ? sched + 2 * launches : nullptr;
            ++launches;
            BpConfig c = cfg;
            c.group = group;
            // single-slice launches run beside the two-slice ones
            const bool on_side = forked && group == 1;
            cudaError_t e = launch_backproject_batch(*L, c, 0, on_side ? fork->side : s);
            if (e != cudaSuccess) return e;
        }
    }
    if (forked) {
        // the main stream waits for the side stream (also when it ran nothing,
        // so a captured fork always joins)
        cudaError_t e = cudaEventRecord(fork->join, fork->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->join, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Host-side checks shared by the batch calls.
fbp_status check_many(const char *fn, const fbp_plan_t *plans, int n, const fbp_batch_io *io,
                      int dev)
{
    if (plans == nullptr || io == nullptr || n < 1 || n > kBpMaxSlices) {
        set_error("%s: need 1..%d slices with plans and buffers (got %d)", fn, kBpMaxSlices, n);
        return FBP_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        const fbp_batch_io &b = io[i];
        if (p == nullptr || p->device != dev) {
            set_error("%s: slice %d: NULL plan or plan of another device", fn, i);
            return FBP_ERR_INVALID_ARG;
        }
        if (p->dtype != FBP_F32) {
            set_error("%s: slice %d: only FP32 plans batch", fn, i);
            return FBP_ERR_UNSUPPORTED;
        }
        if (!b.sino || !b.image || !b.workspace || b.ld_sino < p->D) {
            set_error("%s: slice %d: NULL buffer or ld_sino < n_det", fn, i);
            return FBP_ERR_INVALID_ARG;
        }
        if (!aligned16(b.sino) || !aligned16(b.image) || !aligned16(b.workspace)) {
            set_error("%s: slice %d: buffer not 16-byte aligned", fn, i);
            return FBP_ERR_ALIGNMENT;
        }
    }
    return FBP_OK;
}

}  // namespace fbp

extern "C" {

fbp_status fbp_batch_build(fbp_batch_t *out, const fbp_plan_t *plans, int n,
                           const fbp_batch_io *io, fbp_stream_t stream)
{
    return fbp_batch_build_parts(out, plans, n, io, FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT,
                                 stream);
}

fbp_status fbp_batch_build_parts(fbp_batch_t *out, const fbp_plan_t *plans, int n,
                                 const fbp_batch_io *io, int parts, fbp_stream_t stream)
{
    if (out == nullptr) {
        set_error("fbp_batch_build: out is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    if (parts <= 0 || (parts & ~(FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT)) != 0) {
        set_error("fbp_batch_build: parts %d is not a combination of FBP_BATCH_* flags", parts);
        return FBP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("fbp_batch_build: no current CUDA device");
        return FBP_ERR_CUDA;
    }
    fbp_status st = check_many("fbp_batch_build", plans, n, io, dev);
    if (st != FBP_OK) return st;

    fbp_batch_s *b = new fbp_batch_s();
    b->device = dev;
    b->n = n;
    b->d_status = nullptr;
    b->d_sched = nullptr;
    b->graph = nullptr;
    b->exec = nullptr;
    b->updates = 0;
    b->parts = parts;
    for (int i = 0; i < n; ++i) {
        b->plans.push_back(reinterpret_cast<const Plan *>(plans[i]));
        b->io.push_back(io[i]);
        b->updates += (long long)b->plans.back()->n * b->plans.back()->n * b->plans.back()->A;
    }
    const size_t sched_bytes = sizeof(int) * 2 * kSchedSets * kSchedPerSet;
    cudaError_t e = cudaMalloc(&b->d_status, sizeof(int) * kStatusWords);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int) * kStatusWords);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sched, sched_bytes);
    if (e == cudaSuccess) e = cudaMemset(b->d_sched, 0, sched_bytes);
    if (e != cudaSuccess) {
        free_batch(b);
        set_error("fbp_batch_build: %s", cudaGetErrorString(e));
        return FBP_ERR_OUT_OF_MEMORY;
    }

    // Capture the whole batch once into a graph on a private stream, the
    // single-slice-item backprojection launches (Kahan and point-pair
    // configurations) on a forked branch.
    cudaStream_t cs = nullptr;
    BpFork fork = {nullptr, nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&fork.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = enqueue_many(b->plans.data(), b->io.data(), n, parts, b->d_status, cs,
                                      b->d_sched, kSchedPerSet, &fork);
        cudaError_t ee = cudaStreamEndCapture(cs, &b->graph);
        e = (le != cudaSuccess) ? le : ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (fork.side) cudaStreamDestroy(fork.side);
    if (fork.fork) cudaEventDestroy(fork.fork);
    if (fork.join) cudaEventDestroy(fork.join);
    if (e != cudaSuccess) {
        free_batch(b);
        set_error("fbp_batch_build: graph capture: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    (void)stream;
    *out = reinterpret_cast<fbp_batch_t>(b);
    return FBP_OK;
}

fbp_status fbp_reconstruct_many(const fbp_plan_t *plans, int n, const fbp_batch_io *io,
                                fbp_stream_t stream)
{
    NvtxRange range("fbp_reconstruct_many");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("fbp_reconstruct_many: no current CUDA device");
        return FBP_ERR_CUDA;
    }
    fbp_status st = check_many("fbp_reconstruct_many", plans, n, io, dev);
    if (st != FBP_OK) return st;
    std::vector<const Plan *> ps((size_t)n);
    for (int i = 0; i < n; ++i) ps[(size_t)i] = reinterpret_cast<const Plan *>(plans[i]);
    cudaError_t e = enqueue_many(ps.data(), io, n, FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT,
                                 ps[0]->d_status, stream, nullptr, 0);
    if (e == cudaErrorInvalidValue) return FBP_ERR_CUDA;  // tensor map (message set)
    if (e != cudaSuccess) {
        set_error("fbp_reconstruct_many: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_batch_launch(fbp_batch_t batch, fbp_stream_t stream)
{
    NvtxRange range("fbp_batch_launch (graph replay)");
    fbp_batch_s *b = reinterpret_cast<fbp_batch_s *>(batch);
    if (b == nullptr) {
        set_error("fbp_batch_launch: batch is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, stream);
    if (e != cudaSuccess) {
        set_error("fbp_batch_launch: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_batch_run_host(fbp_batch_t batch, const void *const *host_sinos,
                              void *const *host_images, fbp_stream_t stream)
{
    NvtxRange range("fbp_batch_run_host");
    fbp_batch_s *b = reinterpret_cast<fbp_batch_s *>(batch);
    if (b == nullptr || host_sinos == nullptr || host_images == nullptr) {
        set_error("fbp_batch_run_host: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    for (int i = 0; i < b->n; ++i) {
        if (host_sinos[i] == nullptr || host_images[i] == nullptr) {
            set_error("fbp_batch_run_host: slice %d: NULL host buffer", i);
            return FBP_ERR_INVALID_ARG;
        }
    }
    cudaError_t e = cudaSuccess;
    if (b->s_in == nullptr) {
        e = cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->s_comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
        for (int c = 0; c < kRunHostChunks && e == cudaSuccess; ++c) {
            e = cudaEventCreateWithFlags(&b->ev_in[c], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            set_error("fbp_batch_run_host: stream/event setup: %s", cudaGetErrorString(e));
            return FBP_ERR_CUDA;
        }
    }
    const int chunks = b->n >= 16 ? kRunHostChunks : (b->n >= 4 ? 2 : 1);
    // The copies of this call start after everything already on `stream`
    // (the previous call's compute still reads these device buffers).
    e = cudaEventRecord(b->ev_start, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_in, b->ev_start, 0);
    for (int c = 0; c < chunks && e == cudaSuccess; ++c) {
        const int lo = chunk_begin(b->n, chunks, c);
        const int hi = chunk_begin(b->n, chunks, c + 1);
        for (int i = lo; i < hi && e == cudaSuccess; ++i) {
            const Plan &p = *b->plans[(size_t)i];
            const fbp_batch_io &io = b->io[(size_t)i];
            const size_t row = sizeof(float) * (size_t)p.D;
            if (io.ld_sino == p.D)
                e = cudaMemcpyAsync(const_cast<void *>(io.sino), host_sinos[i], row * (size_t)p.A,
                                    cudaMemcpyHostToDevice, b->s_in);
            else
                e = cudaMemcpy2DAsync(const_cast<void *>(io.sino), sizeof(float) * io.ld_sino,
                                      host_sinos[i], row, row, p.A, cudaMemcpyHostToDevice, b->s_in);
        }
        // consecutive chunks compute on alternate streams, each with its own
        // work counters, so one chunk's launches start in the SMs the
        // previous chunk's last work items leave idle
        cudaStream_t cs = (c & 1) ? b->s_comp : stream;
        int *sched = b->d_sched + 2 * kSchedPerSet * (c & 1);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_in[c], b->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->ev_in[c], 0);
        if (e == cudaSuccess)
            e = enqueue_many(b->plans.data() + lo, b->io.data() + lo, hi - lo, b->parts,
                             b->d_status, cs, sched, kSchedPerSet);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_done[c], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_out, b->ev_done[c], 0);
        for (int i = lo; i < hi && e == cudaSuccess; ++i) {
            const Plan &p = *b->plans[(size_t)i];
            e = cudaMemcpyAsync(host_images[i], b->io[(size_t)i].image,
                                sizeof(float) * (size_t)p.n * (size_t)p.n, cudaMemcpyDeviceToHost,
                                b->s_out);
        }
    }
    // `stream` is done with this call once the last image copy is.
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->ev_out, 0);
    if (e != cudaSuccess) {
        set_error("fbp_batch_run_host: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_batch_kernel_count(fbp_batch_t batch, int *count)
{
    fbp_batch_s *b = reinterpret_cast<fbp_batch_s *>(batch);
    if (b == nullptr || count == nullptr) {
        set_error("fbp_batch_kernel_count: NULL argument");
        return FBP_ERR_INVALID_ARG;
    }
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(b->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n > 0) e = cudaGraphGetNodes(b->graph, nodes.data(), &n);
    int kernels = 0;
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    if (e != cudaSuccess) {
        set_error("fbp_batch_kernel_count: %s", cudaGetErrorString(e));
        return FBP_ERR_CUDA;
    }
    *count = kernels;
    return FBP_OK;
}

fbp_status fbp_batch_status(fbp_batch_t batch)
{
    fbp_batch_s *b = reinterpret_cast<fbp_batch_s *>(batch);
    if (b == nullptr) {
        set_error("fbp_batch_status: batch is NULL");
        return FBP_ERR_INVALID_ARG;
    }
    const fbp_status st = take_device_status(b->d_status, "fbp_batch_status");
    if (st == FBP_ERR_TIMEOUT) {
        // a launch that gave up left its work counter where it stopped
        cudaMemset(b->d_sched, 0, sizeof(int) * 2 * kSchedSets * kSchedPerSet);
    }
    return st;
}

fbp_status fbp_batch_destroy(fbp_batch_t batch)
{
    fbp_batch_s *b = reinterpret_cast<fbp_batch_s *>(batch);
    if (b == nullptr) return FBP_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return FBP_OK;
}

}  // extern "C"
