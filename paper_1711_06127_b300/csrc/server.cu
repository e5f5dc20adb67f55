// server.cu -- real-time request loop over the supra_* entry points.
//
// The paper's runtime streams frames through a node graph on one GPU (Sec. 2);
// this is the B300 form of that loop for many concurrent acquisitions:
//
//  * Memory admission.  One device arena is allocated at start-up; each
//    request's footprint (ingested channel data, output image, scratch) is
//    carved from it with a first-fit allocator.  Requests are admitted in
//    arrival order as memory frees up; a request that does not fit waits.
//  * Continuous batching.  Whenever the worker wakes (a submission or a
//    completion), the admissible requests of one kind are formed into the next
//    batch: B-mode requests of any plans in one uneven supra_bmode_batched
//    call, MV and learned-apodization requests as one sequence of launches.
//  * Overlap.  Batches go round-robin to n_streams CUDA streams, so copies
//    and kernels of different batches overlap on the device.
//  * Graphs.  A batch whose bucket (stream, kind, plan sequence) has been seen
//    before is captured into a CUDA graph; the instantiated graph is cached per
//    bucket and refreshed with cudaGraphExecUpdate when only buffer addresses
//    changed.  A first-seen bucket launches directly.
//  * Completion.  A host function enqueued after the batch timestamps its
//    completion; the worker then frees the batch's memory and publishes the
//    per-request completions (submission, admission and completion times).
//
// Plans (geometry, delay tables, taps, scan-conversion maps) stay resident:
// requests refer to plans the caller created once.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "supra.h"
#include "arena.h"

namespace {

constexpr size_t kAlign = supra::OffsetArena::kAlign;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// One device allocation; offsets handed out by a first-fit OffsetArena.
class Arena {
   public:
    bool init(size_t bytes) {
        bytes = bytes / kAlign * kAlign;
        if (bytes == 0 || cudaMalloc(&base_, bytes) != cudaSuccess) return false;
        off_.reset(bytes);
        return true;
    }
    void release() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    size_t alloc(size_t bytes) { return off_.alloc(bytes); }
    void free(size_t off) { off_.free(off); }
    char *ptr(size_t off) const { return static_cast<char *>(base_) + off; }
    size_t size() const { return off_.size(); }
    size_t used() const { return off_.used(); }
    size_t peak() const { return off_.peak(); }

   private:
    void *base_ = nullptr;
    supra::OffsetArena off_;
};

struct Req {
    int64_t ticket = 0;
    supra_request r{};
    supra_plan_info info{};
    double t_submit = 0.0, t_admit = 0.0;
    size_t in_off = SIZE_MAX, out_off = SIZE_MAX, scratch_off = SIZE_MAX;
    size_t in_bytes = 0, out_bytes = 0, scratch_bytes = 0;
};

struct Batch;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::list<std::string>::iterator lru;
};

}  // namespace

struct supra_server {
    supra_server_config cfg{};
    int device = 0;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv, idle_cv;
    std::deque<Req> pending;
    std::deque<Batch *> done;
    std::deque<supra_completion> completed;
    std::unordered_map<int64_t, size_t> held;   // ticket -> output offset kept on the device
    int inflight = 0;
    int64_t next_ticket = 1, next_batch = 0;
    int64_t submitted = 0, n_completed = 0, n_batches = 0, graph_launches = 0, graph_inst = 0, graph_updates = 0;
    bool stop = false;
    std::thread worker;
    std::vector<std::thread> feeders;
    std::chrono::steady_clock::time_point t0;
    // graph cache (worker thread only): a bucket gets a graph once it recurs
    std::unordered_map<std::string, GraphEntry> graphs;
    std::unordered_map<std::string, int> seen;
    std::list<std::string> lru;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

struct Batch {
    supra_server *s = nullptr;
    int64_t id = 0;
    int kind = 0;
    int stream = 0;
    std::vector<Req> reqs;
    size_t ws_off = SIZE_MAX, ws_bytes = 0;
    int status = SUPRA_OK;
    double t_done = 0.0;
};

constexpr int kGraphCacheMax = 64;

void CUDART_CB on_batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    supra_server *s = b->s;
    std::lock_guard<std::mutex> lk(s->mu);
    b->t_done = s->now();
    s->done.push_back(b);
    s->cv.notify_all();
}

// Scratch of one MV / learned-apodization request: rf and envelope (float
// lines) and the log-compressed lines (uint8) when the plan scan-converts.
size_t scratch_bytes(const supra_request &r, const supra_plan_info &info) {
    if (r.kind == SUPRA_KIND_DAS) return 0;
    return align_up((size_t)info.rf_bytes) * 2 + (info.has_grid ? align_up((size_t)info.bmode_bytes) : 0);
}

size_t out_bytes(const supra_plan_info &info) {
    return (size_t)(info.has_grid ? info.image_bytes : info.bmode_bytes);
}

// Reserves the memory of one request; false (nothing held) when it does not fit.
bool reserve(Arena &a, Req &q) {
    q.in_off = q.out_off = q.scratch_off = SIZE_MAX;   // an earlier failed attempt may have left offsets
    q.in_bytes = q.r.ch_host ? (size_t)q.info.channel_bytes : 0;
    q.out_bytes = out_bytes(q.info);
    q.scratch_bytes = scratch_bytes(q.r, q.info);
    if (q.in_bytes && (q.in_off = a.alloc(q.in_bytes)) == SIZE_MAX) return false;
    if ((q.out_off = a.alloc(q.out_bytes)) == SIZE_MAX) {
        if (q.in_bytes) a.free(q.in_off), q.in_off = SIZE_MAX;
        return false;
    }
    if (q.scratch_bytes && (q.scratch_off = a.alloc(q.scratch_bytes)) == SIZE_MAX) {
        if (q.in_bytes) a.free(q.in_off), q.in_off = SIZE_MAX;
        a.free(q.out_off), q.out_off = SIZE_MAX;
        return false;
    }
    return true;
}

void unreserve(Arena &a, Req &q, bool keep_out) {
    if (q.in_off != SIZE_MAX) a.free(q.in_off), q.in_off = SIZE_MAX;
    if (q.scratch_off != SIZE_MAX) a.free(q.scratch_off), q.scratch_off = SIZE_MAX;
    if (!keep_out && q.out_off != SIZE_MAX) a.free(q.out_off), q.out_off = SIZE_MAX;
}

// Next batch from the pending queue (caller holds the lock): the head request
// and up to max_batch - 1 further requests of its kind among the next
// 4 * max_batch, each admitted only if its memory can be reserved.
Batch *form_batch(supra_server *s) {
    if (s->pending.empty()) return nullptr;
    Arena &a = s->arena;
    const int kind = s->pending.front().r.kind;
    const int max_b = std::max(1, s->cfg.max_batch);
    const size_t window = (size_t)4 * max_b;
    std::vector<size_t> take;
    std::vector<Req> got;
    for (size_t i = 0; i < s->pending.size() && i < window && (int)got.size() < max_b; ++i) {
        Req &q = s->pending[i];
        if (q.r.kind != kind) continue;
        if (!reserve(a, q)) break;   // arrival order within a kind: nothing passes a request that waits
        take.push_back(i);
        got.push_back(q);
    }
    if (got.empty()) return nullptr;
    Batch *b = new Batch;
    b->s = s;
    b->kind = kind;
    if (kind == SUPRA_KIND_DAS) {
        std::vector<const supra_plan *> plans;
        for (const Req &q : got) plans.push_back(q.r.plan);
        // one contiguous workspace; drop requests from the tail until it fits
        while (!got.empty()) {
            b->ws_bytes = supra_bmode_workspace_size((int32_t)plans.size(), plans.data());
            if (b->ws_bytes == 0 || (b->ws_off = a.alloc(b->ws_bytes)) != SIZE_MAX) break;
            unreserve(a, got.back(), false);
            got.pop_back();
            take.pop_back();
            plans.pop_back();
        }
        if (got.empty()) {
            delete b;
            return nullptr;
        }
    }
    const double t = s->now();
    for (Req &q : got) q.t_admit = t;
    // frames of one plan side by side: they share DAS tiles (and bucket keys repeat)
    std::stable_sort(got.begin(), got.end(), [](const Req &x, const Req &y) {
        return reinterpret_cast<uintptr_t>(x.r.plan) < reinterpret_cast<uintptr_t>(y.r.plan);
    });
    for (size_t j = take.size(); j-- > 0;) s->pending.erase(s->pending.begin() + (long)take[j]);
    b->reqs = std::move(got);
    b->id = s->next_batch++;
    b->stream = (int)(b->id % (int64_t)s->streams.size());
    return b;
}

const int16_t *input_of(const supra_server *s, const Req &q) {
    return q.in_off != SIZE_MAX ? reinterpret_cast<const int16_t *>(s->arena.ptr(q.in_off)) : q.r.ch;
}

// The device work of a batch, in stream order.
int enqueue_compute(supra_server *s, Batch *b, cudaStream_t st) {
    const size_t n = b->reqs.size();
    if (b->kind == SUPRA_KIND_DAS) {
        std::vector<const supra_plan *> plans(n);
        std::vector<const int16_t *> ch(n);
        std::vector<uint8_t *> out(n);
        for (size_t k = 0; k < n; ++k) {
            plans[k] = b->reqs[k].r.plan;
            ch[k] = input_of(s, b->reqs[k]);
            out[k] = reinterpret_cast<uint8_t *>(s->arena.ptr(b->reqs[k].out_off));
        }
        void *ws = b->ws_bytes ? s->arena.ptr(b->ws_off) : nullptr;
        return supra_bmode_batched((int32_t)n, plans.data(), ch.data(), out.data(), ws, b->ws_bytes, st);
    }
    for (Req &q : b->reqs) {
        char *scr = s->arena.ptr(q.scratch_off);
        float *rf = reinterpret_cast<float *>(scr);
        float *env = reinterpret_cast<float *>(scr + align_up((size_t)q.info.rf_bytes));
        uint8_t *out = reinterpret_cast<uint8_t *>(s->arena.ptr(q.out_off));
        uint8_t *bm = q.info.has_grid ? reinterpret_cast<uint8_t *>(scr + 2 * align_up((size_t)q.info.rf_bytes)) : out;
        int rc = q.r.kind == SUPRA_KIND_MV
                     ? supra_mv(q.r.plan, q.r.mv_subaperture, q.r.mv_loading, input_of(s, q), rf, st)
                     : supra_apod_mlp(q.r.plan, q.r.apod_params, input_of(s, q), rf, st);
        if (!rc) rc = supra_envelope(q.r.plan, rf, env, st);
        if (!rc) rc = supra_logcompress(q.r.plan, env, bm, st);
        if (!rc && q.info.has_grid) rc = supra_scanconvert(q.r.plan, bm, out, st);
        if (rc) return rc;
    }
    return SUPRA_OK;
}

std::string bucket_key(const Batch *b) {
    std::string k = std::to_string(b->stream) + ":" + std::to_string(b->kind);
    for (const Req &q : b->reqs) k += ":" + std::to_string(reinterpret_cast<uintptr_t>(q.r.plan));
    return k;
}

// Captures the batch's compute into a graph and launches the cached
// executable of its bucket (updated in place, or instantiated anew).
int launch_graph(supra_server *s, Batch *b, cudaStream_t st) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SUPRA_ECUDA;
    const int rc = enqueue_compute(s, b, st);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rc || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : SUPRA_ECUDA;
    }
    const std::string key = bucket_key(b);
    auto it = s->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != s->graphs.end()) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(it->second.exec, g, &info) == cudaSuccess) {
            exec = it->second.exec;
            ++s->graph_updates;
            s->lru.erase(it->second.lru);
            s->lru.push_front(key);
            it->second.lru = s->lru.begin();
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(it->second.exec);
            s->lru.erase(it->second.lru);
            s->graphs.erase(it);
        }
    }
    if (!exec) {
        if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return SUPRA_ECUDA;
        }
        ++s->graph_inst;
        if ((int)s->graphs.size() >= kGraphCacheMax) {
            const std::string old = s->lru.back();
            s->lru.pop_back();
            cudaGraphExecDestroy(s->graphs[old].exec);   // later launches of it are already ordered on their streams
            s->graphs.erase(old);
        }
        s->lru.push_front(key);
        s->graphs[key] = GraphEntry{exec, s->lru.begin()};
    }
    cudaGraphDestroy(g);
    ++s->graph_launches;
    return cudaGraphLaunch(exec, st) == cudaSuccess ? SUPRA_OK : SUPRA_ECUDA;
}

void launch_batch(supra_server *s, Batch *b) {
    cudaStream_t st = s->streams[b->stream];
    int rc = SUPRA_OK;
    for (Req &q : b->reqs)
        if (!rc && q.in_off != SIZE_MAX &&
            cudaMemcpyAsync(s->arena.ptr(q.in_off), q.r.ch_host, q.in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = SUPRA_ECUDA;
    bool graph = false;
    if (!rc && s->cfg.use_graphs) {
        // first sight of a bucket: launch directly (an instantiation would not be repaid)
        const std::string key = bucket_key(b);
        int &n = s->seen[key];
        graph = ++n >= 2;
        if (s->seen.size() > 4096) s->seen.clear();
    }
    if (!rc) rc = graph ? launch_graph(s, b, st) : enqueue_compute(s, b, st);
    for (Req &q : b->reqs)
        if (!rc && q.r.out_host &&
            cudaMemcpyAsync(q.r.out_host, s->arena.ptr(q.out_off), q.out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = SUPRA_ECUDA;
    b->status = rc;
    if (cudaLaunchHostFunc(st, on_batch_done, b) != cudaSuccess) {
        // nothing will call back: retire now (after the stream's work ends)
        cudaStreamSynchronize(st);
        b->status = b->status ? b->status : SUPRA_ECUDA;
        on_batch_done(b);
    }
}

void retire(supra_server *s, Batch *b) {
    for (Req &q : b->reqs) {
        const bool keep = b->status == SUPRA_OK && !q.r.out_host;
        supra_completion c{};
        c.ticket = q.ticket;
        c.tag = q.r.tag;
        c.status = b->status;
        c.batch_size = (int32_t)b->reqs.size();
        c.out = keep ? reinterpret_cast<const uint8_t *>(s->arena.ptr(q.out_off)) : nullptr;
        c.out_bytes = (int64_t)q.out_bytes;
        c.t_submit = q.t_submit;
        c.t_admit = q.t_admit;
        c.t_done = b->t_done;
        if (keep) s->held[q.ticket] = q.out_off;
        unreserve(s->arena, q, keep);
        s->completed.push_back(c);
        ++s->n_completed;
    }
    if (b->ws_off != SIZE_MAX) s->arena.free(b->ws_off);
    --s->inflight;
    delete b;
}

void worker_loop(supra_server *s) {
    cudaSetDevice(s->device);
    const int max_inflight = 2 * (int)s->streams.size();
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (!s->done.empty()) {
            Batch *b = s->done.front();
            s->done.pop_front();
            retire(s, b);
        }
        if (s->pending.empty() && s->inflight == 0) s->idle_cv.notify_all();
        if (s->stop && s->pending.empty() && s->inflight == 0) break;
        bool launched = false;
        while (s->inflight < max_inflight) {
            Batch *b = form_batch(s);
            if (!b) break;
            ++s->inflight;
            ++s->n_batches;
            lk.unlock();
            launch_batch(s, b);
            lk.lock();
            launched = true;
        }
        if (!launched && s->done.empty()) s->cv.wait(lk);
    }
}

bool valid_request(const supra_server *s, const supra_request &r, supra_plan_info &info) {
    if (!r.plan || (r.ch == nullptr) == (r.ch_host == nullptr)) return false;
    if (r.kind != SUPRA_KIND_DAS && r.kind != SUPRA_KIND_MV && r.kind != SUPRA_KIND_APOD) return false;
    if (supra_plan_get_info(r.plan, &info) != SUPRA_OK) return false;
    if (r.kind == SUPRA_KIND_APOD && (!r.apod_params || info.n_el > SUPRA_APOD_INPUTS)) return false;
    if (r.kind == SUPRA_KIND_MV && (r.mv_subaperture < 1 || r.mv_subaperture > 32 || !(r.mv_loading > 0.0f)))
        return false;
    // the request alone must fit the arena (with its share of a batch workspace)
    const size_t need = (r.ch_host ? align_up((size_t)info.channel_bytes) : 0) + align_up(out_bytes(info)) +
                        align_up(scratch_bytes(r, info)) +
                        (r.kind == SUPRA_KIND_DAS ? align_up(supra_bmode_workspace_size(1, &r.plan)) : 0);
    return need <= s->arena.size();
}

}  // namespace

extern "C" {

int supra_server_create(const supra_server_config *cfg, supra_server **out) {
    if (!cfg || !out || cfg->memory_bytes < kAlign || cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_batch < 1)
        return SUPRA_EINVAL;
    *out = nullptr;
    auto *s = new (std::nothrow) supra_server;
    if (!s) return SUPRA_ENOMEM;
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return SUPRA_ECUDA;
    }
    if (!s->arena.init(cfg->memory_bytes)) {
        cudaGetLastError();
        delete s;
        return SUPRA_ENOMEM;
    }
    for (int i = 0; i < cfg->n_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            s->arena.release();
            delete s;
            return SUPRA_ECUDA;
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return SUPRA_OK;
}

int supra_server_submit(supra_server *s, const supra_request *r, int64_t *ticket) {
    if (!s || !r) return SUPRA_EINVAL;
    Req q;
    q.r = *r;
    if (!valid_request(s, q.r, q.info)) return SUPRA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SUPRA_EINVAL;
    q.ticket = s->next_ticket++;
    q.t_submit = s->now();
    if (ticket) *ticket = q.ticket;
    s->pending.push_back(q);
    ++s->submitted;
    s->cv.notify_all();
    return SUPRA_OK;
}

int supra_server_submit_trace(supra_server *s, int32_t n, const supra_request *reqs, const double *t_arrival,
                              int64_t *tickets) {
    if (!s || n < 0 || (n && (!reqs || !t_arrival))) return SUPRA_EINVAL;
    std::vector<supra_request> rs(reqs, reqs + n);
    std::vector<double> ts(t_arrival, t_arrival + n);
    for (int i = 0; i < n; ++i) {
        supra_plan_info info;
        if (!valid_request(s, rs[i], info) || (i > 0 && ts[i] < ts[i - 1])) return SUPRA_EINVAL;
    }
    const double start = s->now();
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t first = s->next_ticket;
    s->next_ticket += n;
    if (tickets)
        for (int i = 0; i < n; ++i) tickets[i] = first + i;
    s->feeders.emplace_back([s, rs = std::move(rs), ts = std::move(ts), start, first]() {
        for (size_t i = 0; i < rs.size(); ++i) {
            const double due = start + ts[i];
            double t = s->now();
            while (t < due) {
                const double wait = due - t;
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
                t = s->now();
            }
            Req q;
            q.r = rs[i];
            supra_plan_get_info(q.r.plan, &q.info);
            q.ticket = first + (int64_t)i;
            q.t_submit = due;   // latency counts from the scheduled arrival
            std::lock_guard<std::mutex> g(s->mu);
            s->pending.push_back(q);
            ++s->submitted;
            s->cv.notify_all();
        }
    });
    return SUPRA_OK;
}

int supra_server_poll(supra_server *s, supra_completion *out, int32_t max, int32_t *n) {
    if (!s || !n || max < 0 || (max && !out)) return SUPRA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && !s->completed.empty()) {
        out[k++] = s->completed.front();
        s->completed.pop_front();
    }
    *n = k;
    return SUPRA_OK;
}

int supra_server_wait(supra_server *s, int64_t n_submitted, double timeout_s) {
    if (!s) return SUPRA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto ok = s->idle_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return s->submitted >= n_submitted && s->pending.empty() && s->inflight == 0;
    });
    return ok ? SUPRA_OK : SUPRA_ETIMEOUT;
}

int supra_server_release(supra_server *s, int64_t ticket) {
    if (!s) return SUPRA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->held.find(ticket);
    if (it == s->held.end()) return SUPRA_EINVAL;
    s->arena.free(it->second);
    s->held.erase(it);
    s->cv.notify_all();   // memory freed: waiting requests may fit now
    return SUPRA_OK;
}

int supra_server_get_stats(supra_server *s, supra_server_stats *st) {
    if (!s || !st) return SUPRA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->n_completed;
    st->batches = s->n_batches;
    st->graph_launches = s->graph_launches;
    st->graph_instantiations = s->graph_inst;
    st->graph_updates = s->graph_updates;
    st->memory_used = (int64_t)s->arena.used();
    st->memory_peak = (int64_t)s->arena.peak();
    st->pending = (int32_t)s->pending.size();
    st->inflight = s->inflight;
    return SUPRA_OK;
}

double supra_server_now(const supra_server *s) { return s ? s->now() : -1.0; }

void supra_server_destroy(supra_server *s) {
    if (!s) return;
    std::vector<std::thread> feeders;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        feeders.swap(s->feeders);
    }
    for (std::thread &f : feeders) f.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second.exec);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    s->arena.release();
    delete s;
}

}  // extern "C"
