// Continuous-batching embedding server (host runtime, C ABI in include/gee.h).
//
// Requests (host edge lists) are admitted as device memory from one pool frees up:
// each admitted request gets its inputs and Z in the pool.  A copy thread moves the
// inputs to the device on a copy stream (pinned inputs directly, pageable ones through a
// ring of pinned staging buffers).  A worker thread keeps forming batches of copied
// requests and launches each batch through the batch path (gee_embed_batch) on the next
// of several compute streams, so batches that are admitted while others run overlap on
// the device.  A batch's workspace (which holds the CSR of its graphs) and each request's
// Z stay resident until the request is released.  Latency is measured from submission to
// the moment the stream passes the batch (a host function enqueued after it).
//
// Locking: the request mutex guards the queues, the pool and the request states only.
// No CUDA call that can block (a copy from pageable memory, a batch launch with its
// descriptor upload) runs while it is held, so submit, poll and release never wait
// behind a copy.
#include "../../include/gee.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kPoolAlign = 256;
constexpr int kPollLimitSeconds = 120;

size_t align_up(size_t x) { return (x + kPoolAlign - 1) & ~(kPoolAlign - 1); }

// First-fit sub-allocator over one device region; free blocks coalesce.
class Pool {
  public:
    void init(char *base, size_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    char *alloc(size_t n) {
        n = align_up(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                sizes_[off] = n;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(char *p) {
        if (!p) return;
        const size_t off = (size_t)(p - base_);
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t n = s->second;
        sizes_.erase(s);
        used_ -= n;
        size_t start = off;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + n) {
            n += next->second;
            free_.erase(next);
        }
        auto prev = free_.lower_bound(off);
        if (prev != free_.begin()) {
            --prev;
            if (prev->first + prev->second == off) {
                start = prev->first;
                n += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = n;
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;           // offset -> bytes
    std::unordered_map<size_t, size_t> sizes_;  // offset -> bytes of live blocks
};

enum class RState { Queued, Admitted, Running, Done, Cancelled };

constexpr size_t kStageSlotBytes = 16u << 20;  // pinned staging for pageable inputs
constexpr int kStageSlots = 4;

struct Batch;

struct Request {
    int64_t ticket = 0;
    gee_request in{};
    RState state = RState::Queued;
    char *block = nullptr;  // pool block: inputs + Z
    int32_t *d_src = nullptr, *d_dst = nullptr, *d_y = nullptr;
    float *d_w = nullptr, *d_Z = nullptr;
    size_t bytes = 0;            // inputs + Z
    size_t ws_reserve = 0;       // a workspace for this request alone (batch of one)
    char *ws_block = nullptr;    // held from admission until its batch is launched
    cudaEvent_t copied = nullptr;
    std::shared_ptr<Batch> batch;
    int index_in_batch = 0;
    Clock::time_point t_submit;
    double latency_ms = -1.0;
    bool failed = false;  // its batch hit a CUDA error
};

struct Batch {
    char *ws = nullptr;        // pool block: the batch workspace (CSR of every graph)
    uint32_t *d_status = nullptr;
    std::vector<std::shared_ptr<Request>> reqs;
    int stream = 0;
    cudaEvent_t done = nullptr;
    std::atomic<bool> finished{false};
    bool host_failed = false;  // the launch itself returned an error
    Clock::time_point t_done;
    int live = 0;  // requests not yet released
};

size_t request_bytes(const gee_request &r) {
    size_t b = 0;
    b += align_up(sizeof(int32_t) * (size_t)r.E) * 2;
    if (r.w) b += align_up(sizeof(float) * (size_t)r.E);
    b += align_up(sizeof(int32_t) * (size_t)r.N);
    b += align_up(sizeof(float) * (size_t)r.N * (size_t)r.K);
    return b;
}

}  // namespace

struct gee_server {
    gee_server_config cfg{};
    int device = 0;
    char *pool_mem = nullptr;
    Pool pool;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;  // batches in flight per stream
    cudaStream_t copy_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;   // waiting for memory
    std::deque<std::shared_ptr<Request>> tocopy;  // admitted, inputs not copied yet
    std::deque<std::shared_ptr<Request>> ready;   // copied (in stream order), waiting for a launch
    std::unordered_map<int64_t, std::shared_ptr<Request>> all;
    std::vector<std::shared_ptr<Batch>> inflight;
    int64_t next_ticket = 1;
    gee_server_stats stats{};
    bool stop = false;
    std::thread worker, copier;
    int last_error = GEE_OK;
    // pinned staging ring of the copy thread (pageable inputs), one event per slot
    char *stage = nullptr;
    cudaEvent_t stage_ev[kStageSlots] = {};
    int stage_next = 0;
};

namespace {

void CUDART_CB on_batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    b->t_done = Clock::now();
    b->finished.store(true, std::memory_order_release);
}

// Admit queued requests in arrival order while their inputs, Z and a workspace of their
// own fit in the pool (the own workspace guarantees every admitted request can run even
// when the pool is fragmented).  Admission is strictly first-come first-served: a
// request that does not fit yet stops admission, so later requests can never take the
// memory an earlier one is waiting for.  Called with the mutex held: it only reserves
// memory and hands the request to the copy thread.
void admit(gee_server *s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        auto r = *it;
        char *blk = s->pool.alloc(r->bytes);
        char *wsb = blk ? s->pool.alloc(r->ws_reserve) : nullptr;
        if (!blk || !wsb) {
            s->pool.release(blk);
            break;
        }
        r->block = blk;
        r->ws_block = wsb;
        size_t off = 0;
        auto take = [&](size_t n) {
            char *p = blk + off;
            off += align_up(n);
            return p;
        };
        r->d_src = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)r->in.E));
        r->d_dst = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)r->in.E));
        r->d_w = r->in.w ? reinterpret_cast<float *>(take(sizeof(float) * (size_t)r->in.E)) : nullptr;
        r->d_y = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)r->in.N));
        r->d_Z = reinterpret_cast<float *>(take(sizeof(float) * (size_t)r->in.N * (size_t)r->in.K));
        r->state = RState::Admitted;
        s->tocopy.push_back(r);
        it = s->queue.erase(it);
    }
    s->stats.queued = (int64_t)s->queue.size();
}

bool host_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Host -> device copy of n bytes on the copy stream: pinned sources directly, pageable
// ones chunk by chunk through the staging ring (a slot is reused once the copy that last
// read it has finished).  Runs on the copy thread without the mutex.
int copy_in(gee_server *s, void *dst, const void *src, size_t n) {
    if (n == 0) return GEE_OK;
    cudaStream_t cs = s->copy_stream;
    if (!s->stage || host_pinned(src))
        return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, cs) == cudaSuccess ? GEE_OK : GEE_ERR_CUDA;
    for (size_t off = 0; off < n; off += kStageSlotBytes) {
        const size_t m = std::min(kStageSlotBytes, n - off);
        const int k = s->stage_next;
        s->stage_next = (k + 1) % kStageSlots;
        if (cudaEventSynchronize(s->stage_ev[k]) != cudaSuccess) return GEE_ERR_CUDA;
        char *slot = s->stage + (size_t)k * kStageSlotBytes;
        std::memcpy(slot, static_cast<const char *>(src) + off, m);
        if (cudaMemcpyAsync(static_cast<char *>(dst) + off, slot, m, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return GEE_ERR_CUDA;
        if (cudaEventRecord(s->stage_ev[k], cs) != cudaSuccess) return GEE_ERR_CUDA;
    }
    return GEE_OK;
}

// The copy thread: takes admitted requests in order, copies their inputs and passes them
// on to the worker (ready) with an event that marks the end of their copies.
void copier_loop(gee_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        if (s->tocopy.empty()) {
            s->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        auto r = s->tocopy.front();
        s->tocopy.pop_front();
        lk.unlock();
        int rc = GEE_OK;
        if (r->in.E > 0) {
            rc = copy_in(s, r->d_src, r->in.src, sizeof(int32_t) * (size_t)r->in.E);
            if (rc == GEE_OK) rc = copy_in(s, r->d_dst, r->in.dst, sizeof(int32_t) * (size_t)r->in.E);
            if (rc == GEE_OK && r->in.w) rc = copy_in(s, r->d_w, r->in.w, sizeof(float) * (size_t)r->in.E);
        }
        if (rc == GEE_OK && r->in.N > 0)
            rc = copy_in(s, r->d_y, r->in.labels, sizeof(int32_t) * (size_t)r->in.N);
        if (rc == GEE_OK && cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming) != cudaSuccess)
            rc = GEE_ERR_CUDA;
        if (rc == GEE_OK && cudaEventRecord(r->copied, s->copy_stream) != cudaSuccess) rc = GEE_ERR_CUDA;
        lk.lock();
        if (rc != GEE_OK) s->last_error = rc;  // the request still runs; its batch reports
        s->ready.push_back(r);
        s->cv.notify_all();
    }
}

gee_graph graph_of(const Request &r) {
    return gee_graph{r.d_src, r.d_dst, r.d_w, r.d_y, r.d_Z, r.in.E, r.in.N, r.in.K};
}

// Form one batch from copied requests and reserve it, with the mutex held: as many ready
// requests (up to max_batch) as a fresh contiguous workspace can be found for; failing
// that, the oldest ready request alone in its own workspace.  Returns null when nothing
// can be launched now.  The caller launches the batch without the mutex (launch_batch).
struct PendingLaunch {
    std::shared_ptr<Batch> b;
    std::vector<gee_graph> gs;
    char *ws = nullptr;
    size_t ws_bytes = 0;
};

bool reserve_batch(gee_server *s, PendingLaunch &pl) {
    if (s->ready.empty()) return false;
    int si = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i)
        if (s->stream_busy[i] == 0) {
            si = i;
            break;
        }
    if (si < 0) return false;
    gee_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.flags = s->cfg.flags;
    size_t n = std::min(s->ready.size(), (size_t)s->cfg.max_batch);
    std::vector<gee_graph> gs;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    while (n >= 2) {
        gs.clear();
        for (size_t i = 0; i < n; ++i) gs.push_back(graph_of(*s->ready[i]));
        ws_bytes = gee_batch_workspace_size(gs.data(), (int32_t)n, &opts) + align_up(sizeof(uint32_t) * n);
        ws = s->pool.alloc(ws_bytes);
        if (ws) break;
        n /= 2;
    }
    bool own = false;
    if (!ws) {  // the oldest request runs alone in the workspace it was admitted with
        n = 1;
        gs.assign(1, graph_of(*s->ready.front()));
        ws = s->ready.front()->ws_block;
        ws_bytes = s->ready.front()->ws_reserve;
        own = true;
    }
    auto b = std::make_shared<Batch>();
    b->ws = own ? nullptr : ws;
    b->stream = si;
    b->d_status = reinterpret_cast<uint32_t *>(ws + ws_bytes - align_up(sizeof(uint32_t) * n));
    for (size_t i = 0; i < n; ++i) {
        auto r = s->ready.front();
        s->ready.pop_front();
        r->state = RState::Running;
        r->batch = b;
        r->index_in_batch = (int)i;
        if (!own) {  // the shared workspace replaces the request's own
            s->pool.release(r->ws_block);
            r->ws_block = nullptr;
        }
        b->reqs.push_back(r);
    }
    b->live = (int)n;
    s->stream_busy[si] += 1;
    s->stats.launches += 1;
    pl.b = b;
    pl.gs = std::move(gs);
    pl.ws = ws;
    pl.ws_bytes = ws_bytes;
    return true;
}

// Enqueue a reserved batch on its stream (no mutex held): wait for its inputs' copies,
// run the batch path, then the completion event and host function.
int launch_batch(gee_server *s, PendingLaunch &pl) {
    Batch &b = *pl.b;
    cudaStream_t st = s->streams[b.stream];
    int rc = GEE_OK;
    for (auto &r : b.reqs)
        if (r->copied && cudaStreamWaitEvent(st, r->copied, 0) != cudaSuccess) rc = GEE_ERR_CUDA;
    gee_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.flags = s->cfg.flags;
    const size_t n = b.reqs.size();
    if (rc == GEE_OK)
        rc = gee_embed_batch(pl.gs.data(), (int32_t)n, &opts, pl.ws, pl.ws_bytes - align_up(sizeof(uint32_t) * n),
                             st, b.d_status);
    cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    cudaEventRecord(b.done, st);
    cudaLaunchHostFunc(st, on_batch_done, pl.b.get());
    return rc;
}

void reap(gee_server *s) {
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        auto &b = *it;
        bool failed = false;
        if (!b->finished.load(std::memory_order_acquire)) {
            // a launch that failed on the device never reaches its host function: finish
            // its requests with an error instead of waiting for them forever
            const cudaError_t q = b->done ? cudaEventQuery(b->done) : cudaSuccess;
            if (q == cudaErrorNotReady || q == cudaSuccess) {
                ++it;
                continue;
            }
            failed = true;
            b->t_done = Clock::now();
            s->last_error = GEE_ERR_CUDA;
        }
        failed = failed || b->host_failed;
        for (auto &r : b->reqs) {
            r->latency_ms = std::chrono::duration<double, std::milli>(b->t_done - r->t_submit).count();
            r->failed = failed;
            r->state = RState::Done;
            s->stats.completed += 1;
            s->stats.edges_done += r->in.E;
        }
        s->stream_busy[b->stream] -= 1;
        it = s->inflight.erase(it);
    }
    s->stats.running = 0;
    for (auto &b : s->inflight) s->stats.running += (int64_t)b->reqs.size();
}

void worker_loop(gee_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        reap(s);
        admit(s);
        bool launched = false;
        PendingLaunch pl;
        while (reserve_batch(s, pl)) {
            launched = true;
            lk.unlock();
            const int rc = launch_batch(s, pl);
            lk.lock();
            if (rc != GEE_OK) {
                s->last_error = rc;
                pl.b->host_failed = true;
            }
            s->inflight.push_back(pl.b);
            pl = PendingLaunch();
        }
        s->stats.bytes_in_use = s->pool.used();
        s->stats.peak_bytes_in_use = s->pool.peak();
        s->cv.notify_all();
        if (!launched) s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

void free_request(gee_server *s, const std::shared_ptr<Request> &r) {
    if (r->copied) cudaEventDestroy(r->copied);
    r->copied = nullptr;
    s->pool.release(r->block);
    r->block = nullptr;
    s->pool.release(r->ws_block);
    r->ws_block = nullptr;
    if (r->batch) {
        auto b = r->batch;
        r->batch.reset();
        if (--b->live == 0) {
            if (b->done) cudaEventDestroy(b->done);
            s->pool.release(b->ws);
        }
    }
}

}  // namespace

extern "C" {

int gee_server_create(const gee_server_config *cfg, gee_server **out) {
    if (!cfg || !out || cfg->hbm_budget < (1u << 20) || cfg->reserved != 0) return GEE_ERR_ARG;
    *out = nullptr;
    auto *s = new gee_server();
    s->cfg = *cfg;
    if (s->cfg.max_batch <= 0) s->cfg.max_batch = 1024;
    if (s->cfg.streams <= 0) s->cfg.streams = 2;
    s->cfg.flags &= GEE_ALL_OPTIONS;
    cudaGetDevice(&s->device);
    // the server owns one pool of the given budget: every request input, Z and batch
    // workspace is carved from it, so admission can never exceed the budget
    if (cudaMalloc(&s->pool_mem, s->cfg.hbm_budget) != cudaSuccess) {
        delete s;
        return GEE_ERR_NOMEM;
    }
    s->pool.init(s->pool_mem, s->cfg.hbm_budget);
    s->stats.pool_bytes = s->cfg.hbm_budget;
    s->streams.resize(s->cfg.streams);
    s->stream_busy.assign(s->cfg.streams, 0);
    for (auto &st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    // pinned staging for pageable inputs; without it such copies go straight from the
    // pageable source (slower, still correct)
    if (cudaHostAlloc(reinterpret_cast<void **>(&s->stage), kStageSlotBytes * kStageSlots, cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        s->stage = nullptr;
    }
    for (int k = 0; s->stage && k < kStageSlots; ++k)
        if (cudaEventCreateWithFlags(&s->stage_ev[k], cudaEventDisableTiming) != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaEventDestroy(s->stage_ev[j]);
            cudaFreeHost(s->stage);
            s->stage = nullptr;
        }
    s->worker = std::thread(worker_loop, s);
    s->copier = std::thread(copier_loop, s);
    *out = s;
    return GEE_OK;
}

int gee_server_submit(gee_server *s, const gee_request *req, int64_t *ticket) {
    if (!s || !req || !ticket) return GEE_ERR_ARG;
    if (req->E < 0 || req->N < 0 || req->K < 1) return GEE_ERR_ARG;
    if (req->N > GEE_MAX_N || req->E >= GEE_MAX_E || req->K > GEE_MAX_K) return GEE_ERR_TOO_LARGE;
    if (req->E > 0 && (!req->src || !req->dst)) return GEE_ERR_ARG;
    if (req->N > 0 && !req->labels) return GEE_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->in = *req;
    r->bytes = request_bytes(*req);
    gee_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.flags = s->cfg.flags;
    // the workspace of a batch holding only this request (plus its status word)
    gee_graph one{req->src, req->dst, req->w, req->labels, nullptr, req->E, req->N, req->K};
    one.Z = reinterpret_cast<float *>(1);  // any non-NULL address: sizing does not read it
    const size_t ws_one = gee_batch_workspace_size(&one, 1, &opts);
    if (ws_one == 0) return GEE_ERR_ARG;
    r->ws_reserve = align_up(ws_one) + align_up(sizeof(uint32_t));
    // a request that could never fit, even alone in an empty pool, is refused now
    if (align_up(r->bytes) + align_up(r->ws_reserve) > s->cfg.hbm_budget) return GEE_ERR_NOMEM;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    s->stats.submitted += 1;
    *ticket = r->ticket;
    s->cv.notify_all();
    return GEE_OK;
}

int gee_server_poll(gee_server *s, int64_t ticket, int wait, const float **d_Z, uint32_t *status, double *latency_ms) {
    if (!s) return GEE_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GEE_ERR_STATE;
    auto r = it->second;
    if (r->state == RState::Cancelled) return GEE_ERR_STATE;
    // bounded wait: a request not done within kPollLimit is reported as pending
    const auto give_up = Clock::now() + std::chrono::seconds(kPollLimitSeconds);
    while (wait && r->state != RState::Done && !s->stop && Clock::now() < give_up)
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
    if (r->state != RState::Done) return GEE_PENDING;
    if (r->failed) return GEE_ERR_CUDA;
    if (d_Z) *d_Z = r->d_Z;
    if (latency_ms) *latency_ms = r->latency_ms;
    if (status) {
        uint32_t st = 0;
        lk.unlock();
        if (cudaMemcpy(&st, r->batch ? r->batch->d_status + r->index_in_batch : nullptr, sizeof(uint32_t),
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return GEE_ERR_CUDA;
        *status = st;
    }
    return GEE_OK;
}

int gee_server_fetch(gee_server *s, int64_t ticket, float *Z_host) {
    const float *dz = nullptr;
    const int rc = gee_server_poll(s, ticket, 1, &dz, nullptr, nullptr);
    if (rc != GEE_OK) return rc;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r = s->all[ticket];
    }
    const size_t n = sizeof(float) * (size_t)r->in.N * (size_t)r->in.K;
    if (n && (!Z_host || cudaMemcpy(Z_host, dz, n, cudaMemcpyDeviceToHost) != cudaSuccess)) return GEE_ERR_CUDA;
    return GEE_OK;
}

int gee_server_cancel(gee_server *s, int64_t ticket) {
    if (!s) return GEE_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GEE_ERR_STATE;
    auto r = it->second;
    if (r->state != RState::Queued) return GEE_ERR_STATE;  // admitted work runs to completion
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
    r->state = RState::Cancelled;
    s->all.erase(it);
    s->stats.queued = (int64_t)s->queue.size();
    return GEE_OK;
}

int gee_server_release(gee_server *s, int64_t ticket) {
    if (!s) return GEE_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GEE_ERR_STATE;
    auto r = it->second;
    if (r->state != RState::Done) return GEE_ERR_STATE;
    free_request(s, r);
    s->all.erase(it);
    s->stats.bytes_in_use = s->pool.used();
    s->cv.notify_all();
    return GEE_OK;
}

int gee_server_get_stats(gee_server *s, gee_server_stats *out) {
    if (!s || !out) return GEE_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.bytes_in_use = s->pool.used();
    s->stats.peak_bytes_in_use = s->pool.peak();
    s->stats.last_error = s->last_error;
    *out = s->stats;
    return GEE_OK;
}

void gee_server_destroy(gee_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->copier.joinable()) s->copier.join();
    cudaDeviceSynchronize();
    for (auto &kv : s->all) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
    }
    for (auto &b : s->inflight)
        if (b->done) cudaEventDestroy(b->done);
    for (auto &st : s->streams) cudaStreamDestroy(st);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->stage) {
        for (int k = 0; k < kStageSlots; ++k) cudaEventDestroy(s->stage_ev[k]);
        cudaFreeHost(s->stage);
    }
    cudaFree(s->pool_mem);
    delete s;
}

}  // extern "C"
