// Online serving: continuous batching of kNN requests over resident indexes.
//
// The paper's online design (Sec. 5.2 double buffering, Sec. 6 Algorithm 3
// DTAHE) decides when a GPU buffer of queued queries is sent to the GPU: when
// it is full, or when the GPU is idle.  Without the CPU branch (there is no
// CPU kNN here) that rule is the dispatcher below:
//   - a batch is dispatched when no batch is running on the GPU, or when the
//     queued queries fill a batch (max_batch_queries), or -- a latency bound
//     the paper's rule does not have -- when the oldest queued request has
//     waited max_wait_us, so that under load batches overlap on the GPU
//     instead of queueing behind the one in flight;
//   - several batches may run at once, one per stream ("slot"), so requests
//     that arrive while others are on the GPU overlap with them;
//   - all device state of in-flight requests (queries, per-query depths,
//     results) lives in one arena of exactly hbm_budget bytes; a batch is
//     formed only from requests whose state fits in the free arena, so
//     admission waits for memory to free up, and a request that cannot fit
//     even alone is refused at submission (HC_ERR_BUDGET).
// Every query is answered independently by the query kernel (one warp per
// query), so a request's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hc_index.h"
#include "hc_trace.h"

using namespace hc;

namespace {

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) (byte offsets into the device arena and
// its pinned host mirror).
class Arena {
  public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t t_submit = 0, t_done = 0;   // steady-clock ns
    uint64_t ticket = 0;
    uint32_t index_id = 0, nq = 0, k = 0, p = 0;
    std::vector<uint8_t> q;
    std::vector<int32_t> ids;
    std::vector<uint32_t> dist;
    int status = HC_PENDING;
    bool in_batch = false;
};

// Device bytes of one request inside a batch (per-part 256-byte rounding is
// taken on the whole batch, so this is an upper bound for one request).
size_t request_bytes(uint32_t nq, uint32_t k, uint32_t row_bytes) {
    return round256((size_t)nq * row_bytes) + round256((size_t)nq * 4) +
           2 * round256((size_t)nq * k * 4);
}

struct Batch {
    int slot = -1;
    uint32_t index_id = 0, k = 0, nq = 0;
    std::vector<Request*> reqs;
    size_t off = 0, bytes = 0;
    size_t q_off = 0, p_off = 0, ids_off = 0, dist_off = 0;
    cudaEvent_t done = nullptr;
    int status = HC_OK;
};

}  // namespace

struct Predictor {
    hc_mlp* mlp = nullptr;
    float margin = 0.f;
    uint32_t p_lo = 1, p_hi = 512;
};

struct hc_server {
    std::vector<hc_index*> idx;
    std::vector<Predictor> pred;
    uint64_t budget = 0;
    hc_serve_params params{};
    int device = 0;
    char* arena_dev = nullptr;
    char* arena_host = nullptr;
    Arena* arena = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::vector<cudaEvent_t> events;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    uint64_t queued_queries = 0;
    std::unordered_map<uint64_t, Request*> live;
    std::vector<Batch*> inflight;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread dispatcher;
    hc_serve_stats stats{};
};

namespace {

void finalize(hc_server* S, Batch* b, int status) {
    // results come back through the pinned mirror of the batch's arena range
    if (status == HC_OK) {
        const int32_t* ids = reinterpret_cast<const int32_t*>(S->arena_host + b->ids_off);
        const uint32_t* dist = reinterpret_cast<const uint32_t*>(S->arena_host + b->dist_off);
        size_t row = 0;
        for (Request* r : b->reqs) {
            const size_t n = (size_t)r->nq * b->k;
            r->ids.assign(ids + row * b->k, ids + row * b->k + n);
            r->dist.assign(dist + row * b->k, dist + row * b->k + n);
            row += r->nq;
        }
    }
    const uint64_t t = now_ns();
    for (Request* r : b->reqs) {
        r->status = status;
        r->t_done = t;
    }
    S->arena->release(b->off, b->bytes);
    S->slot_busy[b->slot] = false;
    S->stats.queries_done += b->nq;
    S->stats.batches_done += 1;
}

// Called with S->mu held.  Takes requests in arrival order that share the
// head request's (index, k), up to max_batch_queries and the free arena.
Batch* form_batch(hc_server* S, int slot) {
    Request* head = S->queue.front();
    const hc_index* ix = S->idx[head->index_id];
    const uint32_t rb = ix->row_bytes;
    std::vector<Request*> take;
    uint32_t nq = 0;
    size_t bytes = 0;
    for (Request* r : S->queue) {
        if (r->index_id != head->index_id || r->k != head->k) continue;
        if (!take.empty() && nq + r->nq > S->params.max_batch_queries) break;
        const uint32_t n2 = nq + r->nq;
        const size_t b2 = request_bytes(n2, head->k, rb);
        size_t probe;
        if (!S->arena->alloc(b2, &probe)) break;   // does the grown batch still fit?
        S->arena->release(probe, b2);
        take.push_back(r);
        nq = n2;
        bytes = b2;
    }
    if (take.empty()) return nullptr;
    // requests whose depth the predictor chooses go first (one contiguous range)
    std::stable_partition(take.begin(), take.end(), [](const Request* r) { return r->p == 0; });
    Batch* b = new Batch();
    if (!S->arena->alloc(bytes, &b->off)) {
        delete b;
        return nullptr;
    }
    b->bytes = bytes;
    b->slot = slot;
    b->index_id = head->index_id;
    b->k = head->k;
    b->nq = nq;
    b->reqs = take;
    b->q_off = b->off;
    b->p_off = b->q_off + round256((size_t)nq * rb);
    b->ids_off = b->p_off + round256((size_t)nq * 4);
    b->dist_off = b->ids_off + round256((size_t)nq * b->k * 4);
    for (Request* r : take) {
        r->in_batch = true;
        S->queued_queries -= r->nq;
    }
    std::deque<Request*> rest;
    for (Request* r : S->queue)
        if (!r->in_batch) rest.push_back(r);
    S->queue.swap(rest);
    S->slot_busy[slot] = true;
    b->done = S->events[slot];
    return b;
}

// Stages the batch (host copies into the pinned mirror) and enqueues copy-in,
// the query kernel and copy-out on the slot's stream.  Called without the lock.
int launch_batch(hc_server* S, Batch* b) {
    TraceRange tr("serve_batch");
    const hc_index* ix = S->idx[b->index_id];
    const uint32_t rb = ix->row_bytes;
    char* hq = S->arena_host + b->q_off;
    uint32_t* hp = reinterpret_cast<uint32_t*>(S->arena_host + b->p_off);
    size_t row = 0;
    for (Request* r : b->reqs) {
        std::memcpy(hq + row * rb, r->q.data(), (size_t)r->nq * rb);
        const uint32_t depth = r->p ? r->p : S->params.default_p;
        for (uint32_t i = 0; i < r->nq; ++i) hp[row + i] = depth;
        row += r->nq;
    }
    cudaStream_t st = S->streams[b->slot];
    const size_t in_bytes = b->ids_off - b->q_off;
    if (cudaMemcpyAsync(S->arena_dev + b->q_off, hq, in_bytes, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return HC_ERR_CUDA;
    // learned depths for the leading p = 0 requests
    const Predictor& pr = S->pred[b->index_id];
    uint32_t n_auto = 0;
    for (Request* r : b->reqs)
        if (r->p == 0) n_auto += r->nq;
    if (pr.mlp && n_auto &&
        launch_predict_depths(pr.mlp, ix, S->arena_dev + b->q_off, n_auto, pr.margin, pr.p_lo,
                              pr.p_hi, reinterpret_cast<uint32_t*>(S->arena_dev + b->p_off),
                              st) != cudaSuccess)
        return HC_ERR_CUDA;
    if (launch_query(view_of(ix), S->arena_dev + b->q_off, b->nq, b->k, 0,
                     reinterpret_cast<int32_t*>(S->arena_dev + b->ids_off),
                     S->arena_dev + b->dist_off, st,
                     reinterpret_cast<const uint32_t*>(S->arena_dev + b->p_off)) != cudaSuccess)
        return HC_ERR_CUDA;
    const size_t out_bytes = b->bytes - (b->ids_off - b->off);
    if (cudaMemcpyAsync(S->arena_host + b->ids_off, S->arena_dev + b->ids_off, out_bytes,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HC_ERR_CUDA;
    if (cudaEventRecord(b->done, st) != cudaSuccess) return HC_ERR_CUDA;
    return HC_OK;
}

void dispatcher_loop(hc_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        // reap finished batches
        bool reaped = false;
        for (size_t i = 0; i < S->inflight.size();) {
            Batch* b = S->inflight[i];
            const cudaError_t e = cudaEventQuery(b->done);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            finalize(S, b, e == cudaSuccess ? b->status : HC_ERR_CUDA);
            if (e != cudaSuccess) cudaGetLastError();
            delete b;
            S->inflight.erase(S->inflight.begin() + i);
            reaped = true;
        }
        if (reaped) S->cv_done.notify_all();
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;

        // DTAHE's flush rule without the CPU branch: dispatch when the GPU is
        // idle, or when the queued queries fill a batch; and when the oldest
        // queued request has waited max_wait_us
        int slot = -1;
        for (size_t s = 0; s < S->slot_busy.size(); ++s)
            if (!S->slot_busy[s]) {
                slot = (int)s;
                break;
            }
        const bool gpu_idle = S->inflight.empty();
        const bool full = S->queued_queries >= S->params.max_batch_queries;
        const bool waited = !S->queue.empty() && S->params.max_wait_us > 0 &&
                            now_ns() - S->queue.front()->t_submit >=
                                1000ull * S->params.max_wait_us;
        if (!S->queue.empty() && slot >= 0 && (gpu_idle || full || waited)) {
            Batch* b = form_batch(S, slot);
            if (b) {
                S->inflight.push_back(b);
                S->stats.batches += 1;
                if (S->inflight.size() > S->stats.max_inflight)
                    S->stats.max_inflight = (uint32_t)S->inflight.size();
                lock.unlock();
                const int rc = launch_batch(S, b);
                lock.lock();
                if (rc != HC_OK) b->status = rc;
                continue;
            }
        }
        // nothing to do right now: wait for a submission or poll the GPU
        if (S->inflight.empty())
            S->cv_work.wait_for(lock, std::chrono::milliseconds(5));
        else
            S->cv_work.wait_for(lock, std::chrono::microseconds(20));
    }
}

void destroy_server(hc_server* S) {
    if (!S) return;
    if (S->dispatcher.joinable()) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        S->dispatcher.join();
    }
    for (auto& kv : S->live) delete kv.second;
    for (cudaStream_t st : S->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : S->events)
        if (e) cudaEventDestroy(e);
    if (S->arena_dev) cudaFree(S->arena_dev);
    if (S->arena_host) cudaFreeHost(S->arena_host);
    delete S->arena;
    cudaGetLastError();
    delete S;
}

}  // namespace

extern "C" {

HC_API int hc_serve_create_ex(hc_index* const* idx, uint32_t n_idx, uint64_t hbm_budget,
                              const hc_serve_params* params, hc_server** out) {
    if (!out) return HC_ERR_ARG;
    *out = nullptr;
    if (!idx || n_idx < 1 || hbm_budget < 4096) return HC_ERR_ARG;
    for (uint32_t i = 0; i < n_idx; ++i)
        if (!idx[i]) return HC_ERR_ARG;
    hc_serve_params P{4, 16384, 128, 200};
    if (params) P = *params;
    if (P.streams < 1 || P.streams > 16 || P.max_batch_queries < 1 || P.default_p < 1 ||
        P.default_p > (1u << 30))
        return HC_ERR_ARG;
    // the server's streams do not wait on the streams that built the
    // indexes: let every build queued so far finish first
    if (cudaDeviceSynchronize() != cudaSuccess) return HC_ERR_CUDA;
    hc_server* S = new (std::nothrow) hc_server();
    if (!S) return HC_ERR_OOM;
    S->idx.assign(idx, idx + n_idx);
    S->pred.assign(n_idx, Predictor());
    S->budget = hbm_budget;
    S->params = P;
    cudaGetDevice(&S->device);
    int rc = HC_OK;
    if (alloc_should_fail() || cudaMalloc(&S->arena_dev, hbm_budget) != cudaSuccess)
        rc = HC_ERR_OOM;
    if (!rc && (alloc_should_fail() ||
                cudaHostAlloc(&S->arena_host, hbm_budget, cudaHostAllocDefault) != cudaSuccess))
        rc = HC_ERR_OOM;
    if (rc) {
        cudaGetLastError();
        destroy_server(S);
        return rc;
    }
    S->arena = new Arena(hbm_budget);
    S->streams.assign(P.streams, nullptr);
    S->events.assign(P.streams, nullptr);
    S->slot_busy.assign(P.streams, false);
    for (uint32_t s = 0; s < P.streams; ++s)
        if (cudaStreamCreateWithFlags(&S->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->events[s], cudaEventDisableTiming) != cudaSuccess) {
            destroy_server(S);
            return HC_ERR_CUDA;
        }
    S->dispatcher = std::thread(dispatcher_loop, S);
    *out = S;
    return HC_OK;
}

HC_API int hc_serve_create(hc_index* const* idx, uint32_t n_idx, uint64_t hbm_budget,
                           hc_server** out) {
    return hc_serve_create_ex(idx, n_idx, hbm_budget, nullptr, out);
}

HC_API int hc_serve_submit(hc_server* S, uint32_t index_id, const void* q_host, uint32_t nq,
                           uint32_t k, uint32_t p, uint64_t* ticket) {
    if (!S || !q_host || !ticket || nq < 1 || k < 1 || k > 128 || p > (1u << 30))
        return HC_ERR_ARG;
    if (index_id >= S->idx.size()) return HC_ERR_ARG;
    const uint32_t rb = S->idx[index_id]->row_bytes;
    if (request_bytes(nq, k, rb) > S->budget) return HC_ERR_BUDGET;
    Request* r = new (std::nothrow) Request();
    if (!r) return HC_ERR_OOM;
    r->index_id = index_id;
    r->nq = nq;
    r->k = k;
    r->p = p;
    r->q.assign(static_cast<const uint8_t*>(q_host),
                static_cast<const uint8_t*>(q_host) + (size_t)nq * rb);
    r->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return HC_ERR_STATE;
        }
        r->ticket = S->next_ticket++;
        S->live[r->ticket] = r;
        S->queue.push_back(r);
        S->queued_queries += nq;
        S->stats.requests += 1;
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return HC_OK;
}

HC_API int hc_serve_poll_ex(hc_server* S, uint64_t ticket, int32_t* ids_host, void* dist_host,
                            uint32_t timeout_us, uint64_t* latency_ns) {
    if (!S) return HC_ERR_ARG;
    uint64_t lat = 0;
    int rc;
    {
        std::unique_lock<std::mutex> lock(S->mu);
        auto it = S->live.find(ticket);
        if (it == S->live.end()) return HC_ERR_STATE;
        Request* r = it->second;
        if (r->status == HC_PENDING && timeout_us > 0)
            S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us),
                                [&] { return r->status != HC_PENDING; });
        if (r->status == HC_PENDING) return HC_PENDING;
        rc = r->status;
        lat = r->t_done - r->t_submit;
        if (rc == HC_OK) {
            if (!ids_host || !dist_host) return HC_ERR_ARG;
            std::memcpy(ids_host, r->ids.data(), r->ids.size() * sizeof(int32_t));
            std::memcpy(dist_host, r->dist.data(), r->dist.size() * sizeof(uint32_t));
        }
        S->live.erase(it);
        delete r;
    }
    if (latency_ns) *latency_ns = lat;
    return rc;
}

HC_API int hc_serve_poll(hc_server* S, uint64_t ticket, int32_t* ids_host, void* dist_host,
                         uint32_t timeout_us) {
    return hc_serve_poll_ex(S, ticket, ids_host, dist_host, timeout_us, nullptr);
}

HC_API int hc_serve_attach_predictor(hc_server* S, uint32_t index_id, hc_mlp* mlp, float margin,
                                     uint32_t p_lo, uint32_t p_hi) {
    if (!S || index_id >= S->idx.size() || p_lo > p_hi || p_hi > (1u << 30)) return HC_ERR_ARG;
    const hc_index* ix = S->idx[index_id];
    if (mlp) {
        if (ix->params.dtype != HC_U8 || ix->params.partitions != 1 || ix->params.curves > 16)
            return HC_ERR_ARG;
        if (int rc = mlp_prepare_inference(mlp, ix, S->streams[0])) return rc;
    }
    std::lock_guard<std::mutex> g(S->mu);
    Predictor& p = S->pred[index_id];
    p.mlp = mlp;
    p.margin = margin;
    p.p_lo = p_lo;
    p.p_hi = p_hi;
    return HC_OK;
}

HC_API int hc_serve_stats_get(hc_server* S, hc_serve_stats* out) {
    if (!S || !out) return HC_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->stats;
    out->arena_used = S->arena->used();
    out->queued_queries = S->queued_queries;
    return HC_OK;
}

HC_API void hc_serve_destroy(hc_server* S) { destroy_server(S); }

}  // extern "C"
