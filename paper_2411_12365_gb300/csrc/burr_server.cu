// burr_server.cu -- a build/query request server on one GPU (continuous
// batching of the many-small-structures use of retrieval, Sec. 1).
//
// Worker threads share the device:
//   * each build worker (cfg.build_workers of them, one stream each) takes
//     every queued build request that the memory budget admits (its estimate
//     fits next to the resident structures and the builds in flight) and
//     builds them together: one burr_build_batch call per value width, inputs
//     copied straight from each request's host buffer into the batch's device
//     arrays; structures too large for a batch get burr_build of their own.
//     Requests that arrive while a batch is on the GPU are taken by an idle
//     build worker at once, so batches overlap on the device; with every
//     worker busy they join the next batch;
//   * the query worker runs each query on its own stream as soon as the
//     structure it targets is resident, overlapping the build worker's
//     kernels.
// Request payloads are copied at submission into a page-locked staging
// region (DMA-able, so the host-to-device copies run at link speed), or into
// pageable memory when the region is full.  Built structures stay resident
// until released.  Every request records its latency from submission to
// completion.  The partition size is fixed by the server's parameters, so a
// structure's export does not depend on which other requests shared its
// batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "burr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

uint32_t vbytes_of(uint32_t r) { return r <= 8 ? 1u : (r <= 16 ? 2u : 4u); }
uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t first_layer_slots(uint64_t n, double alpha) {
    if (n == 0) return 0;
    return ((uint64_t)std::ceil((double)n / alpha) + 64 + 63) & ~63ull;
}

// Device bytes a build of n keys holds at its peak: the input copies, the
// sorted copies and the sort's scratch, the band of every partition, the
// bumped lists and the tables (a conservative model of the build's arena).
uint64_t build_estimate(uint64_t n, uint32_t r, double alpha) {
    const uint64_t vb = vbytes_of(r);
    const uint64_t m = first_layer_slots(n, alpha);
    return n * (8 + vb) * 4 + m * (8 + vb) * 2 + (m / 64) * r * 8 + (1u << 20);
}

// Page-locked host region carved first-fit into blocks (caller holds the lock).
struct Staging {
    uint8_t *base = nullptr;
    std::map<uint64_t, uint64_t> free_;   // offset -> bytes, coalesced

    void init(uint64_t bytes) {
        if (bytes == 0) return;
        if (cudaHostAlloc((void **)&base, bytes, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;   // no staging: every payload goes to pageable memory
            return;
        }
        free_[0] = bytes;
    }
    uint8_t *alloc(uint64_t bytes) {
        if (!base) return nullptr;
        bytes = align_up(std::max<uint64_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            return base + off;
        }
        return nullptr;
    }
    void release(uint8_t *p, uint64_t bytes) {
        if (!p) return;
        bytes = align_up(std::max<uint64_t>(bytes, 1), 256);
        uint64_t off = (uint64_t)(p - base);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    ~Staging() {
        if (base) cudaFreeHost(base);
    }
};

struct Request {
    uint64_t id = 0;
    bool is_build = true;
    uint64_t n = 0;
    uint32_t r = 8;                   // build: value bits; query: the target's
    // payload: n keys, then (from byte align16(8n)) n values of a build or the
    // n results of a query; page-locked when `stage` is set, else in `heap`
    uint8_t *stage = nullptr;
    uint64_t payload_bytes = 0;
    std::vector<uint8_t> heap;
    uint64_t bytes = 0;               // build: estimate while queued, table bytes once resident
    burr_handle *handle = nullptr;    // build: the resident structure
    uint64_t target = 0;              // query: build ticket of the structure
    void *out = nullptr;              // query: caller's host output
    int status = 1;                   // 1 pending, 0 done, < 0 error code
    std::string message;              // error message of a failed request
    Clock::time_point t_submit, t_done;

    uint8_t *payload() { return stage ? stage : heap.data(); }
    const uint64_t *keys() { return (const uint64_t *)payload(); }
    uint8_t *tail() { return payload() + align_up(n * 8, 16); }
};

}  // namespace

struct burr_server {
    burr_params params;
    burr_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> build_queue, query_queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_id = 1;
    uint64_t bytes_resident = 0, bytes_inflight = 0;
    uint64_t running_query_target = 0;   // build ticket of the query in progress
    uint64_t batches = 0, batched_structures = 0, staged = 0, pageable = 0, built_keys = 0;
    double build_busy_ms = 0, query_busy_ms = 0;
    uint64_t running_builds = 0, max_running_builds = 0;   // admitted batches on the device
    Staging staging;
    bool stop = false;
    std::vector<std::thread> build_threads;
    std::thread query_thread;
    std::vector<cudaStream_t> build_streams;
    cudaStream_t query_stream = nullptr;
};

namespace {

// Payload space for a request: staging if it has room, else pageable memory.
// Called without the lock held; returns false if host memory ran out.
bool make_payload(burr_server *S, Request &q, uint32_t tail_bytes_per_key) {
    q.payload_bytes = align_up(q.n * 8, 16) + q.n * tail_bytes_per_key;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q.stage = S->staging.alloc(q.payload_bytes);
        (q.stage ? S->staged : S->pageable) += 1;
    }
    if (q.stage) return true;
    try {
        q.heap.resize(q.payload_bytes);
    } catch (...) {
        return false;
    }
    return true;
}

// Under the lock: record the outcome and give back the payload space.
void finish(burr_server *S, Request &q, int status, const char *msg) {
    q.status = status;
    if (status < 0) q.message = msg ? msg : "";
    q.t_done = Clock::now();
    if (q.stage) S->staging.release(q.stage, q.payload_bytes);
    q.stage = nullptr;
    q.heap.clear();
    q.heap.shrink_to_fit();
}

// Take every queued build that fits the budget, in arrival order (one that
// does not fit waits; later ones that fit may pass it).  Under the lock.
std::vector<std::shared_ptr<Request>> admit(burr_server *S) {
    std::vector<std::shared_ptr<Request>> batch;
    std::deque<uint64_t> rest;
    uint64_t keys_in_batch = 0;
    for (uint64_t id : S->build_queue) {
        auto &q = S->reqs[id];
        const bool fits = S->bytes_resident + S->bytes_inflight + q->bytes <= S->cfg.memory_budget;
        if (fits && batch.size() < S->cfg.max_batch_structures && keys_in_batch + q->n < (1ull << 32)) {
            S->bytes_inflight += q->bytes;
            keys_in_batch += q->n;
            batch.push_back(q);
        } else {
            rest.push_back(id);
        }
    }
    S->build_queue.swap(rest);
    return batch;
}

int build_solo(burr_server *S, Request &q, cudaStream_t st) {
    burr_handle *h = nullptr;
    const int rc = burr_build(q.keys(), q.tail(), q.n, q.r, &S->params, st, &h);
    q.handle = rc == BURR_OK ? h : nullptr;
    if (rc) q.message = burr_last_error();
    return rc;
}

// One burr_build_batch over requests of one value width: their payloads are
// copied into the batch's device arrays, then built in one pass.
int build_group(burr_server *S, std::vector<Request *> &g, uint32_t vb, cudaStream_t st) {
    std::vector<uint64_t> offs(g.size() + 1, 0);
    std::vector<uint32_t> rs(g.size());
    for (size_t j = 0; j < g.size(); ++j) {
        offs[j + 1] = offs[j] + g[j]->n;
        rs[j] = g[j]->r;
    }
    const uint64_t N = offs.back();
    uint64_t *dk = nullptr;
    uint8_t *dv = nullptr;
    if (N) {
        if (burr::dev_alloc((void **)&dk, N * 8, st) != cudaSuccess ||
            burr::dev_alloc((void **)&dv, N * vb, st) != cudaSuccess) {
            cudaGetLastError();
            if (dk) burr::dev_free_async(dk, st);
            return burr::set_error(BURR_ERR_OOM, "batch input allocation failed");
        }
        for (size_t j = 0; j < g.size(); ++j) {
            if (!g[j]->n) continue;
            if (cudaMemcpyAsync(dk + offs[j], g[j]->keys(), g[j]->n * 8, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(dv + offs[j] * vb, g[j]->tail(), g[j]->n * vb, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess) {
                burr::dev_free_async(dk, st);
                burr::dev_free_async(dv, st);
                return burr::set_error(BURR_ERR_CUDA, "batch input copy failed");
            }
        }
    }
    std::vector<burr_handle *> hs(g.size(), nullptr);
    const int rc = burr_build_batch(dk, dv, offs.data(), rs.data(), (uint32_t)g.size(), &S->params, st, hs.data());
    if (N) {
        burr::dev_free_async(dk, st);
        burr::dev_free_async(dv, st);
    }
    if (rc == BURR_OK)
        for (size_t j = 0; j < g.size(); ++j) g[j]->handle = hs[j];
    return rc;
}

// Build the requests of one admitted batch; returns per-request status.
std::vector<int> build_all(burr_server *S, std::vector<std::shared_ptr<Request>> &batch, cudaStream_t st) {
    std::vector<int> rc(batch.size(), BURR_OK);
    std::vector<Request *> groups[3];   // by value width 1, 2, 4 bytes
    std::vector<size_t> gidx[3];
    for (size_t i = 0; i < batch.size(); ++i) {
        Request &q = *batch[i];
        const uint64_t m = first_layer_slots(q.n, S->params.load_factor);
        const uint64_t nb = m == 0 ? 0 : (m - 64 + 128) / 128;
        if (S->params.bucket_slots == 128 && (nb + 63) / 64 <= burr::kMaxGroupsPerStruct) {
            const int c = q.r <= 8 ? 0 : (q.r <= 16 ? 1 : 2);
            groups[c].push_back(&q);
            gidx[c].push_back(i);
        } else {
            rc[i] = build_solo(S, q, st);
        }
    }
    for (int c = 0; c < 3; ++c) {
        if (groups[c].empty()) continue;
        if (build_group(S, groups[c], 1u << c, st) == BURR_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->batches += 1;
            S->batched_structures += groups[c].size();
        } else {
            // one failing structure fails the whole batch: build each on its
            // own so that only the failing request reports the error
            for (size_t j = 0; j < groups[c].size(); ++j) rc[gidx[c][j]] = build_solo(S, *groups[c][j], st);
        }
    }
    return rc;
}

void build_worker(burr_server *S, size_t idx) {
    cudaSetDevice(S->device);
    cudaStream_t st = S->build_streams[idx];
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop) {
            for (uint64_t id : S->build_queue) finish(S, *S->reqs[id], BURR_ERR_INVALID, "server stopped");
            S->build_queue.clear();
            S->cv_done.notify_all();
            S->cv_work.notify_all();
            return;
        }
        auto batch = admit(S);
        if (batch.empty()) {
            // idle, or waiting for resident structures to be released
            S->cv_work.wait(lk);
            continue;
        }
        S->running_builds += 1;
        S->max_running_builds = std::max(S->max_running_builds, S->running_builds);
        lk.unlock();
        const auto t0 = Clock::now();
        std::vector<int> rc = build_all(S, batch, st);
        const double busy = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        lk.lock();
        S->running_builds -= 1;
        S->build_busy_ms += busy;
        for (auto &q : batch) S->built_keys += q->n;
        for (size_t i = 0; i < batch.size(); ++i) {
            Request &q = *batch[i];
            S->bytes_inflight -= q.bytes;
            if (rc[i] == BURR_OK) {
                uint64_t b = 0;
                burr_size_bytes(q.handle, &b);
                q.bytes = b;
                S->bytes_resident += b;
            } else {
                q.bytes = 0;
            }
            const std::string msg = q.message;
            finish(S, q, rc[i], msg.c_str());
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

void query_worker(burr_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // the oldest query whose structure is no longer pending
        std::shared_ptr<Request> q;
        burr_handle *h = nullptr;
        for (auto it = S->query_queue.begin(); it != S->query_queue.end(); ++it) {
            auto &cand = S->reqs[*it];
            auto tg = S->reqs.find(cand->target);
            if (tg == S->reqs.end() || tg->second->status != 1) {
                q = cand;
                if (tg != S->reqs.end() && tg->second->status == 0) h = tg->second->handle;
                S->query_queue.erase(it);
                break;
            }
        }
        if (!q) {
            if (S->stop && S->build_queue.empty() && S->query_queue.empty()) return;
            S->cv_work.wait(lk);
            continue;
        }
        S->running_query_target = q->target;
        lk.unlock();
        int rc = BURR_ERR_INVALID;
        std::string msg = "the structure failed to build";
        const auto t0 = Clock::now();
        if (h) {
            // host keys and results: returns once the results are in the payload
            rc = burr_query(h, q->keys(), q->tail(), q->n, S->query_stream);
            if (rc) msg = burr_last_error();
            else if (q->n) memcpy(q->out, q->tail(), q->n * vbytes_of(q->r));
        }
        lk.lock();
        S->query_busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        S->running_query_target = 0;
        finish(S, *q, rc, msg.c_str());
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int burr_server_create(const burr_server_config *cfg, const burr_params *p, burr_server **out) {
    if (!out || !cfg) return burr::set_error(BURR_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->memory_budget == 0) return burr::set_error(BURR_ERR_INVALID, "memory_budget is 0");
    burr_params prm;
    if (p) prm = *p;
    else burr_default_params(&prm);
    if (prm.partition_slots == 0)
        return burr::set_error(BURR_ERR_INVALID, "the server needs a fixed partition_slots (> 0)");
    auto *S = new (std::nothrow) burr_server();
    if (!S) return burr::set_error(BURR_ERR_OOM, "host allocation");
    S->cfg = *cfg;
    S->params = prm;
    if (S->cfg.max_batch_structures == 0) S->cfg.max_batch_structures = 4096;
    if (S->cfg.build_workers == 0) S->cfg.build_workers = 1;
    if (S->cfg.build_workers > 8) {
        delete S;
        return burr::set_error(BURR_ERR_INVALID, "build_workers must be at most 8");
    }
    cudaGetDevice(&S->device);
    bool ok = cudaStreamCreateWithFlags(&S->query_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (uint32_t i = 0; ok && i < S->cfg.build_workers; ++i) {
        cudaStream_t b = nullptr;
        ok = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) S->build_streams.push_back(b);
    }
    if (!ok) {
        for (auto b : S->build_streams) cudaStreamDestroy(b);
        if (S->query_stream) cudaStreamDestroy(S->query_stream);
        delete S;
        return burr::set_error(BURR_ERR_CUDA, "stream creation failed");
    }
    S->staging.init(cfg->host_staging_bytes);
    for (size_t i = 0; i < S->build_streams.size(); ++i) S->build_threads.emplace_back(build_worker, S, i);
    S->query_thread = std::thread(query_worker, S);
    *out = S;
    return BURR_OK;
}

int burr_server_submit_build(burr_server *S, const uint64_t *keys, const void *values, uint64_t n, uint32_t r,
                             uint64_t *ticket) {
    if (!S || !ticket || (n && (!keys || !values))) return burr::set_error(BURR_ERR_INVALID, "NULL argument");
    if (r < 1 || r > 32) return burr::set_error(BURR_ERR_INVALID, "r outside [1,32]");
    if (n >= (1ull << 32)) return burr::set_error(BURR_ERR_INVALID, "n >= 2^32");
    auto q = std::make_shared<Request>();
    q->is_build = true;
    q->r = r;
    q->n = n;
    q->bytes = build_estimate(n, r, S->params.load_factor);
    if (q->bytes > S->cfg.memory_budget)
        return burr::set_error(BURR_ERR_OOM, "the build needs more device memory than the server's budget");
    const uint32_t vb = vbytes_of(r);
    if (!make_payload(S, *q, vb)) return burr::set_error(BURR_ERR_OOM, "host allocation");
    if (n) {
        memcpy(q->payload(), keys, n * 8);
        memcpy(q->tail(), values, n * vb);
    }
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        finish(S, *q, BURR_ERR_INVALID, "server stopped");
        return burr::set_error(BURR_ERR_INVALID, "server stopped");
    }
    q->id = S->next_id++;
    S->reqs[q->id] = q;
    S->build_queue.push_back(q->id);
    *ticket = q->id;
    S->cv_work.notify_all();
    return BURR_OK;
}

int burr_server_submit_query(burr_server *S, uint64_t build_ticket, const uint64_t *keys, uint64_t n, void *out,
                             uint64_t *ticket) {
    if (!S || !ticket || (n && (!keys || !out))) return burr::set_error(BURR_ERR_INVALID, "NULL argument");
    auto q = std::make_shared<Request>();
    q->is_build = false;
    q->target = build_ticket;
    q->n = n;
    q->out = out;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto tg = S->reqs.find(build_ticket);
        if (tg == S->reqs.end() || !tg->second->is_build)
            return burr::set_error(BURR_ERR_INVALID, "unknown build ticket");
        q->r = tg->second->r;
    }
    if (!make_payload(S, *q, vbytes_of(q->r))) return burr::set_error(BURR_ERR_OOM, "host allocation");
    if (n) memcpy(q->payload(), keys, n * 8);
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    auto tg = S->reqs.find(build_ticket);
    if (S->stop || tg == S->reqs.end()) {
        finish(S, *q, BURR_ERR_INVALID, "");
        return burr::set_error(BURR_ERR_INVALID, S->stop ? "server stopped" : "unknown build ticket");
    }
    q->id = S->next_id++;
    S->reqs[q->id] = q;
    S->query_queue.push_back(q->id);
    *ticket = q->id;
    S->cv_work.notify_all();
    return BURR_OK;
}

int burr_server_wait(burr_server *S, uint64_t ticket, double *latency_ms) {
    if (!S) return burr::set_error(BURR_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return burr::set_error(BURR_ERR_INVALID, "unknown ticket");
    auto q = it->second;
    S->cv_done.wait(lk, [&] { return q->status != 1; });
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    if (!q->is_build) S->reqs.erase(q->id);   // a query ticket is retired by its wait
    if (q->status < 0) return burr::set_error(q->status, q->message.c_str());
    return BURR_OK;
}

int burr_server_handle(burr_server *S, uint64_t build_ticket, const burr_handle **out) {
    if (!S || !out) return burr::set_error(BURR_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(build_ticket);
    if (it == S->reqs.end() || !it->second->is_build || it->second->status != 0)
        return burr::set_error(BURR_ERR_INVALID, "no resident structure for this ticket");
    *out = it->second->handle;
    return BURR_OK;
}

int burr_server_release(burr_server *S, uint64_t build_ticket) {
    if (!S) return burr::set_error(BURR_ERR_INVALID, "NULL server");
    burr_handle *h = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->reqs.find(build_ticket);
        if (it == S->reqs.end() || !it->second->is_build)
            return burr::set_error(BURR_ERR_INVALID, "unknown build ticket");
        if (it->second->status == 1) return burr::set_error(BURR_ERR_INVALID, "the build is still pending");
        for (uint64_t qid : S->query_queue)
            if (S->reqs[qid]->target == build_ticket)
                return burr::set_error(BURR_ERR_INVALID, "queries on this structure are still queued");
        S->cv_done.wait(lk, [&] { return S->running_query_target != build_ticket; });
        auto q = S->reqs.find(build_ticket);   // the map may have changed during the wait
        if (q == S->reqs.end()) return burr::set_error(BURR_ERR_INVALID, "unknown build ticket");
        h = q->second->handle;
        S->bytes_resident -= q->second->status == 0 ? q->second->bytes : 0;
        S->reqs.erase(q);
    }
    burr_free(h);
    S->cv_work.notify_all();   // memory came free: queued builds may now fit
    return BURR_OK;
}

int burr_server_stats(burr_server *S, burr_server_stats_t *st) {
    if (!S || !st) return burr::set_error(BURR_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof(*st));
    st->bytes_resident = S->bytes_resident;
    st->bytes_inflight = S->bytes_inflight;
    st->queued_builds = S->build_queue.size();
    st->queued_queries = S->query_queue.size();
    st->batches = S->batches;
    st->batched_structures = S->batched_structures;
    st->staged_requests = S->staged;
    st->pageable_requests = S->pageable;
    st->built_keys = S->built_keys;
    st->build_busy_ms = S->build_busy_ms;
    st->query_busy_ms = S->query_busy_ms;
    st->max_concurrent_batches = S->max_running_builds;
    for (auto &kv : S->reqs)
        if (kv.second->is_build && kv.second->status == 0) st->resident_structures += 1;
    return BURR_OK;
}

void burr_server_destroy(burr_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->build_threads)
        if (t.joinable()) t.join();
    S->cv_work.notify_all();
    if (S->query_thread.joinable()) S->query_thread.join();
    for (auto &kv : S->reqs)
        if (kv.second->is_build && kv.second->handle) burr_free(kv.second->handle);
    for (auto b : S->build_streams) cudaStreamDestroy(b);
    cudaStreamDestroy(S->query_stream);
    delete S;   // frees the staging region
}

}  // extern "C"
