// Continuous-batching request loop for several resident spectrum databases.
//
// The paper's server answers batches of q-bar queries per database with one
// kernel per batch (Alg. 3 / Alg. 4, Sec. 5.2).  Here the server runs as a
// native request loop:
//  - submit() admits a request by memory: its query and answer live in a
//    mapped pinned host arena (first-fit, coalescing); if the arena or the
//    in-flight limit is full, submit returns QPADL_EBUSY (the caller retries).
//  - one loop thread forms launches as requests arrive: whenever a launch
//    stream is free it picks the database whose oldest queued request has
//    waited longest (among databases with no launch in flight: a handle's
//    scratch serves one launch at a time), takes up to max_batch of its
//    queued requests, carves the batch buffers from a device arena, and
//    enqueues on that stream: a gather kernel that pulls every query
//    straight from pinned host memory, the batched Response (the streaming
//    kernel for tiny batches, the exact tensor-core GEMM otherwise), and a
//    scatter kernel that writes every answer straight into its request's
//    pinned buffer.  A host callback at the end of the stream marks the
//    requests done and frees the device region.
//  - several launch streams let launches of different databases run at the
//    same time and new arrivals start while earlier launches are still on
//    the GPU (continuous batching, not a single queue).
//  - a watchdog fails requests whose launch has not completed within
//    watchdog_ms (their buffers stay reserved until the GPU really finishes).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "qpadl_pir.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over a byte range [0, size), 256-byte granules, coalescing frees.
class RangeAllocator {
  public:
    void reset(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = (bytes + 255) & ~uint64_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes;
                const uint64_t roff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + 255) & ~uint64_t(255);
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
    uint64_t used() const { return used_; }
    uint64_t size() const { return size_; }

  private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t size_ = 0, used_ = 0;
};

enum ReqState { kQueued = 0, kLaunched = 1, kDone = 2, kFailed = 3 };

struct Request {
    uint64_t ticket = 0;
    int db = 0;
    int state = kQueued;
    int error = QPADL_OK;
    double t_submit = 0, t_launch = 0, t_done = 0;
    uint64_t host_off = 0, host_bytes = 0;   // query (C words) then answer (R words) in the pinned arena
    uint32_t *q = nullptr;
    uint32_t *a = nullptr;
};

struct DbEntry {
    qpadl_db *db = nullptr;
    uint64_t R = 0, C = 0;
    std::deque<Request *> queue;
    bool busy = false;   // a launch of this database is in flight
};

struct Launch;

struct StreamSlot {
    cudaStream_t stream = nullptr;
    Launch *busy = nullptr;
    // per-slot pointer tables in mapped pinned memory, read by the gather/scatter kernels
    const uint32_t **q_src = nullptr;
    uint32_t **a_dst = nullptr;
    uint32_t table_cap = 0;
};

struct Group {
    int db;
    uint32_t first, count;   // requests [first, first+count) of the launch
    uint64_t dq_off, da_off; // device batch buffers (arena offsets)
};

struct Launch {
    qpadl_server *srv = nullptr;
    int slot = 0;
    uint64_t id = 0;
    double t_launch = 0;
    std::vector<Request *> reqs;
    std::vector<Group> groups;
    uint64_t dev_off = 0, dev_bytes = 0;
    bool failed_by_watchdog = false;
    bool gpu_done = false;
    bool drop_completion = false;   // test hook: the completion is not reported to requests
};

// Copies queries of a launch from pinned host memory into the device batch
// buffer: block (x, b) copies part of query b.
__global__ void gather_queries_kernel(const uint32_t *const *src, uint32_t *dst, uint64_t C) {
    const uint32_t b = blockIdx.y;
    const uint32_t *s = src[b];
    uint32_t *d = dst + (uint64_t)b * C;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < C; j += (uint64_t)gridDim.x * blockDim.x)
        d[j] = s[j];
}

__global__ void scatter_answers_kernel(const uint32_t *src, uint32_t *const *dst, uint64_t R) {
    const uint32_t b = blockIdx.y;
    uint32_t *d = dst[b];
    const uint32_t *s = src + (uint64_t)b * R;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += (uint64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

}  // namespace

struct qpadl_server {
    qpadl_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<DbEntry> dbs;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1, next_launch = 1;
    uint32_t inflight = 0;       // admitted and not yet polled
    uint32_t queued = 0;
    RangeAllocator host_alloc, dev_alloc;
    uint8_t *host_arena = nullptr;
    uint8_t *dev_arena = nullptr;
    std::vector<StreamSlot> slots;
    std::vector<Launch *> active;
    std::thread loop;
    bool stop = false;
    bool started = false;
    // counters
    uint64_t n_launches = 0, n_done = 0, n_failed = 0, n_busy = 0;
    double busy_batch_sum = 0;

    void run();
    bool form_launch(int slot_idx, std::unique_lock<std::mutex> &lk);
    void complete(Launch *L);
    void finalize(Launch *L);
};

namespace {

void CUDART_CB on_launch_done(void *arg) {
    Launch *L = static_cast<Launch *>(arg);
    L->srv->complete(L);
}

}  // namespace

// Called (from the CUDA callback thread) once the GPU has finished a launch.
void qpadl_server::complete(Launch *L) {
    std::lock_guard<std::mutex> g(mu);
    L->gpu_done = true;
    // a dropped completion (test hook) is not reported: the launch stays
    // active and holds its stream until the watchdog fails it
    if (L->drop_completion && !L->failed_by_watchdog) return;
    finalize(L);
}

// Reports a finished launch and releases what it holds (lock held).
void qpadl_server::finalize(Launch *L) {
    const double t = now_s();
    if (!L->failed_by_watchdog) {
        for (Request *r : L->reqs) {
            r->state = kDone;
            r->t_done = t;
        }
        n_done += L->reqs.size();
    }
    dev_alloc.release(L->dev_off, L->dev_bytes);
    slots[L->slot].busy = nullptr;
    for (const Group &g : L->groups) dbs[g.db].busy = false;
    active.erase(std::remove(active.begin(), active.end(), L), active.end());
    // requests failed by the watchdog and already polled kept their host
    // buffers reserved until the GPU was done with them
    for (Request *r : L->reqs) {
        if (r->state == kFailed && r->ticket == 0) {
            host_alloc.release(r->host_off, r->host_bytes);
            delete r;
        }
    }
    delete L;
    cv.notify_all();
}

bool qpadl_server::form_launch(int si, std::unique_lock<std::mutex> &lk) {
    // the database whose oldest queued request has waited longest, among those
    // with no launch in flight (a handle's scratch serves one launch at a time)
    int d = -1;
    double oldest = 0;
    for (int k = 0; k < static_cast<int>(dbs.size()); ++k) {
        DbEntry &e = dbs[k];
        if (e.queue.empty() || e.busy) continue;
        if (d < 0 || e.queue.front()->t_submit < oldest) {
            d = k;
            oldest = e.queue.front()->t_submit;
        }
    }
    if (d < 0) return false;
    DbEntry &e = dbs[d];
    const uint32_t take = static_cast<uint32_t>(std::min<size_t>(e.queue.size(), cfg.max_batch));
    const uint64_t qbytes = (4ull * take * e.C + 255) & ~255ull;
    const uint64_t need = qbytes + ((4ull * take * e.R + 255) & ~255ull);
    uint64_t off = 0;
    if (!dev_alloc.alloc(need, &off)) return false;   // wait for a launch to free device memory
    Launch *L = new Launch();
    L->srv = this;
    L->slot = si;
    L->id = next_launch++;
    L->dev_off = off;
    L->dev_bytes = need;
    L->groups.push_back(Group{d, 0, take, 0, qbytes});
    for (uint32_t i = 0; i < take; ++i) {
        L->reqs.push_back(e.queue.front());
        e.queue.pop_front();
    }
    e.busy = true;
    queued -= take;
    L->t_launch = now_s();
    for (Request *r : L->reqs) {
        r->state = kLaunched;
        r->t_launch = L->t_launch;
    }
    if (cfg.test_drop_completion_launch && L->id == cfg.test_drop_completion_launch) L->drop_completion = true;
    StreamSlot &S = slots[si];
    S.busy = L;
    active.push_back(L);
    ++n_launches;
    busy_batch_sum += static_cast<double>(take);
    // enqueue the GPU work without holding the lock
    lk.unlock();
    for (uint32_t i = 0; i < take; ++i) {
        S.q_src[i] = L->reqs[i]->q;
        S.a_dst[i] = L->reqs[i]->a;
    }
    uint32_t *dq = reinterpret_cast<uint32_t *>(dev_arena + off);
    uint32_t *da = reinterpret_cast<uint32_t *>(dev_arena + off + qbytes);
    const unsigned bx = static_cast<unsigned>(std::min<uint64_t>((e.C + 1023) / 1024, 32));
    gather_queries_kernel<<<dim3(bx, take), 256, 0, S.stream>>>(S.q_src, dq, e.C);
    bool ok = cudaGetLastError() == cudaSuccess;
    ok = ok && qpadl_pir_answer_batch(e.db, dq, take, da, S.stream) == QPADL_OK;
    const unsigned by = static_cast<unsigned>(std::min<uint64_t>((e.R + 1023) / 1024, 32));
    if (ok) {
        scatter_answers_kernel<<<dim3(by, take), 256, 0, S.stream>>>(da, S.a_dst, e.R);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (!ok) {
        lk.lock();
        for (Request *r : L->reqs) {
            r->state = kFailed;
            r->error = QPADL_ECUDA;
        }
        n_failed += take;
        L->failed_by_watchdog = true;   // completion must not overwrite the failure
        lk.unlock();
    }
    // the callback runs after every kernel above and releases slot, database and memory
    if (cudaLaunchHostFunc(S.stream, on_launch_done, L) != cudaSuccess) {
        cudaStreamSynchronize(S.stream);
        complete(L);
    }
    lk.lock();
    return true;
}

void qpadl_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        // watchdog: fail the requests of launches that have not completed in
        // time; their buffers stay reserved until the GPU is really done
        const double t = now_s();
        std::vector<Launch *> finished;
        for (Launch *L : active) {
            if (!L->failed_by_watchdog && t - L->t_launch > cfg.watchdog_ms * 1e-3) {
                L->failed_by_watchdog = true;
                for (Request *r : L->reqs) {
                    if (r->state == kLaunched) {
                        r->state = kFailed;
                        r->error = QPADL_ETIMEOUT;
                        ++n_failed;
                    }
                }
                if (L->gpu_done) finished.push_back(L);
            }
        }
        for (Launch *L : finished) finalize(L);
        int free_slot = -1;
        for (size_t i = 0; i < slots.size(); ++i)
            if (!slots[i].busy) {
                free_slot = static_cast<int>(i);
                break;
            }
        if (queued > 0 && free_slot >= 0) {
            // optionally hold a short while so a lone request can gather company
            bool hold = false;
            if (cfg.hold_us > 0 && !active.empty()) {
                double oldest = t;
                for (auto &e : dbs)
                    if (!e.queue.empty()) oldest = std::min(oldest, e.queue.front()->t_submit);
                hold = (t - oldest) * 1e6 < cfg.hold_us && queued < cfg.max_batch;
            }
            if (!hold) {
                if (form_launch(free_slot, lk)) continue;
            }
        }
        cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

extern "C" {

int qpadl_server_create(const qpadl_server_config *cfg, qpadl_server **out) {
    if (!cfg || !out) return QPADL_EINVAL;
    *out = nullptr;
    if (cfg->max_batch == 0 || cfg->max_inflight == 0 || cfg->num_streams == 0 || cfg->num_streams > 8 ||
        cfg->host_budget_bytes < 4096 || cfg->device_budget_bytes < 4096 || cfg->max_batch > 65535)
        return QPADL_EINVAL;
    qpadl_server *s = new (std::nothrow) qpadl_server();
    if (!s) return QPADL_ENOMEM;
    s->cfg = *cfg;
    if (s->cfg.watchdog_ms <= 0) s->cfg.watchdog_ms = 10000.0;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return QPADL_ECUDA;
    }
    if (cudaHostAlloc(reinterpret_cast<void **>(&s->host_arena), cfg->host_budget_bytes, cudaHostAllocMapped) !=
        cudaSuccess) {
        cudaGetLastError();
        delete s;
        return QPADL_ENOMEM;
    }
    if (cudaMalloc(reinterpret_cast<void **>(&s->dev_arena), cfg->device_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(s->host_arena);
        delete s;
        return QPADL_ENOMEM;
    }
    s->host_alloc.reset(cfg->host_budget_bytes);
    s->dev_alloc.reset(cfg->device_budget_bytes);
    s->slots.resize(cfg->num_streams);
    const uint32_t cap = std::min<uint32_t>(cfg->max_inflight, 65536u) * 4;
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.q_src), cap * sizeof(void *), cudaHostAllocMapped) !=
                cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.a_dst), cap * sizeof(void *), cudaHostAllocMapped) !=
                cudaSuccess) {
            cudaGetLastError();
            qpadl_server_destroy(s);
            return QPADL_ECUDA;
        }
        sl.table_cap = cap;
    }
    *out = s;
    return QPADL_OK;
}

int qpadl_server_add_db(qpadl_server *s, qpadl_db *db, int *db_id) {
    if (!s || !db || !db_id) return QPADL_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->started) return QPADL_EINVAL;
    uint64_t R = 0, C = 0;
    if (qpadl_pir_shape(db, &R, &C) != QPADL_OK) return QPADL_EINVAL;
    // size the handle's scratch for the largest batch now, so launches never allocate
    if (qpadl_pir_reserve(db, s->cfg.max_batch, nullptr) != QPADL_OK) return QPADL_ENOMEM;
    DbEntry e;
    e.db = db;
    e.R = R;
    e.C = C;
    s->dbs.push_back(e);
    *db_id = static_cast<int>(s->dbs.size() - 1);
    return QPADL_OK;
}

int qpadl_server_start(qpadl_server *s) {
    if (!s) return QPADL_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->started) return QPADL_OK;
    if (s->dbs.empty()) return QPADL_EINVAL;
    s->started = true;
    s->loop = std::thread([s] { s->run(); });
    return QPADL_OK;
}

int qpadl_server_submit(qpadl_server *s, int db_id, const uint32_t *q_host, uint64_t *ticket) {
    if (!s || !q_host || !ticket) return QPADL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->started || db_id < 0 || db_id >= static_cast<int>(s->dbs.size())) return QPADL_EINVAL;
    DbEntry &e = s->dbs[db_id];
    if (s->inflight >= s->cfg.max_inflight) {
        ++s->n_busy;
        return QPADL_EBUSY;
    }
    const uint64_t bytes = 4ull * (e.C + e.R) + 256;
    uint64_t off = 0;
    if (!s->host_alloc.alloc(bytes, &off)) {
        ++s->n_busy;
        return QPADL_EBUSY;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) {
        s->host_alloc.release(off, bytes);
        return QPADL_ENOMEM;
    }
    r->ticket = s->next_ticket++;
    r->db = db_id;
    r->host_off = off;
    r->host_bytes = bytes;
    r->q = reinterpret_cast<uint32_t *>(s->host_arena + off);
    r->a = reinterpret_cast<uint32_t *>(s->host_arena + off + ((4ull * e.C + 255) & ~255ull));
    r->t_submit = now_s();
    s->reqs[r->ticket] = r;
    ++s->inflight;
    lk.unlock();
    std::memcpy(r->q, q_host, 4ull * e.C);   // outside the lock; the request is not queued yet
    lk.lock();
    e.queue.push_back(r);
    ++s->queued;
    *ticket = r->ticket;
    s->cv.notify_all();
    return QPADL_OK;
}

int qpadl_server_poll(qpadl_server *s, uint64_t ticket, uint32_t *ans_host, qpadl_request_times *times) {
    if (!s) return QPADL_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return QPADL_EINVAL;
    Request *r = it->second;
    if (r->state == kQueued || r->state == kLaunched) return QPADL_EAGAIN;
    const int rc = r->state == kDone ? QPADL_OK : r->error;
    if (times) {
        times->submit_s = r->t_submit;
        times->launch_s = r->t_launch;
        times->done_s = r->t_done;
    }
    if (r->state == kDone && ans_host) std::memcpy(ans_host, r->a, 4ull * s->dbs[r->db].R);
    s->reqs.erase(it);
    --s->inflight;
    bool in_flight_on_gpu = false;
    if (r->state == kFailed) {
        for (Launch *L : s->active)
            for (Request *x : L->reqs)
                if (x == r) in_flight_on_gpu = true;
    }
    if (in_flight_on_gpu) {
        r->ticket = 0;   // the completion callback releases its buffers later
    } else {
        s->host_alloc.release(r->host_off, r->host_bytes);
        delete r;
    }
    return rc;
}

int qpadl_server_stats(qpadl_server *s, qpadl_server_stats_t *st) {
    if (!s || !st) return QPADL_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    st->launches = s->n_launches;
    st->completed = s->n_done;
    st->failed = s->n_failed;
    st->refused = s->n_busy;
    st->inflight = s->inflight;
    st->queued = s->queued;
    st->mean_launch_requests = s->n_launches ? s->busy_batch_sum / static_cast<double>(s->n_launches) : 0.0;
    st->host_bytes_used = s->host_alloc.used();
    st->device_bytes_used = s->dev_alloc.used();
    return QPADL_OK;
}

int qpadl_server_destroy(qpadl_server *s) {
    if (!s) return QPADL_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->loop.joinable()) s->loop.join();
    for (auto &sl : s->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    {
        // every callback has run once its stream drained
        std::lock_guard<std::mutex> g(s->mu);
        for (auto &kv : s->reqs) delete kv.second;
        s->reqs.clear();
    }
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.q_src) cudaFreeHost(sl.q_src);
        if (sl.a_dst) cudaFreeHost(sl.a_dst);
    }
    if (s->dev_arena) cudaFree(s->dev_arena);
    if (s->host_arena) cudaFreeHost(s->host_arena);
    delete s;
    return QPADL_OK;
}

// Open-loop load generator: submits request i at t0 + arrival_s[i] (retrying
// while admission refuses), polls completions and records per-request
// latency = completion time - scheduled arrival time.
int qpadl_server_replay(qpadl_server *s, uint64_t n, const double *arrival_s, const int32_t *db_ids,
                        const uint32_t *const *q_host, uint32_t *const *ans_host, double *latency_s,
                        int32_t *status) {
    if (!s || !arrival_s || !db_ids || !q_host || !latency_s || !status) return QPADL_EINVAL;
    std::vector<uint64_t> tickets(n, 0);
    std::atomic<uint64_t> submitted{0};
    std::atomic<int> submit_err{QPADL_OK};
    const double t0 = now_s();
    std::thread submitter([&] {
        for (uint64_t i = 0; i < n; ++i) {
            const double due = t0 + arrival_s[i];
            while (now_s() < due) {
            }
            uint64_t tk = 0;
            int rc;
            while ((rc = qpadl_server_submit(s, db_ids[i], q_host[i], &tk)) == QPADL_EBUSY) {
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            }
            if (rc != QPADL_OK) {
                submit_err = rc;
                tk = 0;
            }
            tickets[i] = tk;
            submitted.store(i + 1, std::memory_order_release);
        }
    });
    uint64_t done = 0;
    std::vector<char> finished(n, 0);
    uint64_t scan_from = 0;
    while (done < n) {
        const uint64_t avail = submitted.load(std::memory_order_acquire);
        bool progress = false;
        for (uint64_t i = scan_from; i < avail; ++i) {
            if (finished[i]) continue;
            if (tickets[i] == 0) {
                finished[i] = 1;
                status[i] = submit_err.load();
                latency_s[i] = -1;
                ++done;
                progress = true;
                continue;
            }
            qpadl_request_times tm;
            const int rc = qpadl_server_poll(s, tickets[i], ans_host ? ans_host[i] : nullptr, &tm);
            if (rc == QPADL_EAGAIN) continue;
            finished[i] = 1;
            status[i] = rc;
            latency_s[i] = (rc == QPADL_OK) ? tm.done_s - (t0 + arrival_s[i]) : -1;
            ++done;
            progress = true;
        }
        while (scan_from < avail && finished[scan_from]) ++scan_from;
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    submitter.join();
    return QPADL_OK;
}

}  // extern "C"
