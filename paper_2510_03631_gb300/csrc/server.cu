// Continuous-batching request loop for several resident spectrum databases.
//
// The paper's server answers batches of q-bar queries per database with one
// kernel per batch (Alg. 3 / Alg. 4, Sec. 5.2).  Here the server runs as a
// native request loop:
//  - submit() admits a request by memory: its query and answer live in a
//    mapped pinned host arena (first-fit, coalescing); if the arena or the
//    in-flight limit is full, submit returns QPADL_EBUSY (the caller retries).
//  - one loop thread forms launches as requests arrive: whenever a launch
//    stream is free it takes up to max_batch queued requests of the database
//    holding the oldest request and of every other database of about the
//    same size (group_size_ratio), carves a workspace for them from a device
//    arena, and enqueues on that stream one grouped cycle: a gather kernel that pulls every
//    query straight from pinned host memory; ONE grouped exact byte-limb
//    GEMM over the uint8 digits of every database in the cycle, however
//    uneven their counts (the tiles of every database form one work list
//    dealt over the SMs); the streaming kernel when the cycle holds a lone
//    database with 1 or 2 queries (two in one pass); the fp16-copy GEMM only
//    for a database with more queries than its uint8-digit GEMM limit; and a
//    scatter kernel that writes every answer
//    straight into its request's pinned buffer.  A host callback at the end
//    of the stream marks the requests done and frees the workspace.
//  - each launch uses only its own workspace (the handles' operand copies
//    are read-only), so launches of the same database overlap on several
//    streams: new arrivals start while earlier launches are still running
//    (continuous batching, not a single queue).
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

#include "internal.cuh"
#include "limb_gemm.cuh"
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

// One copy job per request of a launch: n words from src to dst.
struct CopyJob {
    const uint32_t *src;
    uint32_t *dst;
    uint64_t n;
};

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
    uint64_t R = 0, C = 0, pitch = 0;
    uint32_t u8_max = 0;     // largest group the uint8-digit GEMM takes (QPADL_OPT_U8_MAX_BATCH)
    std::deque<Request *> queue;
};

struct Launch;

struct StreamSlot {
    cudaStream_t stream = nullptr;
    Launch *busy = nullptr;
    // per-slot job tables in mapped pinned memory, read by the gather/scatter kernels
    CopyJob *q_jobs = nullptr;
    CopyJob *a_jobs = nullptr;
    uint32_t table_cap = 0;
};

struct Group {
    int db;
    uint32_t first, count;             // requests [first, first+count) of the launch
    uint64_t dq_off, da_off, dl_off;   // device batch buffers and limb workspace (offsets in the launch region)
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
    bool gemm = false;              // carries a batch of 3 or more (tensor-core GEMM)
    bool drop_completion = false;   // test hook: the completion is not reported to requests
};

// Block (x, j) copies part of job j (queries: pinned host -> device batch
// buffer; answers: device -> pinned host).
__global__ void copy_jobs_kernel(const CopyJob *jobs) {
    const CopyJob J = jobs[blockIdx.y];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += (uint64_t)gridDim.x * blockDim.x)
        J.dst[i] = J.src[i];
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
    uint64_t n_launches = 0, n_done = 0, n_failed = 0, n_busy = 0, n_grouped = 0;
    uint32_t active_gemm = 0;    // launches in flight that carry a GEMM
    double busy_batch_sum = 0;
    double enqueue_s = 0;   // host time spent enqueueing launches
    uint64_t stream_kernels = 0, gemm_kernels = 0;   // Response kernels enqueued, by kind

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
    if (L->gemm) --active_gemm;
    slots[L->slot].busy = nullptr;
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

namespace {
constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }
constexpr size_t kMaxGemmLaunches = 2;   // launches in flight at once while a GEMM is among them

// Device workspace of one group of `take` requests: queries, answers and the byte limbs of the
// queries (any group can join a grouped GEMM).
uint64_t group_bytes(const DbEntry &e, uint32_t take) {
    return align256(4ull * take * e.C) + align256(4ull * take * e.R) + align256(8ull * take * e.pitch);
}
}  // namespace

bool qpadl_server::form_launch(int si, std::unique_lock<std::mutex> &lk) {
    // databases with queued requests join this cycle with up to max_batch of them each
    std::vector<Group> groups;
    uint64_t need = 0;
    uint32_t total = 0;
    const uint64_t cap_bytes = dev_alloc.size();
    // the database holding the oldest queued request leads the launch; other
    // databases join only if their scan costs about the same (within
    // group_size_ratio), so no request waits on a much larger scan
    int lead = -1;
    for (int d = 0; d < static_cast<int>(dbs.size()); ++d)
        if (!dbs[d].queue.empty() &&
            (lead < 0 || dbs[d].queue.front()->t_submit < dbs[lead].queue.front()->t_submit))
            lead = d;
    if (lead < 0) return false;
    const double lead_size = static_cast<double>(dbs[lead].R) * static_cast<double>(dbs[lead].C);
    std::vector<int> order{lead};
    for (int d = 0; d < static_cast<int>(dbs.size()); ++d) {
        if (d == lead || dbs[d].queue.empty() || cfg.group_size_ratio < 1.0) continue;
        const double sz = static_cast<double>(dbs[d].R) * static_cast<double>(dbs[d].C);
        if (sz <= lead_size * cfg.group_size_ratio && sz * cfg.group_size_ratio >= lead_size) order.push_back(d);
    }
    for (int d : order) {
        DbEntry &e = dbs[d];
        uint32_t take = static_cast<uint32_t>(std::min<size_t>(e.queue.size(), cfg.max_batch));
        take = std::min(take, slots[si].table_cap - total);
        // shrink the batch until its workspace fits in what the arena can ever hold
        while (take > 0 && need + group_bytes(e, take) > cap_bytes) take = take > 3 ? take / 2 : take - 1;
        if (take == 0) break;
        Group g{d, total, take, 0, 0, 0};
        g.dq_off = need;
        need += align256(4ull * take * e.C);
        g.da_off = need;
        need += align256(4ull * take * e.R);
        g.dl_off = need;
        need += align256(8ull * take * e.pitch);
        total += take;
        groups.push_back(g);
    }
    if (groups.empty()) return false;
    // A launch over several databases, or with 3 or more queries, runs a tensor-core GEMM whose
    // grid fills every SM.  While one runs, at most kMaxGemmLaunches launches of any kind are in
    // flight: more would only split the SMs and shrink each batch.  With no GEMM in flight, a
    // lone database's one- and two-query streaming launches may take every free stream, so a
    // lone query does not queue behind another.
    const bool lone = groups.size() == 1;
    bool gemm = !lone;
    for (const Group &g : groups) gemm = gemm || g.count >= 3;
    if ((gemm || active_gemm > 0) && active.size() >= kMaxGemmLaunches) return false;
    uint64_t off = 0;
    if (!dev_alloc.alloc(need, &off)) return false;   // wait for a launch to free device memory
    Launch *L = new Launch();
    L->srv = this;
    L->slot = si;
    L->id = next_launch++;
    L->dev_off = off;
    L->dev_bytes = need;
    L->groups = groups;
    L->gemm = gemm;
    if (gemm) ++active_gemm;
    for (const Group &g : groups) {
        DbEntry &e = dbs[g.db];
        for (uint32_t i = 0; i < g.count; ++i) {
            L->reqs.push_back(e.queue.front());
            e.queue.pop_front();
        }
    }
    queued -= total;
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
    if (groups.size() > 1) ++n_grouped;
    busy_batch_sum += static_cast<double>(total);
    // enqueue the GPU work without holding the lock
    lk.unlock();
    const double t_enq0 = now_s();
    uint8_t *base = dev_arena + off;
    uint64_t maxC = 0, maxR = 0;
    for (const Group &g : groups) {
        const DbEntry &e = dbs[g.db];
        maxC = std::max(maxC, e.C);
        maxR = std::max(maxR, e.R);
        for (uint32_t i = 0; i < g.count; ++i) {
            Request *r = L->reqs[g.first + i];
            S.q_jobs[g.first + i] = CopyJob{r->q, reinterpret_cast<uint32_t *>(base + g.dq_off) + i * e.C, e.C};
            S.a_jobs[g.first + i] = CopyJob{reinterpret_cast<uint32_t *>(base + g.da_off) + i * e.R, r->a, e.R};
        }
    }
    bool ok = true;
    uint64_t n_stream_k = 0, n_gemm_k = 0;   // Response kernels this launch enqueues
    const unsigned gx = static_cast<unsigned>(std::min<uint64_t>((maxC + 1023) / 1024, 32));
    copy_jobs_kernel<<<dim3(gx, total), 256, 0, S.stream>>>(S.q_jobs);
    ok = ok && cudaGetLastError() == cudaSuccess;
    // Response kernels.  A lone database with 1 or 2 queries takes the streaming kernel (one
    // pass, lowest latency).  Otherwise every database whose queries the uint8-digit GEMM takes
    // (up to its QPADL_OPT_U8_MAX_BATCH) joins one grouped GEMM launch (up to kMaxGemmGroups
    // databases per launch), however uneven their counts; a database with more queries than
    // that takes the fp16-copy GEMM.
    std::vector<const Group *> small;
    for (const Group &g : groups) {
        const DbEntry &e = dbs[g.db];
        uint32_t *dq = reinterpret_cast<uint32_t *>(base + g.dq_off);
        uint32_t *da = reinterpret_cast<uint32_t *>(base + g.da_off);
        __half *dl = reinterpret_cast<__half *>(base + g.dl_off);
        if (lone && g.count == 1) {
            ok = ok && qpadl::db_answer_one_noscratch(e.db, dq, da, S.stream) == QPADL_OK;
            ++n_stream_k;
        } else if (lone && g.count == 2) {
            // both queries in one pass over the database
            ok = ok && qpadl::db_answer_two_noscratch(e.db, dq, e.C, da, e.R, S.stream) == QPADL_OK;
            ++n_stream_k;
        } else if (g.count <= e.u8_max) {
            // the limbs, and zeroed answers for the tiles the GEMM splits between CTAs
            ok = ok && qpadl::launch_vec_limbs(dq, e.C, g.count, e.C, dl, e.pitch, qpadl::db_num_sms(e.db),
                                               S.stream, da, (uint64_t)g.count * e.R) == cudaSuccess;
            small.push_back(&g);
        } else {
            ok = ok && qpadl::db_answer_f16_ws(e.db, dq, g.count, da, dl, S.stream) == QPADL_OK;
            ++n_gemm_k;
        }
    }
    for (size_t k0 = 0; k0 < small.size() && ok; k0 += qpadl::kMaxGemmGroups) {
        const size_t k1 = std::min(small.size(), k0 + qpadl::kMaxGemmGroups);
        uint32_t maxb = 0;
        for (size_t k = k0; k < k1; ++k) maxb = std::max(maxb, small[k]->count);
        // one tile width for the launch; a larger group takes several tiles of it
        const int bn = std::min(qpadl::limb_gemm_bn_for(maxb), 128);
        const int ks = qpadl::limb_gemm_u8_default_ks(bn);
        // one launch takes one form: the pair form when every database in it allows it
        bool pair = qpadl::limb_gemm_u8_pair_ok(bn, ks);
        for (size_t k = k0; k < k1; ++k) pair = pair && qpadl::db_pair_gemm(dbs[small[k]->db].db);
        qpadl::GroupedGemmArgs args;
        std::memset(&args, 0, sizeof(args));
        uint32_t units = 0;
        for (size_t k = k0; k < k1 && ok; ++k) {
            const Group &g = *small[k];
            const DbEntry &e = dbs[g.db];
            uint32_t u = 0;
            ok = qpadl::db_fill_u8_group(e.db, args, static_cast<int>(k - k0),
                                         reinterpret_cast<const __half *>(base + g.dl_off), g.count,
                                         reinterpret_cast<uint32_t *>(base + g.da_off), bn, ks, units, &u,
                                         pair) == QPADL_OK;
            units += u;
        }
        args.ngroups = static_cast<uint32_t>(k1 - k0);
        args.total_units = units;
        // a programmatic dependent of the kernel before it: every earlier kernel (the limb
        // kernels of this launch's groups among them) has completed when it starts, and it waits
        // for that kernel before its limb loads and output stores
        ok = ok && qpadl::launch_limb_gemm_u8(bn, ks, args, qpadl::db_num_sms(dbs[small[k0]->db].db),
                                              qpadl::db_status_word(dbs[small[k0]->db].db), S.stream, pair,
                                              true) == cudaSuccess;
        ++n_gemm_k;
    }
    if (ok) {
        const unsigned gy = static_cast<unsigned>(std::min<uint64_t>((maxR + 1023) / 1024, 32));
        copy_jobs_kernel<<<dim3(gy, total), 256, 0, S.stream>>>(S.a_jobs);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (!ok) {
        lk.lock();
        for (Request *r : L->reqs) {
            r->state = kFailed;
            r->error = QPADL_ECUDA;
        }
        n_failed += total;
        L->failed_by_watchdog = true;   // completion must not overwrite the failure
        lk.unlock();
    }
    // the callback runs after every kernel above and releases the stream and the workspace
    if (cudaLaunchHostFunc(S.stream, on_launch_done, L) != cudaSuccess) {
        cudaStreamSynchronize(S.stream);
        complete(L);
    }
    const double t_enq = now_s() - t_enq0;
    lk.lock();
    enqueue_s += t_enq;
    stream_kernels += n_stream_k;
    gemm_kernels += n_gemm_k;
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
        cfg->host_budget_bytes < 4096 || cfg->device_budget_bytes < 4096 || cfg->max_batch > 65535 ||
        !(cfg->group_size_ratio >= 0.0))   // also rejects NaN
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
    // one cycle takes at most max_batch requests of each database; 65535 is the grid's y limit
    const uint32_t cap = std::min<uint32_t>(std::min<uint32_t>(cfg->max_inflight, 65535u), 65535u);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.q_jobs), cap * sizeof(CopyJob), cudaHostAllocMapped) !=
                cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.a_jobs), cap * sizeof(CopyJob), cudaHostAllocMapped) !=
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
    // build the operand copies the launches read now, so launches never allocate
    int64_t u8_max = 0;
    if (qpadl_pir_get_option(db, QPADL_OPT_U8_MAX_BATCH, &u8_max) != QPADL_OK) return QPADL_EINVAL;
    if (qpadl::db_prepare_u8(db, nullptr) != QPADL_OK) return QPADL_ENOMEM;
    if (s->cfg.max_batch > static_cast<uint64_t>(u8_max) && qpadl::db_prepare_f16(db, nullptr) != QPADL_OK)
        return QPADL_ENOMEM;
    if (cudaDeviceSynchronize() != cudaSuccess) return QPADL_ECUDA;
    DbEntry e;
    e.db = db;
    e.R = R;
    e.C = C;
    e.pitch = qpadl::db_limb_pitch(db);
    e.u8_max = static_cast<uint32_t>(std::min<int64_t>(u8_max, 1ll << 30));
    if (group_bytes(e, 1) > s->dev_alloc.size()) return QPADL_ENOMEM;   // not even one request fits
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
    if (db_id < 0 || db_id >= static_cast<int>(s->dbs.size())) return QPADL_EINVAL;
    const uint64_t C = s->dbs[db_id].C, R = s->dbs[db_id].R;
    if (s->inflight >= s->cfg.max_inflight) {
        ++s->n_busy;
        return QPADL_EBUSY;
    }
    const uint64_t bytes = 4ull * (C + R) + 256;
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
    r->a = reinterpret_cast<uint32_t *>(s->host_arena + off + ((4ull * C + 255) & ~255ull));
    r->t_submit = now_s();
    s->reqs[r->ticket] = r;
    ++s->inflight;
    lk.unlock();
    std::memcpy(r->q, q_host, 4ull * C);   // outside the lock; the request is not queued yet
    lk.lock();
    s->dbs[db_id].queue.push_back(r);   // re-indexed: add_db may have grown the table meanwhile
    ++s->queued;
    *ticket = r->ticket;
    s->cv.notify_all();
    return QPADL_OK;
}

int qpadl_server_poll(qpadl_server *s, uint64_t ticket, uint32_t *ans_host, qpadl_request_times *times) {
    if (!s) return QPADL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
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
    s->reqs.erase(it);
    --s->inflight;
    if (r->state == kDone) {
        // the GPU is done with this request and no one else can reach it:
        // copy the answer out without holding the lock
        if (ans_host) {
            const uint64_t R = s->dbs[r->db].R;
            lk.unlock();
            std::memcpy(ans_host, r->a, 4ull * R);
            lk.lock();
        }
        s->host_alloc.release(r->host_off, r->host_bytes);
        delete r;
        return rc;
    }
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
    st->grouped_launches = s->n_grouped;
    st->mean_enqueue_us = s->n_launches ? 1e6 * s->enqueue_s / static_cast<double>(s->n_launches) : 0.0;
    st->stream_kernels = s->stream_kernels;
    st->gemm_kernels = s->gemm_kernels;
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
        if (sl.q_jobs) cudaFreeHost(sl.q_jobs);
        if (sl.a_jobs) cudaFreeHost(sl.a_jobs);
    }
    if (s->dev_arena) cudaFree(s->dev_arena);
    if (s->host_arena) cudaFreeHost(s->host_arena);
    delete s;
    return QPADL_OK;
}

// Open-loop load generator: request i is submitted at t0 + arrival_s[i]
// (arrival_s non-decreasing; retried while admission refuses) and its latency
// is its completion time minus that scheduled arrival.  Up to four client
// threads share the requests round-robin; each submits its own requests when
// they fall due (sleeping through long gaps, spinning over short ones) and
// polls the ones it has outstanding.
int qpadl_server_replay(qpadl_server *s, uint64_t n, const double *arrival_s, const int32_t *db_ids,
                        const uint32_t *const *q_host, uint32_t *const *ans_host, double *latency_s,
                        int32_t *status, qpadl_request_times *times) {
    if (!s || !arrival_s || !db_ids || !q_host || !latency_s || !status) return QPADL_EINVAL;
    for (uint64_t i = 1; i < n; ++i)
        if (arrival_s[i] < arrival_s[i - 1]) return QPADL_EINVAL;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const uint64_t T = std::max<uint64_t>(1, std::min<uint64_t>({n, 4, hw / 4 ? hw / 4 : 1}));
    const double t0 = now_s() + 1e-3;
    auto client = [&](uint64_t first) {
        struct Out {
            uint64_t i, ticket;
        };
        std::vector<Out> out;
        uint64_t next = first;
        double last_poll = 0.0;
        while (next < n || !out.empty()) {
            bool progress = false;
            const double t = now_s();
            while (next < n && t >= t0 + arrival_s[next]) {
                uint64_t tk = 0;
                const int rc = qpadl_server_submit(s, db_ids[next], q_host[next], &tk);
                if (rc == QPADL_EBUSY) break;   // admission refused: retry on the next pass
                if (rc != QPADL_OK) {
                    status[next] = rc;
                    latency_s[next] = -1;
                } else {
                    out.push_back(Out{next, tk});
                }
                next += T;
                progress = true;
            }
            // poll at most every 20 us: spinning pollers would otherwise crowd the server's lock
            const double tp = now_s();
            const bool poll_now = tp - last_poll >= 20e-6 || next >= n;
            if (poll_now) last_poll = tp;
            for (size_t k = 0; poll_now && k < out.size();) {
                qpadl_request_times tm;
                const uint64_t i = out[k].i;
                const int rc = qpadl_server_poll(s, out[k].ticket, ans_host ? ans_host[i] : nullptr, &tm);
                if (rc == QPADL_EAGAIN) {
                    ++k;
                    continue;
                }
                status[i] = rc;
                latency_s[i] = (rc == QPADL_OK) ? tm.done_s - (t0 + arrival_s[i]) : -1;
                if (times) {
                    // relative to the scheduled arrival of request i
                    times[i].submit_s = tm.submit_s - (t0 + arrival_s[i]);
                    times[i].launch_s = tm.launch_s - (t0 + arrival_s[i]);
                    times[i].done_s = tm.done_s - (t0 + arrival_s[i]);
                }
                out[k] = out.back();
                out.pop_back();
                progress = true;
            }
            if (!progress) {
                // sleep through long gaps (waking 100 us early) and spin over the last stretch,
                // so submissions leave on schedule despite the OS timer slack
                const double gap = next < n ? t0 + arrival_s[next] - now_s() : 1e-3;
                if (gap > 2e-4)
                    std::this_thread::sleep_for(std::chrono::duration<double>(std::min(gap - 1e-4, 1e-3)));
                else
                    std::this_thread::yield();
            }
        }
    };
    std::vector<std::thread> threads;
    for (uint64_t k = 1; k < T; ++k) threads.emplace_back(client, k);
    client(0);
    for (auto &th : threads) th.join();
    return QPADL_OK;
}

}  // extern "C"
