// Serving engine: a request loop over the join library.
//
// Requests arrive on any host thread (jn_server_submit) and wait in one
// queue.  `slots` worker threads, each with its own context and CUDA stream,
// take requests as soon as they free up, so the work of several requests
// overlaps on the device (continuous batching: a request that arrives while
// others run is admitted as soon as a slot and memory allow, not after the
// current group ends).  A worker that finds small requests at the head of the
// queue takes up to max_batch of them and runs them as one jn_batch (one
// launch sequence for the group); a large request runs alone.  The first
// small_slots workers take small requests only, so a small request has a
// lane where it never waits behind a large join.  Admission is
// by device memory: a request reserves its scratch estimate, and the join's
// own exact count pass, through the context's admission hook, reserves the
// exact output bytes before the output is allocated.  A run that does not fit
// next to the outputs still held frees its scratch, waits until output and
// scratch fit together, and runs again; a request that can never fit is
// refused with JN_ERR_OOM.  Tables registered with the
// server stay resident on the device across requests.
//
// The engine only calls the public entry points of jn.h; it adds no join
// arithmetic of its own.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "jn_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct OutBuf {  // one output allocation, shared by the requests of a batch
    jn_pair* ptr = nullptr;
    uint64_t bytes = 0;
    int refs = 0;
};

struct Job {
    uint64_t ticket = 0;
    jn_request req{};
    Clock::time_point submitted, started, finished;
    bool done = false;
    bool collected = false;  // its result was returned by a wait
    jn_status status = JN_OK;
    uint64_t pairs = 0;
    jn_pair* out = nullptr;
    std::shared_ptr<OutBuf> buf;
    std::string err;
};

struct Resident {
    jn_table t{};
    std::vector<void*> owned;
    uint64_t bytes = 0;
};

}  // namespace

struct jn_server {
    int device = 0;
    jn_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::map<int32_t, Resident> tables;
    int32_t next_handle = 1;
    uint64_t next_ticket = 1;
    uint64_t mem_held = 0;  // bytes of outputs not yet released + scratch reserved by running requests
    int running = 0;        // requests holding a reservation (their end frees their scratch)
    uint64_t queued_small = 0;  // queued requests below coalesce_rows
    std::deque<uint64_t> done_order;  // tickets in completion order, for jn_server_wait_any
    bool stop = false;
    std::vector<std::thread> workers;
    jn_server_stats stats{};
};

namespace {

uint64_t rows_of(const jn_request& r) { return (uint64_t)r.R.n + (uint64_t)r.S.n; }

// Device bytes a request needs besides its output: the partitioned copies
// and bookkeeping of the radix passes (two passes, rows of 8 or 16 bytes).
uint64_t scratch_estimate(const jn_request& r) {
    const uint64_t row = r.R.key_type == JN_KEY_I64 ? 16 : 8;
    return 3 * row * rows_of(r) + (16ull << 20);
}

jn_status resolve(jn_server* s, const jn_request& in, jn_request* out) {
    *out = in;
    std::lock_guard<std::mutex> g(s->mu);
    if (in.r_handle > 0) {
        auto it = s->tables.find(in.r_handle);
        if (it == s->tables.end()) return JN_ERR_INVALID;
        out->R = it->second.t;
    }
    if (in.s_handle > 0) {
        auto it = s->tables.find(in.s_handle);
        if (it == s->tables.end()) return JN_ERR_INVALID;
        out->S = it->second.t;
    }
    return JN_OK;
}

void finish(jn_server* s, const std::shared_ptr<Job>& j, jn_status st, uint64_t pairs, jn_pair* out,
            const std::shared_ptr<OutBuf>& buf, const char* err) {
    if (st == JN_OK && pairs > 0 && !jnx::is_device_pointer(out)) {
        st = JN_ERR_CUDA;  // never hand out a pointer the device does not own
        err = "result pointer is not device memory";
    }
    std::lock_guard<std::mutex> g(s->mu);
    j->finished = Clock::now();
    j->status = st;
    j->pairs = pairs;
    j->out = out;
    j->buf = buf;
    if (err) j->err = err;
    j->done = true;
    s->done_order.push_back(j->ticket);
    s->stats.completed++;
    if (st != JN_OK) s->stats.failed++;
    s->cv_done.notify_all();
}

// Reserves `bytes` of the budget for a run (false: refused).  While another
// request runs it waits for it (its end frees scratch).  With nothing
// running, only the client can free memory, by releasing results it holds:
// the request waits at most hold_wait_ms (summed over such stretches) and is
// then refused, since that release may itself wait on this request.
bool reserve(jn_server* s, uint64_t bytes) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (bytes > s->cfg.memory_budget) return false;
    auto fits = [&] { return s->stop || s->mem_held + bytes <= s->cfg.memory_budget; };
    auto idle_left = std::chrono::milliseconds(s->cfg.hold_wait_ms);
    while (!fits()) {
        if (s->running > 0) {
            s->cv_mem.wait(lk);
            continue;
        }
        if (idle_left.count() <= 0) break;
        const auto t0 = Clock::now();
        s->cv_mem.wait_for(lk, idle_left);
        idle_left -= std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0) +
                     std::chrono::milliseconds(1);
    }
    if (s->stop || s->mem_held + bytes > s->cfg.memory_budget) return false;
    s->mem_held += bytes;
    s->running++;
    if (s->mem_held > s->stats.peak_bytes) s->stats.peak_bytes = s->mem_held;
    return true;
}

// Ends a run's reservation, returning `bytes` to the budget.
void unreserve(jn_server* s, uint64_t bytes) {
    std::lock_guard<std::mutex> g(s->mu);
    s->mem_held -= bytes;
    s->running--;
    s->cv_mem.notify_all();
}

// Admission state of one worker, read by its context's admission hook.  The
// join calls the hook once its exact count is known and before it allocates
// the output, so a request is admitted by its exact output bytes without a
// count pass of its own.
struct Admit {
    jn_server* s = nullptr;
    jn_ctx* ctx = nullptr;  // the worker's context (its launch counter)
    uint64_t granted = 0;  // output bytes the hook reserved for the current run
    uint64_t prepaid = 0;  // output bytes reserved before a second run
    uint64_t wanted = 0;   // output bytes the last hook call asked for
    bool asked = false;
    bool never = false;    // output plus scratch exceed the whole budget
    void reset() {
        granted = prepaid = wanted = 0;
        asked = never = false;
    }
};

jn_status admit_hook(void* user, uint64_t out_bytes, uint64_t scratch_bytes) {
    Admit* a = static_cast<Admit*>(user);
    jn_server* s = a->s;
    std::lock_guard<std::mutex> g(s->mu);
    a->asked = true;
    a->wanted = out_bytes;
    if (a->prepaid >= out_bytes) {  // a second run, its bytes already reserved
        a->granted = a->prepaid;
        a->prepaid = 0;
        return JN_OK;
    }
    if (out_bytes + scratch_bytes > s->cfg.memory_budget) {
        a->never = true;
        return JN_ERR_OOM;
    }
    if (s->mem_held + out_bytes > s->cfg.memory_budget) return JN_ERR_OOM;  // not now
    s->mem_held += out_bytes;
    if (s->mem_held > s->stats.peak_bytes) s->stats.peak_bytes = s->mem_held;
    a->granted = out_bytes;
    return JN_OK;
}

// Runs `call` under admission: scratch is reserved first (its estimate); a
// run the hook turned away for lack of memory frees its scratch, waits until
// output and scratch fit together, and runs once more with the output bytes
// reserved in advance.  Returns the status; a->granted holds the reserved
// output bytes of a successful run.
template <typename Call>
jn_status admitted_run(jn_server* s, Admit* a, cudaStream_t stream, uint64_t scratch, Call call) {
    const uint64_t l0 = a->ctx ? jn_launch_count(a->ctx) : 0;
    struct Count {  // kernels of this run (and of a second one) go to the server's stats
        jn_server* s;
        Admit* a;
        uint64_t l0;
        ~Count() {
            if (!a->ctx) return;
            const uint64_t n = jn_launch_count(a->ctx) - l0;
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.kernel_launches += n;
        }
    } count{s, a, l0};
    a->reset();
    if (!reserve(s, scratch)) return JN_ERR_OOM;
    jn_status st = call();
    if (st == JN_ERR_OOM && a->asked && !a->never && a->granted == 0) {
        unreserve(s, scratch);
        const uint64_t need = a->wanted;
        a->reset();
        if (!reserve(s, need + scratch)) return JN_ERR_OOM;
        a->prepaid = need;
        st = call();
    }
    if (st == JN_OK && cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        st = JN_ERR_CUDA;
    }
    unreserve(s, scratch + (st == JN_OK ? 0 : a->granted) + a->prepaid);
    if (st != JN_OK) a->granted = 0;
    a->prepaid = 0;
    return st;
}

void run_single(jn_server* s, jn_ctx* ctx, Admit* a, cudaStream_t stream, const std::shared_ptr<Job>& j) {
    jn_request r;
    if (resolve(s, j->req, &r) != JN_OK) {
        finish(s, j, JN_ERR_INVALID, 0, nullptr, nullptr, "unknown table handle");
        return;
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        j->started = Clock::now();
    }
    jn_pair* out = nullptr;
    uint64_t n = 0;
    const jn_status st = admitted_run(s, a, stream, scratch_estimate(r), [&] {
        out = nullptr;
        n = 0;
        return r.band >= 0 ? jn_theta(ctx, &r.R, &r.S, r.op, r.band, &out, 0, &n)
                           : jn_hash(ctx, &r.R, &r.S, &out, 0, &n);
    });
    if (st != JN_OK) {
        finish(s, j, st, st == JN_ERR_OOM ? n : 0, nullptr, nullptr,
               st == JN_ERR_OOM ? "request does not fit the memory budget" : jn_last_error(ctx));
        return;
    }
    auto buf = std::make_shared<OutBuf>();
    buf->ptr = out;
    buf->bytes = a->granted;
    buf->refs = 1;
    finish(s, j, JN_OK, n, out, buf, nullptr);
}

void run_group(jn_server* s, jn_ctx* ctx, Admit* a, cudaStream_t stream, std::vector<std::shared_ptr<Job>>& g) {
    std::vector<jn_join> joins;
    std::vector<std::shared_ptr<Job>> live;
    uint64_t scratch = 0;
    for (auto& j : g) {
        jn_request r;
        if (resolve(s, j->req, &r) != JN_OK) {
            finish(s, j, JN_ERR_INVALID, 0, nullptr, nullptr, "unknown table handle");
            continue;
        }
        jn_join x;
        memset(&x, 0, sizeof(x));
        x.R = r.R;
        x.S = r.S;
        x.op = r.op;
        x.band = r.band;
        joins.push_back(x);
        live.push_back(j);
        scratch += scratch_estimate(r);
    }
    if (live.empty()) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = Clock::now();
        for (auto& j : live) j->started = now;
        s->stats.batches++;
    }
    std::vector<uint64_t> first(live.size()), cnt(live.size());
    jn_pair* out = nullptr;
    uint64_t total = 0;
    const jn_status st = admitted_run(s, a, stream, scratch, [&] {
        out = nullptr;
        total = 0;
        return jn_batch(ctx, (int32_t)joins.size(), joins.data(), &out, 0, &total, first.data(), cnt.data());
    });
    if (st != JN_OK) {
        for (auto& j : live)
            finish(s, j, st, 0, nullptr, nullptr,
                   st == JN_ERR_OOM ? "batch does not fit the memory budget" : jn_last_error(ctx));
        return;
    }
    // outputs of a group are one allocation: accounted for until all are released
    auto buf = std::make_shared<OutBuf>();
    buf->ptr = out;
    buf->bytes = a->granted;
    buf->refs = (int)live.size();
    for (size_t i = 0; i < live.size(); i++) finish(s, live[i], JN_OK, cnt[i], out ? out + first[i] : nullptr, buf, nullptr);
}

void worker_main(jn_server* s, int slot) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    if (slot < s->cfg.small_slots) {
        // the small-request lane's stream has the highest priority: its
        // blocks go first as SMs free up, ahead of the large joins' kernels
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        cudaStreamCreateWithPriority(&stream, cudaStreamNonBlocking, greatest);
    } else {
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    }
    jn_ctx* ctx = nullptr;
    if (jn_create(&ctx, s->device, stream) != JN_OK) {
        cudaStreamDestroy(stream);
        return;
    }
    jn_tuning t;
    jn_get_tuning(ctx, &t);
    t.graphs = s->cfg.graphs ? 1 : 0;
    if (slot >= s->cfg.small_slots && s->cfg.small_slots > 0 && s->cfg.small_sms > 0) {
        // the large-request workers' persistent grids leave small_sms SMs'
        // worth of room, where the small lane's kernels start at once
        // instead of waiting for a whole large kernel to end
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        t.sms = sms > s->cfg.small_sms ? sms - s->cfg.small_sms : 1;
    }
    jn_set_tuning(ctx, &t);
    Admit adm;
    adm.s = s;
    adm.ctx = ctx;
    jn_set_admission(ctx, admit_hook, &adm);
    // the first small_slots workers form the small-request lane: they take
    // only requests below coalesce_rows, so those never queue behind a large
    // join; the other workers take the queue in order
    const bool small_lane = slot < s->cfg.small_slots;
    const uint64_t small_rows = (uint64_t)s->cfg.coalesce_rows;
    while (true) {
        std::vector<std::shared_ptr<Job>> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || (small_lane ? s->queued_small > 0 : !s->queue.empty()); });
            if (s->stop && s->queue.empty()) break;
            if (s->stop && small_lane && s->queued_small == 0) break;
            auto hit = s->queue.begin();
            if (small_lane)
                while (rows_of((*hit)->req) >= small_rows) ++hit;  // queued_small > 0: one exists
            auto head = *hit;
            s->queue.erase(hit);
            take.push_back(head);
            if (rows_of(head->req) < small_rows) {
                s->queued_small--;
                // coalesce the small requests waiting now
                for (auto it = s->queue.begin(); it != s->queue.end() && (int)take.size() < s->cfg.max_batch;) {
                    if (rows_of((*it)->req) < small_rows && (*it)->req.R.key_type == head->req.R.key_type) {
                        take.push_back(*it);
                        it = s->queue.erase(it);
                        s->queued_small--;
                    } else {
                        ++it;
                    }
                }
            }
        }
        if (take.size() == 1 && rows_of(take[0]->req) >= (uint64_t)s->cfg.coalesce_rows)
            run_single(s, ctx, &adm, stream, take[0]);
        else
            run_group(s, ctx, &adm, stream, take);
    }
    jn_destroy(ctx);
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

jn_status jn_server_create(jn_server** out, int device, const jn_server_config* cfg) {
    if (!out || !cfg || cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch < 1 || cfg->small_slots < 0 ||
        cfg->small_slots >= cfg->slots || cfg->hold_wait_ms < 0 || cfg->small_sms < 0 || cfg->reserved != 0)
        return JN_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return JN_ERR_INVALID;
    }
    jn_server* s = new jn_server();
    s->device = device;
    s->cfg = *cfg;
    for (int i = 0; i < cfg->slots; i++) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return JN_OK;
}

void jn_server_destroy(jn_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
    for (auto& t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->jobs)
        if (kv.second->buf && kv.second->buf->ptr && --kv.second->buf->refs == 0) cudaFree(kv.second->buf->ptr);
    for (auto& kv : s->tables)
        for (void* p : kv.second.owned) cudaFree(p);
    delete s;
}

jn_status jn_server_register(jn_server* s, const jn_table* t, int32_t* handle) {
    if (!s || !t || !handle || (t->key_type != JN_KEY_I32 && t->key_type != JN_KEY_I64) || t->n < 0 ||
        t->n > INT32_MAX || (t->n > 0 && !t->key))
        return JN_ERR_INVALID;
    cudaSetDevice(s->device);
    Resident r;
    r.t = *t;
    const size_t kb = (size_t)t->n * (size_t)t->key_type;
    auto copy = [&](const void* src, size_t bytes, const void** dst) -> jn_status {
        if (!src || bytes == 0) {
            *dst = src && bytes == 0 ? nullptr : *dst;
            return JN_OK;
        }
        void* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
            cudaGetLastError();
            return JN_ERR_OOM;
        }
        if (cudaMemcpy(d, src, bytes, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            return JN_ERR_CUDA;
        }
        r.owned.push_back(d);
        r.bytes += bytes;
        *dst = d;
        return JN_OK;
    };
    jn_status st = copy(t->key, kb, &r.t.key);
    if (st == JN_OK && t->key2) st = copy(t->key2, kb, &r.t.key2);
    if (st == JN_OK && t->payload) {
        const void* p = nullptr;
        st = copy(t->payload, (size_t)t->n * 4, &p);
        r.t.payload = static_cast<const int32_t*>(p);
    }
    if (st != JN_OK) {
        for (void* p : r.owned) cudaFree(p);
        return st;
    }
    std::lock_guard<std::mutex> g(s->mu);
    *handle = s->next_handle++;
    s->stats.resident_bytes += r.bytes;
    s->tables[*handle] = std::move(r);
    return JN_OK;
}

jn_status jn_server_unregister(jn_server* s, int32_t handle) {
    if (!s) return JN_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tables.find(handle);
    if (it == s->tables.end()) return JN_ERR_INVALID;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();  // requests already running may still read it
    for (void* p : it->second.owned) cudaFree(p);
    s->stats.resident_bytes -= it->second.bytes;
    s->tables.erase(it);
    return JN_OK;
}

jn_status jn_server_submit(jn_server* s, const jn_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || req->reserved != 0 || req->op < JN_EQ || req->op > JN_ANY ||
        (req->band < 0 && req->op != JN_EQ))
        return JN_ERR_INVALID;
    auto j = std::make_shared<Job>();
    j->req = *req;
    {
        std::lock_guard<std::mutex> g(s->mu);
        // resolve sizes of resident tables now, for coalescing decisions
        if (req->r_handle > 0) {
            auto it = s->tables.find(req->r_handle);
            if (it == s->tables.end()) return JN_ERR_INVALID;
            j->req.R.n = it->second.t.n;
            j->req.R.key_type = it->second.t.key_type;
        }
        if (req->s_handle > 0) {
            auto it = s->tables.find(req->s_handle);
            if (it == s->tables.end()) return JN_ERR_INVALID;
            j->req.S.n = it->second.t.n;
            j->req.S.key_type = it->second.t.key_type;
        }
        j->ticket = s->next_ticket++;
        j->submitted = Clock::now();
        s->jobs[j->ticket] = j;
        s->queue.push_back(j);
        if (rows_of(j->req) < (uint64_t)s->cfg.coalesce_rows) s->queued_small++;
        s->stats.submitted++;
        *ticket = j->ticket;
    }
    s->cv_work.notify_all();  // a small-lane worker may not take this request
    return JN_OK;
}

static void fill_result(Job& j, jn_result* res) {
    j.collected = true;
    memset(res, 0, sizeof(*res));
    res->status = j.status;
    res->pairs = j.pairs;
    res->out = j.out;
    using ms = std::chrono::duration<double, std::milli>;
    res->queue_ms = ms(j.started - j.submitted).count();
    res->run_ms = ms(j.finished - j.started).count();
    res->total_ms = ms(j.finished - j.submitted).count();
    if (j.started.time_since_epoch().count() == 0) res->queue_ms = res->run_ms = 0;
}

jn_status jn_server_wait(jn_server* s, uint64_t ticket, jn_result* res) {
    if (!s || !res) return JN_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return JN_ERR_INVALID;
    auto j = it->second;
    s->cv_done.wait(lk, [&] { return j->done; });
    fill_result(*j, res);
    return JN_OK;
}

jn_status jn_server_wait_any(jn_server* s, uint64_t* ticket, jn_result* res, int64_t timeout_ms) {
    if (!s || !ticket || !res) return JN_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    // the oldest completion whose result no wait has returned yet
    auto ready = [&]() -> std::shared_ptr<Job> {
        while (!s->done_order.empty()) {
            auto it = s->jobs.find(s->done_order.front());
            if (it != s->jobs.end() && !it->second->collected) return it->second;
            s->done_order.pop_front();  // released, or returned by jn_server_wait
        }
        return nullptr;
    };
    auto pending = [&] {  // requests whose result is still to be returned
        for (auto& kv : s->jobs)
            if (!kv.second->collected) return true;
        return false;
    };
    std::shared_ptr<Job> j = ready();
    if (!j) {
        if (!pending()) return JN_ERR_INVALID;  // nothing submitted is outstanding
        auto pred = [&] { return (j = ready()) != nullptr; };
        if (timeout_ms < 0)
            s->cv_done.wait(lk, pred);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
            return JN_ERR_TIMEOUT;
    }
    s->done_order.pop_front();
    *ticket = j->ticket;
    fill_result(*j, res);
    return JN_OK;
}

jn_status jn_server_release(jn_server* s, uint64_t ticket) {
    if (!s) return JN_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || !it->second->done) return JN_ERR_INVALID;
    auto buf = it->second->buf;
    s->jobs.erase(it);
    if (buf && --buf->refs == 0) {
        if (buf->ptr) {
            cudaSetDevice(s->device);
            jn_free(nullptr, buf->ptr);
        }
        s->mem_held -= buf->bytes;
        s->cv_mem.notify_all();
    }
    return JN_OK;
}

jn_status jn_server_stats_get(jn_server* s, jn_server_stats* out) {
    if (!s || !out) return JN_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->held_bytes = s->mem_held;
    out->queued = s->queue.size();
    return JN_OK;
}

}  // extern "C"
