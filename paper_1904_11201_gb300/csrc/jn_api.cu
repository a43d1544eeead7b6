// extern "C" entry points of libjn: argument checks, host-column staging,
// dispatch on key type, and the output convention of jn.h.
#include <string.h>

#include <vector>

#include "jn_algos.h"

namespace jnx {

// Admission by exact bytes: the count is known, nothing is allocated yet.
static jn_status admit(jn_ctx* c, uint64_t m, uint64_t out_bytes, OutPlan& plan) {
    if (c->mem_limit && out_bytes + c->scratch_bytes > c->mem_limit) {
        *plan.n_out = m;
        return fail(c, JN_ERR_OOM, "the exact result and the scratch held exceed the memory limit");
    }
    if (c->admit) {
        const jn_status st = c->admit(c->admit_user, out_bytes, c->scratch_bytes);
        if (st != JN_OK) {
            *plan.n_out = m;
            return fail(c, st, "the admission hook refused the run");
        }
    }
    return JN_OK;
}

jn_status out_prepare(jn_ctx* c, Scratch& s, uint64_t m, OutPlan& plan) {
    jn_pair* user = *plan.user_out;
    plan.host_copy = false;
    plan.lib_alloc = false;
    const jn_pair* mapped =
        user && (c->tune.host_io & 2) ? static_cast<const jn_pair*>(host_mapped(user)) : nullptr;
    {
        const bool dev_out =
            user != nullptr && (m == 0 || m > plan.capacity || mapped || is_device_pointer(user));
        JN_TRY(admit(c, m, dev_out ? 0 : m * sizeof(jn_pair), plan));
    }
    if (user == nullptr) {
        plan.lib_alloc = true;
        plan.dev = nullptr;
        if (m > 0) {
            void* p = nullptr;
            JN_TRY(dalloc(c, &p, m * sizeof(jn_pair)));
            plan.dev = static_cast<jn_pair*>(p);
        }
        return JN_OK;
    }
    if (m > plan.capacity) {
        *plan.n_out = m;
        return fail(c, JN_ERR_CAPACITY, "output buffer holds fewer pairs than the result");
    }
    // the kernels store a pair as one 8-byte word: a caller buffer off an
    // 8-byte boundary is filled by a copy from an aligned scratch buffer
    const bool aligned = ((uintptr_t)user & 7) == 0;
    if (m == 0 || (aligned && is_device_pointer(user))) {
        plan.dev = user;
        return JN_OK;
    }
    if (mapped && aligned) {  // page-locked host memory: the kernels write the pairs in place
        plan.dev = const_cast<jn_pair*>(mapped);
        plan.mapped = true;
        return JN_OK;
    }
    plan.host_copy = true;
    return s.get(&plan.dev, m);
}

jn_status out_finish(jn_ctx* c, uint64_t m, OutPlan& plan) {
    if (plan.mapped && m > 0) JN_CUDA(c, cudaStreamSynchronize(c->stream));  // pairs visible to the host
    if (plan.host_copy && m > 0) {
        if (!plan.copied)
            JN_CUDA(c, cudaMemcpyAsync(*plan.user_out, plan.dev, m * sizeof(jn_pair), cudaMemcpyDefault,
                                       c->stream));
        JN_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (plan.lib_alloc) *plan.user_out = plan.dev;
    *plan.n_out = m;
    return JN_OK;
}

static jn_status check_table(jn_ctx* c, const jn_table* t, const char* name, bool need_key2) {
    if (!t) return fail(c, JN_ERR_INVALID, std::string(name) + ": NULL table");
    if (t->key_type != JN_KEY_I32 && t->key_type != JN_KEY_I64)
        return fail(c, JN_ERR_INVALID, std::string(name) + ": key_type must be JN_KEY_I32 or JN_KEY_I64");
    if (t->n < 0 || t->n > INT32_MAX)
        return fail(c, JN_ERR_INVALID, std::string(name) + ": row count out of range");
    if (t->reserved != 0) return fail(c, JN_ERR_INVALID, std::string(name) + ": reserved must be 0");
    if (t->n > 0 && t->key == nullptr) return fail(c, JN_ERR_INVALID, std::string(name) + ": NULL key");
    if (need_key2 && t->n > 0 && t->key2 == nullptr)
        return fail(c, JN_ERR_INVALID, std::string(name) + ": key2 required");
    return JN_OK;
}

static bool valid_op(int op) { return op >= JN_EQ && op <= JN_ANY; }

// Host columns of one run: device scratch for each, filled on the copy
// stream (key columns first, then second columns and payloads), with one
// event when the keys have landed and one when everything has.
struct HostCopies {
    jn_ctx* c;
    struct Job {
        void* dst;
        const void* src;
        size_t bytes;
        bool key;
        bool first;  // a column of the first table staged
    };
    std::vector<Job> jobs;
    bool first_table = true;  // stage() calls of the first table come first
    explicit HostCopies(jn_ctx* ctx) : c(ctx) {}
    ~HostCopies() {
        // the run's stream-ordered frees of the scratch come after every copy
        if (c->copied_all) cudaStreamWaitEvent(c->stream, c->copied_all, 0);
        if (c->copied_keys) cudaEventDestroy(c->copied_keys);
        if (c->copied_r) cudaEventDestroy(c->copied_r);
        if (c->copied_all) cudaEventDestroy(c->copied_all);
        c->copied_keys = c->copied_r = c->copied_all = nullptr;
    }
    // a device column as it is, or scratch that a later copy fills
    jn_status column(Scratch& s, const void* p, size_t bytes, bool key, const void** dp) {
        if (p == nullptr || bytes == 0 || is_device_pointer(p)) {
            *dp = p;
            return JN_OK;
        }
        uint8_t* d = nullptr;
        JN_TRY(s.get(&d, bytes));
        jobs.push_back(Job{d, p, bytes, key, first_table});
        *dp = d;
        return JN_OK;
    }
    jn_status start() {
        if (jobs.empty()) return JN_OK;
        if (!c->copy_stream) JN_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        cudaEvent_t ready;  // the scratch allocations (stream-ordered on the run's stream) come first
        JN_CUDA(c, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        cudaEventRecord(ready, c->stream);
        cudaStreamWaitEvent(c->copy_stream, ready, 0);
        cudaEventDestroy(ready);
        JN_CUDA(c, cudaEventCreateWithFlags(&c->copied_keys, cudaEventDisableTiming));
        JN_CUDA(c, cudaEventCreateWithFlags(&c->copied_r, cudaEventDisableTiming));
        JN_CUDA(c, cudaEventCreateWithFlags(&c->copied_all, cudaEventDisableTiming));
        // keys of both tables, then the rest of the first table, then the rest
        cudaEvent_t marks[3] = {c->copied_keys, c->copied_r, c->copied_all};
        for (int pass = 0; pass < 3; pass++) {
            for (const Job& j : jobs)
                if (pass == 0 ? j.key : (!j.key && j.first == (pass == 1)))
                    JN_CUDA(c, cudaMemcpyAsync(j.dst, j.src, j.bytes, cudaMemcpyHostToDevice, c->copy_stream));
            JN_CUDA(c, cudaEventRecord(marks[pass], c->copy_stream));
        }
        return JN_OK;
    }
};

template <typename K>
static jn_status stage(jn_ctx* c, Scratch& s, HostCopies& hc, const jn_table* t, bool use_key2, Cols<K>* out,
                       bool in_place = false) {
    const size_t kb = (size_t)t->n * sizeof(K);
    const void *k = nullptr, *k2 = nullptr, *p = nullptr;
    // a path that reads each column in a couple of streaming passes reads
    // page-locked host columns in place instead of copying them first
    const void* mk = in_place ? host_mapped(t->key) : nullptr;
    const void* mp = in_place && t->payload ? host_mapped(t->payload) : nullptr;
    out->host = mk && (mp || !t->payload) && !(use_key2 && t->key2);
    if (out->host) {
        k = mk;
        p = mp;
    } else {
        JN_TRY(hc.column(s, t->key, kb, true, &k));
        if (use_key2 && t->key2) JN_TRY(hc.column(s, t->key2, kb, false, &k2));
        if (t->payload) JN_TRY(hc.column(s, t->payload, (size_t)t->n * 4, false, &p));
    }
    out->key = static_cast<const K*>(k);
    out->key2 = static_cast<const K*>(k2);
    out->pay = static_cast<const int32_t*>(p);
    out->n = t->n;
    return JN_OK;
}

template <typename K>
static jn_status dispatch(jn_ctx* c, int algo, const jn_table* R, const jn_table* S, const jn_pred& pr,
                          int mode, OutPlan* plan, RunResult* res) {
    Scratch s(c);
    HostCopies hc(c);
    Cols<K> r, q;
    const bool equi = algo == JN_ALGO_HASH || algo == JN_ALGO_SORT;
    const bool use2 = !equi;
    // the equi joins sample a column, then read it in two streaming passes
    const bool in_place = equi && (c->tune.host_io & 1);
    JN_TRY(stage<K>(c, s, hc, R, use2, &r, in_place));
    hc.first_table = false;
    JN_TRY(stage<K>(c, s, hc, S, use2, &q, in_place));
    JN_TRY(hc.start());
    if (!equi) JN_TRY(wait_copies(c, true));  // the equi joins wait per phase
    switch (algo) {
        case JN_ALGO_HASH: return run_hash<K>(c, r, q, mode, plan, res);
        case JN_ALGO_SORT: return run_hash<K>(c, r, q, mode, plan, res, true);
        case JN_ALGO_NLJ: return run_nlj<K>(c, r, q, pr, mode, plan, res);
        case JN_ALGO_THETA: return run_theta<K>(c, r, q, pr.op_a, pr.band, mode, plan, res);
    }
    return fail(c, JN_ERR_INVALID, "unknown algorithm");
}

static jn_status run(jn_ctx* c, int algo, const jn_table* R, const jn_table* S, const jn_pred* pred,
                     int mode, jn_pair** out, uint64_t capacity, uint64_t* n_out, uint64_t* count,
                     uint64_t* checksum) {
    if (!c) return JN_ERR_INVALID;
    c->err.clear();
    jn_pred pr;
    pr.op_a = JN_EQ;
    pr.op_k = JN_ANY;
    pr.band = -1;
    if (pred) pr = *pred;
    if (!valid_op(pr.op_a) || !valid_op(pr.op_k)) return fail(c, JN_ERR_INVALID, "unknown predicate op");
    if (algo == JN_ALGO_HASH || algo == JN_ALGO_SORT) {
        const bool second = pred && (pr.band >= 0 || pr.op_k != JN_ANY);
        if (pr.op_a != JN_EQ || second)
            return fail(c, JN_ERR_UNSUPPORTED, "the hash and sort-merge joins take the equality predicate only");
    }
    const bool need2 = algo == JN_ALGO_THETA && pr.band >= 0;
    JN_TRY(check_table(c, R, "R", need2));
    JN_TRY(check_table(c, S, "S", need2));
    if (R->key_type != S->key_type) return fail(c, JN_ERR_INVALID, "R and S key types differ");
    if (mode == MODE_EMIT && (!out || !n_out)) return fail(c, JN_ERR_INVALID, "NULL output pointer");
    if (mode != MODE_EMIT && !count) return fail(c, JN_ERR_INVALID, "NULL count pointer");
    JN_CUDA(c, cudaSetDevice(c->device));
    c->info = jn_run_info();
    const uint64_t l0 = c->launches_total;
    OutPlan plan;
    plan.user_out = out;
    plan.capacity = capacity;
    plan.n_out = n_out;
    RunResult res;
    jn_status st = (R->key_type == JN_KEY_I32)
                       ? dispatch<int32_t>(c, algo, R, S, pr, mode, &plan, &res)
                       : dispatch<int64_t>(c, algo, R, S, pr, mode, &plan, &res);
    c->info.kernel_launches = c->launches_total - l0;
    if (st != JN_OK) return st;
    if (count) *count = res.count;
    if (checksum) *checksum = res.checksum;
    return JN_OK;
}

template <typename K>
static jn_status batch_typed(jn_ctx* c, int count, const jn_join* joins, jn_pair** out, uint64_t capacity,
                             uint64_t* n_out, uint64_t* first, uint64_t* pairs, bool count_only) {
    Scratch s(c);
    std::vector<int> eq, bd;
    for (int i = 0; i < count; i++) (joins[i].band < 0 ? eq : bd).push_back(i);
    std::vector<Cols<K>> ER(eq.size()), ES(eq.size()), BR(bd.size()), BS(bd.size());
    std::vector<int> bops(bd.size());
    std::vector<int64_t> bbands(bd.size());
    HostCopies hc(c);
    for (size_t j = 0; j < eq.size(); j++) {
        JN_TRY(stage<K>(c, s, hc, &joins[eq[j]].R, false, &ER[j]));
        JN_TRY(stage<K>(c, s, hc, &joins[eq[j]].S, false, &ES[j]));
    }
    for (size_t j = 0; j < bd.size(); j++) {
        JN_TRY(stage<K>(c, s, hc, &joins[bd[j]].R, true, &BR[j]));
        JN_TRY(stage<K>(c, s, hc, &joins[bd[j]].S, true, &BS[j]));
        bops[j] = joins[bd[j]].op;
        bbands[j] = joins[bd[j]].band;
    }
    JN_TRY(hc.start());
    JN_TRY(wait_copies(c, true));
    // every join is counted before the single output allocation
    std::unique_ptr<BatchRun> he, be;
    if (!eq.empty()) JN_TRY(batch_hash_prepare<K>(c, (int)eq.size(), ER.data(), ES.data(), &he));
    if (!bd.empty())
        JN_TRY(batch_band_prepare<K>(c, (int)bd.size(), BR.data(), BS.data(), bops.data(), bbands.data(), &be));
    const uint64_t te = he ? he->total : 0, tb = be ? be->total : 0;
    if (count_only) {
        for (size_t j = 0; j < eq.size(); j++) pairs[eq[j]] = he->offsets[j + 1] - he->offsets[j];
        for (size_t j = 0; j < bd.size(); j++) pairs[bd[j]] = be->offsets[j + 1] - be->offsets[j];
        *n_out = te + tb;
        c->info.result = te + tb;
        return JN_OK;
    }
    OutPlan plan;
    plan.user_out = out;
    plan.capacity = capacity;
    plan.n_out = n_out;
    JN_TRY(out_prepare(c, s, te + tb, plan));
    if (plan.host_copy && !is_device_pointer(*out))
        return fail(c, JN_ERR_INVALID, "batch outputs must be device memory");
    if (he) JN_TRY(he->emit(c, plan.dev));
    if (be) JN_TRY(be->emit(c, plan.dev + te));
    for (size_t j = 0; j < eq.size(); j++) {
        first[eq[j]] = he->offsets[j];
        pairs[eq[j]] = he->offsets[j + 1] - he->offsets[j];
    }
    for (size_t j = 0; j < bd.size(); j++) {
        first[bd[j]] = te + be->offsets[j];
        pairs[bd[j]] = be->offsets[j + 1] - be->offsets[j];
    }
    JN_TRY(out_finish(c, te + tb, plan));
    uint64_t dummy;
    uint64_t* d_small;
    JN_TRY(s.get(&d_small, 1));
    JN_TRY(read_back(c, d_small, &dummy, 0));  // reports a device wait that ran out
    c->info.result = te + tb;
    return JN_OK;
}

}  // namespace jnx

using namespace jnx;

extern "C" {

jn_status jn_count(jn_ctx* ctx, int32_t algo, const jn_table* R, const jn_table* S, const jn_pred* pred,
                   uint64_t* count) {
    return run(ctx, algo, R, S, pred, MODE_COUNT, nullptr, 0, nullptr, count, nullptr);
}

jn_status jn_aggregate(jn_ctx* ctx, int32_t algo, const jn_table* R, const jn_table* S,
                       const jn_pred* pred, uint64_t* count, uint64_t* checksum) {
    return run(ctx, algo, R, S, pred, MODE_AGG, nullptr, 0, nullptr, count, checksum);
}

jn_status jn_nested_loop(jn_ctx* ctx, const jn_table* R, const jn_table* S, const jn_pred* pred,
                         jn_pair** out, uint64_t capacity, uint64_t* n_out) {
    return run(ctx, JN_ALGO_NLJ, R, S, pred, MODE_EMIT, out, capacity, n_out, nullptr, nullptr);
}

jn_status jn_hash(jn_ctx* ctx, const jn_table* R, const jn_table* S, jn_pair** out, uint64_t capacity,
                  uint64_t* n_out) {
    return run(ctx, JN_ALGO_HASH, R, S, nullptr, MODE_EMIT, out, capacity, n_out, nullptr, nullptr);
}

jn_status jn_sort_merge(jn_ctx* ctx, const jn_table* R, const jn_table* S, jn_pair** out, uint64_t capacity,
                        uint64_t* n_out) {
    return run(ctx, JN_ALGO_SORT, R, S, nullptr, MODE_EMIT, out, capacity, n_out, nullptr, nullptr);
}

static jn_status batch_entry(jn_ctx* ctx, int32_t count, const jn_join* joins, jn_pair** out, uint64_t capacity,
                             uint64_t* n_out, uint64_t* first, uint64_t* pairs, bool count_only) {
    if (!ctx) return JN_ERR_INVALID;
    ctx->err.clear();
    if (count < 0 || (count > 0 && (!joins || !first || !pairs)) || !out || !n_out)
        return fail(ctx, JN_ERR_INVALID, "jn_batch: bad arguments");
    if (count == 0) {
        *n_out = 0;
        return JN_OK;
    }
    const int32_t kt = joins[0].R.key_type;
    for (int i = 0; i < count; i++) {
        const jn_join& j = joins[i];
        const bool band = j.band >= 0;
        JN_TRY(check_table(ctx, &j.R, "R", band));
        JN_TRY(check_table(ctx, &j.S, "S", band));
        if (j.R.key_type != kt || j.S.key_type != kt)
            return fail(ctx, JN_ERR_INVALID, "jn_batch: all tables of a batch share one key type");
        if (j.reserved != 0 || !valid_op(j.op)) return fail(ctx, JN_ERR_INVALID, "jn_batch: bad join");
        if (!band && j.op != JN_EQ)
            return fail(ctx, JN_ERR_UNSUPPORTED, "jn_batch: a join without a band must be an equi-join");
    }
    JN_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->info = jn_run_info();
    const uint64_t l0 = ctx->launches_total;
    jn_status st = kt == JN_KEY_I32
                       ? batch_typed<int32_t>(ctx, count, joins, out, capacity, n_out, first, pairs, count_only)
                       : batch_typed<int64_t>(ctx, count, joins, out, capacity, n_out, first, pairs, count_only);
    ctx->info.kernel_launches = ctx->launches_total - l0;
    return st;
}

jn_status jn_batch(jn_ctx* ctx, int32_t count, const jn_join* joins, jn_pair** out, uint64_t capacity,
                   uint64_t* n_out, uint64_t* first, uint64_t* pairs) {
    return batch_entry(ctx, count, joins, out, capacity, n_out, first, pairs, false);
}

jn_status jn_batch_count(jn_ctx* ctx, int32_t count, const jn_join* joins, uint64_t* pairs, uint64_t* total) {
    if (!ctx) return JN_ERR_INVALID;
    if (count > 0 && !pairs) return fail(ctx, JN_ERR_INVALID, "jn_batch_count: NULL pairs");
    std::vector<uint64_t> first(count > 0 ? count : 1);
    jn_pair* none = nullptr;
    uint64_t n = 0;
    const jn_status st = batch_entry(ctx, count, joins, &none, 0, &n, first.data(), pairs, true);
    if (st == JN_OK && total) *total = n;
    return st;
}

jn_status jn_theta(jn_ctx* ctx, const jn_table* R, const jn_table* S, int32_t op, int64_t band,
                   jn_pair** out, uint64_t capacity, uint64_t* n_out) {
    jn_pred p;
    p.op_a = op;
    p.op_k = JN_ANY;
    p.band = band;
    return run(ctx, JN_ALGO_THETA, R, S, &p, MODE_EMIT, out, capacity, n_out, nullptr, nullptr);
}

}  // extern "C"
