// Autotuner: picks tuning knobs by timing them.
//
// The knobs that shape the work without changing the result -- the hash
// join's partition path and bits, pre-filter and R rows per shared-memory
// table, the theta join's group count, the nested loop's R tile, a batch's
// rows per partition -- are tried on the caller's own inputs (the full join
// when its pairs fit in memory, else the count and checksum), the fastest is
// applied to the context, and the choice is cached per (algorithm, key type,
// log2 |R|, log2 |S|) so a later call for the same size class costs nothing.
// This plays the part of the paper's choice of alpha
// (Sec. 5.1.4 and 5.2.4 sweep it by hand and report the best range).
#include <algorithm>
#include <chrono>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "jn_algos.h"
#include "jn_common.cuh"

namespace {

using Key = std::tuple<int, int, int, int>;
std::mutex g_mu;
std::map<Key, jn_tuning> g_cache;

// Host time of one call that synchronises before it returns.
double time_call(const std::function<jn_status()>& f, jn_status* st) {
    const auto t0 = std::chrono::steady_clock::now();
    *st = f();
    const auto t1 = std::chrono::steady_clock::now();
    return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

}  // namespace

extern "C" {

jn_status jn_autotune(jn_ctx* c, int32_t algo, const jn_table* R, const jn_table* S, const jn_pred* pred,
                      jn_tuning* best) {
    if (!c || !R || !S) return JN_ERR_INVALID;
    const Key key{algo, R->key_type, jnx::ceil_log2((uint64_t)R->n + 1), jnx::ceil_log2((uint64_t)S->n + 1)};
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            jn_tuning t = it->second;
            t.sms = c->tune.sms;  // the SM budget is the context's own, not a tuned knob
            c->tune = t;
            if (best) *best = t;
            return JN_OK;
        }
    }
    const jn_tuning base = c->tune;
    std::vector<jn_tuning> cands;
    if (algo == JN_ALGO_HASH || algo == JN_ALGO_SORT) {
        const int full = jnx::hash_cap(R->key_type);
        // the region path filters a table only at its second level, after
        // moving all of it once; the two-pass path drops the rows the
        // pre-filter rejects in its first pass, which wins when the filter
        // removes most of a large table
        for (int path : {2, 1})
            for (int cap : {full, full / 2})  // R rows per shared-memory table
                for (int pre : {0, 1, 2, 3}) {  // off, both tables, only S, only R
                    const uint64_t target = (pre == 1 || pre == 3) ? cap : cap / 2;  // R rows per partition
                    int b = jnx::ceil_log2(jnx::ceil_div((uint64_t)R->n + 1, target));
                    for (int d = -1; d <= 1; d++) {
                        jn_tuning t = base;
                        t.prefilter = pre;
                        t.radix_bits = std::max(1, std::min(20, b + d));
                        t.radix_bits1 = 0;
                        t.table_rows = cap;
                        t.hash_path = path;
                        cands.push_back(t);
                    }
                }
    } else if (algo == JN_ALGO_THETA) {
        for (int g = 2; g <= 10; g += 2) {
            jn_tuning t = base;
            t.theta_groups = g;
            cands.push_back(t);
        }
    } else if (algo == JN_ALGO_NLJ) {
        for (int tr : {512, 1024, 2048, 4096}) {
            jn_tuning t = base;
            t.nlj_tile_r = tr;
            cands.push_back(t);
        }
    } else {
        return JN_ERR_INVALID;
    }
    uint64_t cnt = 0;
    jn_status st = jn_count(c, algo, R, S, pred, &cnt);  // warm-up (and argument check)
    if (st != JN_OK) return st;
    // Each candidate runs the call the caller will run: the join that writes
    // its pairs when they fit a quarter of the free device memory (the knobs
    // change what the emit pass reads as much as the count pass), otherwise
    // count and checksum.
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const bool emit = cnt > 0 && cnt * sizeof(jn_pair) <= free_b / 4;
    jn_pred pr{JN_EQ, JN_ANY, -1};
    if (pred) pr = *pred;
    auto one = [&]() -> jn_status {
        if (!emit) {
            uint64_t chk = 0;
            return jn_aggregate(c, algo, R, S, pred, &cnt, &chk);
        }
        jn_pair* out = nullptr;
        uint64_t n = 0;
        jn_status r = algo == JN_ALGO_HASH    ? jn_hash(c, R, S, &out, 0, &n)
                      : algo == JN_ALGO_SORT  ? jn_sort_merge(c, R, S, &out, 0, &n)
                      : algo == JN_ALGO_THETA ? jn_theta(c, R, S, pr.op_a, pr.band, &out, 0, &n)
                                              : jn_nested_loop(c, R, S, pred, &out, 0, &n);
        if (out) {
            cudaStreamSynchronize(c->stream);
            jn_free(c, out);
        }
        return r;
    };
    double best_ms = 1e30;
    jn_tuning pick = base;
    for (const jn_tuning& t : cands) {
        c->tune = t;
        double ms = 1e30;
        for (int rep = 0; rep < 2; rep++) {  // the faster of two runs: host noise only adds time
            const double x = time_call([&] {
                const jn_status r = one();
                if (r == JN_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
                    cudaGetLastError();
                    return JN_ERR_CUDA;
                }
                return r;
            }, &st);
            if (st != JN_OK) break;
            ms = std::min(ms, x);
        }
        if (st == JN_OK && ms < best_ms) {
            best_ms = ms;
            pick = t;
        }
    }
    c->tune = pick;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_cache[key] = pick;
    }
    if (best) *best = pick;
    return JN_OK;
}

jn_status jn_autotune_batch(jn_ctx* c, int32_t count, const jn_join* joins, jn_tuning* best) {
    if (!c || count < 1 || !joins) return JN_ERR_INVALID;
    uint64_t rows = 0;
    for (int i = 0; i < count; i++) rows += (uint64_t)joins[i].R.n + (uint64_t)joins[i].S.n;
    const Key key{100, joins[0].R.key_type, jnx::ceil_log2((uint64_t)count), jnx::ceil_log2(rows + 1)};
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            jn_tuning t = it->second;
            t.sms = c->tune.sms;  // the SM budget is the context's own, not a tuned knob
            c->tune = t;
            if (best) *best = t;
            return JN_OK;
        }
    }
    const jn_tuning base = c->tune;
    std::vector<uint64_t> pairs(count), first(count);
    uint64_t total = 0;
    jn_status st = jn_batch_count(c, count, joins, pairs.data(), &total);  // warm-up (and argument check)
    if (st != JN_OK) return st;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    // the whole batch with its pairs when they fit a quarter of the free
    // memory, otherwise its count phases
    const bool emit = total > 0 && total * sizeof(jn_pair) <= free_b / 4;
    auto trial = [&](jn_status* st) {
        if (!emit) {
            *st = jn_batch_count(c, count, joins, pairs.data(), nullptr);
            return;
        }
        jn_pair* out = nullptr;
        uint64_t n = 0;
        *st = jn_batch(c, count, joins, &out, 0, &n, first.data(), pairs.data());
        if (out) {
            cudaStreamSynchronize(c->stream);
            jn_free(c, out);
        }
    };
    double best_ms = 1e30;
    jn_tuning pick = base;
    for (int rows_per_part : {1024, 2048, 4096}) {
        for (int graphs : {0, 1}) {
            jn_tuning t = base;
            t.part_rows = rows_per_part;
            t.graphs = graphs;
            c->tune = t;
            const double ms = time_call([&] { trial(&st); return st; }, &st);
            if (st == JN_OK && ms < best_ms) {
                best_ms = ms;
                pick = t;
            }
        }
    }
    c->tune = pick;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_cache[key] = pick;
    }
    if (best) *best = pick;
    return JN_OK;
}

}  // extern "C"
