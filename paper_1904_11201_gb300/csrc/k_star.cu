// Star join: a centre table R with two join columns (fk1 = key, fk2 = key2)
// against two dimension tables, S1 on fk1 and S2 on fk2.  Sec. 6 leaves
// multi-table joins to future work; this is the two-table method applied
// twice, as a left-deep plan:
//   1. J1 = R (fk1, row index) joined with S1 by the partitioned hash join;
//   2. the fk2 of every J1 pair's R row is gathered into a key column T1;
//   3. J2 = T1 (row index = J1 index) joined with S2 by the same hash join;
//   4. every J2 pair (j, s2) becomes the triple (R payload of J1[j], J1[j].s, s2).
// Both joins keep their exact count pass, so J1, J2 and the triples are each
// allocated once at their exact size.
#include <string.h>

#include "jn_algos.h"

namespace jnx {

constexpr int ST_ILP = 4;  // gathers in flight per thread

// t1key[i] = fk2[J1[i].r]: the second join column of each first-join pair's R
// row.  A block covers 256 * ST_ILP consecutive pairs; each thread issues its
// ST_ILP random reads of fk2 before it stores any (the reads are independent).
template <typename K>
__global__ void __launch_bounds__(256)
k_star_keys(const jn_pair* __restrict__ j1, uint64_t m1, const K* __restrict__ fk2, K* __restrict__ t1key) {
    const uint64_t base = (uint64_t)blockIdx.x * (256 * ST_ILP) + threadIdx.x;
    int32_t r[ST_ILP];
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) {
        const uint64_t i = base + (uint64_t)u * 256;
        r[u] = i < m1 ? j1[i].r : -1;
    }
    K v[ST_ILP];
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) v[u] = r[u] >= 0 ? fk2[r[u]] : K(0);
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) {
        const uint64_t i = base + (uint64_t)u * 256;
        if (i < m1) t1key[i] = v[u];
    }
}

// out[i] = (R payload of J1[J2[i].r] (its row index when rpay is NULL),
// J1[J2[i].r].s, J2[i].s), with ST_ILP independent gather chains per thread.
__global__ void __launch_bounds__(256)
k_star_emit(const jn_pair* __restrict__ j1, const jn_pair* __restrict__ j2, uint64_t m2,
            const int32_t* __restrict__ rpay, jn_triple* __restrict__ out) {
    const uint64_t base = (uint64_t)blockIdx.x * (256 * ST_ILP) + threadIdx.x;
    jn_pair b[ST_ILP], a[ST_ILP];
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) {
        const uint64_t i = base + (uint64_t)u * 256;
        b[u] = i < m2 ? j2[i] : jn_pair{-1, 0};
    }
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) a[u] = b[u].r >= 0 ? j1[b[u].r] : jn_pair{-1, 0};
    int32_t p[ST_ILP];
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) p[u] = (rpay && a[u].r >= 0) ? rpay[a[u].r] : a[u].r;
#pragma unroll
    for (int u = 0; u < ST_ILP; u++) {
        const uint64_t i = base + (uint64_t)u * 256;
        if (i < m2) {
            jn_triple t;
            t.r = p[u];
            t.s1 = a[u].s;
            t.s2 = b[u].s;
            out[i] = t;
        }
    }
}

namespace {

// Library-allocated pairs of an inner join, freed (stream-ordered) on scope exit.
struct Pairs {
    jn_ctx* c;
    jn_pair* p = nullptr;
    uint64_t n = 0;
    explicit Pairs(jn_ctx* ctx) : c(ctx) {}
    ~Pairs() {
        if (p) jn_free(c, p);
    }
};

// One block per 256 * ST_ILP elements.
unsigned grid_for(uint64_t n) { return (unsigned)((n + 256 * ST_ILP - 1) / (256 * ST_ILP)); }

template <typename K>
jn_status star_typed(jn_ctx* c, const jn_table* R, const jn_table* S1, const jn_table* S2, jn_triple** out,
                     uint64_t capacity, uint64_t* n_out, uint64_t* count) {
    // 1. R (fk1, row index) joined with S1
    jn_table r1 = *R;
    r1.key2 = nullptr;
    r1.payload = nullptr;
    Pairs j1(c);
    JN_TRY(jn_hash(c, &r1, S1, &j1.p, 0, &j1.n));
    if (j1.n > (uint64_t)INT32_MAX)
        return fail(c, JN_ERR_UNSUPPORTED, "star join: the first join has more than 2^31 - 1 pairs");
    // 2. the fk2 of each pair's R row
    Scratch s(c);
    K* t1key = nullptr;
    if (j1.n) {
        JN_TRY(s.get(&t1key, j1.n));
        JN_TRY(launch(c, K_STAR, k_star_keys<K>, dim3(grid_for(j1.n)), dim3(256), 0, (const jn_pair*)j1.p,
                      j1.n, (const K*)R->key2, t1key));
    }
    jn_table t1;
    memset(&t1, 0, sizeof(t1));
    t1.key = t1key;
    t1.n = (int64_t)j1.n;
    t1.key_type = R->key_type;
    // 3. joined with S2 (count only when that is all that is asked)
    if (count) return jn_count(c, JN_ALGO_HASH, &t1, S2, nullptr, count);
    Pairs j2(c);
    JN_TRY(jn_hash(c, &t1, S2, &j2.p, 0, &j2.n));
    // 4. the triples, at their exact size, in the caller's buffer or a new one
    const uint64_t m = j2.n;
    jn_triple* user = *out;
    if (user && m > capacity) {
        *n_out = m;
        return fail(c, JN_ERR_CAPACITY, "output buffer holds fewer triples than the result");
    }
    jn_triple* dev = nullptr;
    bool copy_back = false;
    if (!user) {
        if (m) JN_TRY(dalloc(c, reinterpret_cast<void**>(&dev), m * sizeof(jn_triple)));
    } else if (m == 0 || is_device_pointer(user)) {
        dev = user;
    } else {
        JN_TRY(s.get(&dev, m));
        copy_back = true;
    }
    if (m)
        JN_TRY(launch(c, K_STAR, k_star_emit, dim3(grid_for(m)), dim3(256), 0, (const jn_pair*)j1.p,
                      (const jn_pair*)j2.p, m, (const int32_t*)R->payload, dev));
    if (copy_back) JN_CUDA(c, cudaMemcpyAsync(user, dev, m * sizeof(jn_triple), cudaMemcpyDefault, c->stream));
    JN_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!user) *out = dev;
    *n_out = m;
    return JN_OK;
}

jn_status star_entry(jn_ctx* c, const jn_table* R, const jn_table* S1, const jn_table* S2, jn_triple** out,
                     uint64_t capacity, uint64_t* n_out, uint64_t* count) {
    if (!c) return JN_ERR_INVALID;
    c->err.clear();
    if (!R || !S1 || !S2) return fail(c, JN_ERR_INVALID, "star join: NULL table");
    if (count ? false : (!out || !n_out)) return fail(c, JN_ERR_INVALID, "star join: NULL output pointer");
    if (R->key_type != S1->key_type || R->key_type != S2->key_type)
        return fail(c, JN_ERR_INVALID, "star join: key types differ");
    if (R->key_type != JN_KEY_I32 && R->key_type != JN_KEY_I64)
        return fail(c, JN_ERR_INVALID, "star join: key_type must be JN_KEY_I32 or JN_KEY_I64");
    if (R->n < 0 || R->n > INT32_MAX || R->reserved)
        return fail(c, JN_ERR_INVALID, "star join: R row count out of range or reserved set");
    if (R->n > 0 && (!R->key || !R->key2)) return fail(c, JN_ERR_INVALID, "star join: R needs key and key2");
    JN_CUDA(c, cudaSetDevice(c->device));
    // R's second join column and payloads are read by this file's kernels
    if (R->n > 0 && (!is_device_pointer(R->key2) || (R->payload && !is_device_pointer(R->payload))))
        return fail(c, JN_ERR_INVALID, "star join: R's key2 and payload must be device memory");
    const uint64_t l0 = c->launches_total;
    const jn_status st = R->key_type == JN_KEY_I32 ? star_typed<int32_t>(c, R, S1, S2, out, capacity, n_out, count)
                                                   : star_typed<int64_t>(c, R, S1, S2, out, capacity, n_out, count);
    c->info.kernel_launches = c->launches_total - l0;
    return st;
}

}  // namespace
}  // namespace jnx

using namespace jnx;

extern "C" {

jn_status jn_star(jn_ctx* ctx, const jn_table* R, const jn_table* S1, const jn_table* S2, jn_triple** out,
                  uint64_t capacity, uint64_t* n_out) {
    return star_entry(ctx, R, S1, S2, out, capacity, n_out, nullptr);
}

jn_status jn_star_count(jn_ctx* ctx, const jn_table* R, const jn_table* S1, const jn_table* S2,
                        uint64_t* count) {
    if (!count) return JN_ERR_INVALID;
    return star_entry(ctx, R, S1, S2, nullptr, 0, nullptr, count);
}

void jn_free_triples(jn_ctx* ctx, jn_triple* p) {
    if (p) cudaFreeAsync(p, ctx ? ctx->stream : (cudaStream_t)0);
}

}  // extern "C"
