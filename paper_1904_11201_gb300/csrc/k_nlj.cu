// Nested-loop join (Sec. 3.3.1): every (R, S) pair is tested.
//
// The paper's grid gives each thread NB_S = |S|/(m x) + 1 rows of S and
// NB_T = |T|/(n y) + 1 rows of T (Eqs. NBS, NBT, IDS, IDT) and a private
// result buffer of NB_S * NB_T pairs.  Here a block holds a tile of R rows in
// shared memory and a tile of S rows in registers (NLJ_SPT per thread), so
// every R value read from shared memory is compared against NLJ_SPT S rows.
// The predicate of each S row is turned, once, into an interval test on the
// R value ("R.x op s" <=> R.x in [lo, hi], possibly negated), which makes the
// inner loop a subtract and an unsigned compare per column.  A count pass
// writes one count per tile; an exclusive scan gives each tile its exact
// output offset (replacing the NB_S * NB_T per-thread buffers); the emit pass
// repeats the comparisons and writes pairs.
#include <mutex>

#include "jn_algos.h"

namespace jnx {

constexpr int NLJ_T = 256;
#ifndef JN_NLJ_SPT
#define JN_NLJ_SPT 4
#endif
constexpr int NLJ_SPT = JN_NLJ_SPT;  // S rows per thread
constexpr int NLJ_STILE = NLJ_T * NLJ_SPT;

// An R row's two predicate columns, adjacent in shared memory so that one
// load fetches both.
template <typename K>
struct __align__(2 * sizeof(K)) KPair {
    K a, b;
};

template <typename K, bool HAS2, int MODE>
__global__ void __launch_bounds__(NLJ_T)
k_nlj(const K* __restrict__ rk, const K* __restrict__ rk2, const int32_t* __restrict__ rp, int64_t nr,
      const K* __restrict__ sk, const K* __restrict__ sk2, const int32_t* __restrict__ sp, int64_t ns,
      int op_a, int op_k, long long band, int tr, unsigned long long* __restrict__ tile_val,
      unsigned long long* __restrict__ chk, const uint64_t* __restrict__ tile_off,
      jn_pair* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    // R tile: (a, b) pairs with a second column, else the a column alone
    K* s_a = reinterpret_cast<K*>(smem);
    KPair<K>* s_ab = reinterpret_cast<KPair<K>*>(smem);
    int32_t* s_p = reinterpret_cast<int32_t*>(s_a + (HAS2 ? 2 : 1) * tr);
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t s_cur;

    const uint64_t tile = (uint64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (MODE == MODE_EMIT) {
        // tiles without results have nothing to write
        if (tile_off[tile + 1] == tile_off[tile]) return;
    }
    const int64_t r0 = (int64_t)blockIdx.y * tr;
    const int rn = (int)min((int64_t)tr, nr - r0);
    for (int i = threadIdx.x; i < rn; i += NLJ_T) {
        if (HAS2)
            s_ab[i] = KPair<K>{rk[r0 + i], rk2[r0 + i]};
        else
            s_a[i] = rk[r0 + i];
        s_p[i] = rp ? rp[r0 + i] : (int32_t)(r0 + i);
    }
    if (threadIdx.x == 0) s_cur = 0;

    Interval<K> ia[NLJ_SPT], ib[NLJ_SPT];
    int32_t spay[NLJ_SPT];
    bool valid[NLJ_SPT];
    const int64_t s0 = (int64_t)blockIdx.x * NLJ_STILE;
#pragma unroll
    for (int j = 0; j < NLJ_SPT; j++) {
        const int64_t s = s0 + j * NLJ_T + threadIdx.x;
        valid[j] = s < ns;
        K a = valid[j] ? sk[s] : (K)0;
        ia[j] = op_interval<K>(valid[j] ? op_a : JN_ANY, a);
        if (!valid[j]) {  // an empty set: never matches
            ia[j].inv = true;
            ia[j].lo = sizeof(K) == 4 ? (K)INT32_MIN : (K)INT64_MIN;
            ia[j].span = ~(decltype(ia[j].span))0;
        }
        if (HAS2) {
            K b = valid[j] ? sk2[s] : (K)0;
            ib[j] = band >= 0 ? band_interval<K>(b, band) : op_interval<K>(op_k, b);
        }
        spay[j] = valid[j] ? (sp ? sp[s] : (int32_t)s) : 0;
    }
    // Inverted intervals (!=, and the empty sets of invalid rows and of
    // "< min" / "> max") take the general test; a warp whose rows have none
    // runs the plain interval test, which needs no inversion step per pair.
    bool inv = false;
#pragma unroll
    for (int j = 0; j < NLJ_SPT; j++) inv |= ia[j].inv || (HAS2 && ib[j].inv);
    const bool plain = !__any_sync(0xffffffffu, inv);
    __syncthreads();

    unsigned long long acc = 0, csum = 0;
    auto visit = [&](auto test) {
        for (int i = 0; i < rn; i++) {
            K a, b = 0;
            if (HAS2) {
                const KPair<K> ab = s_ab[i];
                a = ab.a;
                b = ab.b;
            } else {
                a = s_a[i];
            }
            if (MODE == MODE_EMIT) {
                // one branch per R row: matches are rare, the tests are not
                uint32_t mask = 0;
#pragma unroll
                for (int j = 0; j < NLJ_SPT; j++) mask |= (uint32_t)test(j, a, b) << j;
                if (mask) {
#pragma unroll
                    for (int j = 0; j < NLJ_SPT; j++) {
                        if ((mask >> j) & 1u) {
                            const uint32_t slot = atomicAdd(&s_cur, 1u);
                            st_pair(out + tile_off[tile] + slot, s_p[i], spay[j]);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < NLJ_SPT; j++) {
                    const bool m = test(j, a, b);
                    acc += m;
                    if (MODE == MODE_AGG && m) csum += chk_f(s_p[i]) * chk_g(spay[j]);
                }
            }
        }
    };
    if (plain)
        visit([&](int j, K a, K b) {
            bool m = in_range(a, ia[j].lo, ia[j].span);
            if (HAS2) m &= in_range(b, ib[j].lo, ib[j].span);
            return m;
        });
    else
        visit([&](int j, K a, K b) {
            bool m = iv_test(ia[j], a);
            if (HAS2) m &= iv_test(ib[j], b);
            return m;
        });
    if (MODE != MODE_EMIT) {
        const unsigned long long t = block_sum(acc, tmp64);
        if (MODE == MODE_AGG) {
            const unsigned long long c = block_sum(csum, tmp64);
            if (threadIdx.x == 0 && c) atomicAdd(chk, c);
        }
        if (threadIdx.x == 0) tile_val[tile] = t;
    }
}

template <typename K, bool HAS2>
static jn_status nlj_launch(jn_ctx* c, int mode, dim3 grid, size_t smem, const Cols<K>& R,
                            const Cols<K>& S, const jn_pred& pr, int tr, unsigned long long* val,
                            unsigned long long* chk, const uint64_t* off, jn_pair* out) {
    const int kid = mode == MODE_EMIT ? K_NLJ_EMIT : K_NLJ_COUNT;
    if (mode == MODE_EMIT)
        return launch(c, kid, k_nlj<K, HAS2, MODE_EMIT>, grid, dim3(NLJ_T), smem, R.key, R.key2, R.pay,
                      R.n, S.key, S.key2, S.pay, S.n, pr.op_a, pr.op_k, (long long)pr.band, tr, val,
                      chk, off, out);
    if (mode == MODE_AGG)
        return launch(c, kid, k_nlj<K, HAS2, MODE_AGG>, grid, dim3(NLJ_T), smem, R.key, R.key2, R.pay,
                      R.n, S.key, S.key2, S.pay, S.n, pr.op_a, pr.op_k, (long long)pr.band, tr, val,
                      chk, off, out);
    return launch(c, kid, k_nlj<K, HAS2, MODE_COUNT>, grid, dim3(NLJ_T), smem, R.key, R.key2, R.pay,
                  R.n, S.key, S.key2, S.pay, S.n, pr.op_a, pr.op_k, (long long)pr.band, tr, val, chk,
                  off, out);
}

template <typename K>
jn_status run_nlj(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, const jn_pred& pred, int mode,
                  OutPlan* plan, RunResult* res) {
    jn_run_info& info = c->info;
    if (R.n == 0 || S.n == 0) {
        res->count = res->checksum = 0;
        if (mode == MODE_EMIT) {
            Scratch s0(c);
            JN_TRY(out_prepare(c, s0, 0, *plan));
            JN_TRY(out_finish(c, 0, *plan));
        }
        return JN_OK;
    }
    const bool has2 = R.key2 != nullptr && S.key2 != nullptr;
    int tr = c->tune.nlj_tile_r ? c->tune.nlj_tile_r : 1024;
    if (ceil_div(R.n, tr) > 65535)
        return fail(c, JN_ERR_UNSUPPORTED, "nested loop: R has more than 65535 tiles; use a larger nlj_tile_r");
    const dim3 grid((unsigned)ceil_div(S.n, NLJ_STILE), (unsigned)ceil_div(R.n, tr));
    const uint64_t tiles = (uint64_t)grid.x * grid.y;
    const size_t smem = (size_t)tr * (sizeof(K) * (has2 ? 2 : 1) + 4);
    Scratch s(c);
    unsigned long long *val, *chk;
    uint64_t *off, *d_small;
    JN_TRY(s.get(&val, tiles));
    JN_TRY(s.get(&off, tiles + 1));
    JN_TRY(s.get(&chk, 1));
    JN_TRY(s.get(&d_small, 2));
    JN_TRY(zero(c, chk, 8));
    const int cm = mode == MODE_AGG ? MODE_AGG : MODE_COUNT;
    if (has2)
        JN_TRY((nlj_launch<K, true>(c, cm, grid, smem, R, S, pred, tr, val, chk, nullptr, nullptr)));
    else
        JN_TRY((nlj_launch<K, false>(c, cm, grid, smem, R, S, pred, tr, val, chk, nullptr, nullptr)));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(val), off, (int64_t)tiles));
    JN_CUDA(c, cudaMemcpyAsync(d_small, off + tiles, 8, cudaMemcpyDeviceToDevice, c->stream));
    JN_CUDA(c, cudaMemcpyAsync(d_small + 1, chk, 8, cudaMemcpyDeviceToDevice, c->stream));
    uint64_t h[2];
    JN_TRY(read_back(c, d_small, h, 2));
    res->count = h[0];
    res->checksum = h[1];
    info.result = h[0];
    info.partitions = tiles;
    info.work_items = tiles;
    info.r_survivors = (uint64_t)R.n;
    info.s_survivors = (uint64_t)S.n;
    info.prefilter = 0;
    info.cartesian_bound = (uint64_t)R.n * (uint64_t)S.n;  // every pair is compared
    if (mode != MODE_EMIT) return JN_OK;
    JN_TRY(out_prepare(c, s, h[0], *plan));
    if (h[0] > 0) {
        if (has2)
            JN_TRY((nlj_launch<K, true>(c, MODE_EMIT, grid, smem, R, S, pred, tr, nullptr, nullptr, off,
                                        plan->dev)));
        else
            JN_TRY((nlj_launch<K, false>(c, MODE_EMIT, grid, smem, R, S, pred, tr, nullptr, nullptr,
                                         off, plan->dev)));
    }
    JN_TRY(out_finish(c, h[0], *plan));
    return JN_OK;
}

// ------------------------------------------------------ allocation-free --
// A nested-loop join for callers that may not allocate device memory at all:
// code running inside a region where the application owns every byte of the
// device (a fixed memory plan, a real-time or serving loop that forbids
// cudaMalloc / cudaFree and the synchronisation they bring), or code that
// must not touch any allocator, the library's pool included.  Its scratch
// (per-tile counts, their scan and the checksum word) lives in the fixed
// device array below, so a call allocates nothing; the caller supplies the
// output buffer.
constexpr int NA_MAX_TILES = 65536;  // R tiles x S tiles per call
static __device__ __align__(256) unsigned long long g_na_scratch[2 * NA_MAX_TILES + 8];

// Device address of g_na_scratch, looked up once per device (host code
// cannot use the symbol itself as an address).
static std::mutex g_na_mu;
static void* g_na_addr[64];

static jn_status na_scratch(void** p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return JN_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_addr[dev]) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_na_scratch) != cudaSuccess || !a) {
            cudaGetLastError();
            return JN_ERR_CUDA;
        }
        g_na_addr[dev] = a;
    }
    *p = g_na_addr[dev];
    return JN_OK;
}

// Single-block exclusive scan of n <= NA_MAX_TILES counts; out[n] = total.
static __global__ void k_na_scan(const unsigned long long* __restrict__ in, int n, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long tmp[33];
    unsigned long long carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < n ? in[i] : 0ull;
        unsigned long long tot;
        const unsigned long long pre = block_excl_scan(v, tmp, &tot);
        if (i < n) out[i] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

template <typename K, bool HAS2>
static jn_status na_run(const jn_table* R, const jn_table* S, const jn_pred& pr, jn_pair* out, uint64_t capacity,
                        uint64_t* n_out, cudaStream_t st) {
    const int tr = 1024;
    const uint64_t gx = ceil_div((uint64_t)S->n, NLJ_STILE), gy = ceil_div((uint64_t)R->n, tr);
    const uint64_t tiles = gx * gy;
    if (tiles > NA_MAX_TILES || gy > 65535) return JN_ERR_INVALID;  // beyond the fixed scratch
    void* base = nullptr;
    JN_TRY(na_scratch(&base));
    unsigned long long* val = static_cast<unsigned long long*>(base);
    unsigned long long* off = val + NA_MAX_TILES;
    unsigned long long* chk = off + NA_MAX_TILES + 1;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    const size_t smem = (size_t)tr * (sizeof(K) * (HAS2 ? 2 : 1) + 4);
    const K* rk = static_cast<const K*>(R->key);
    const K* rk2 = static_cast<const K*>(R->key2);
    const K* sk = static_cast<const K*>(S->key);
    const K* sk2 = static_cast<const K*>(S->key2);
    // the array keeps the previous call's contents: counts are rewritten for
    // every tile of this call, the checksum word is cleared
    if (cudaMemsetAsync(chk, 0, sizeof(unsigned long long), st) != cudaSuccess) return JN_ERR_CUDA;
    k_nlj<K, HAS2, MODE_COUNT><<<grid, NLJ_T, smem, st>>>(rk, rk2, R->payload, R->n, sk, sk2, S->payload, S->n,
                                                          pr.op_a, pr.op_k, (long long)pr.band, tr, val, chk,
                                                          nullptr, nullptr);
    k_na_scan<<<1, 1024, 0, st>>>(val, (int)tiles, off);
    if (cudaGetLastError() != cudaSuccess) return JN_ERR_CUDA;
    uint64_t total = 0;
    if (cudaMemcpyAsync(&total, off + tiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return JN_ERR_CUDA;
    }
    *n_out = total;
    if (total > capacity) return JN_ERR_CAPACITY;
    if (total > 0) {
        k_nlj<K, HAS2, MODE_EMIT><<<grid, NLJ_T, smem, st>>>(rk, rk2, R->payload, R->n, sk, sk2, S->payload, S->n,
                                                             pr.op_a, pr.op_k, (long long)pr.band, tr, nullptr,
                                                             nullptr, reinterpret_cast<const uint64_t*>(off), out);
        if (cudaGetLastError() != cudaSuccess) return JN_ERR_CUDA;
    }
    return JN_OK;
}

template jn_status run_nlj<int32_t>(jn_ctx*, const Cols<int32_t>&, const Cols<int32_t>&,
                                    const jn_pred&, int, OutPlan*, RunResult*);
template jn_status run_nlj<int64_t>(jn_ctx*, const Cols<int64_t>&, const Cols<int64_t>&,
                                    const jn_pred&, int, OutPlan*, RunResult*);

}  // namespace jnx

using namespace jnx;

extern "C" jn_status jn_nested_loop_noalloc(const jn_table* R, const jn_table* S, const jn_pred* pred,
                                            jn_pair* out, uint64_t capacity, uint64_t* n_out, void* stream) {
    if (!R || !S || !n_out || (capacity > 0 && !out)) return JN_ERR_INVALID;
    if (R->key_type != S->key_type || (R->key_type != JN_KEY_I32 && R->key_type != JN_KEY_I64)) return JN_ERR_INVALID;
    if (R->n < 0 || S->n < 0 || R->n > INT32_MAX || S->n > INT32_MAX || R->reserved || S->reserved)
        return JN_ERR_INVALID;
    jn_pred pr;
    pr.op_a = JN_EQ;
    pr.op_k = JN_ANY;
    pr.band = -1;
    if (pred) pr = *pred;
    if (pr.op_a < JN_EQ || pr.op_a > JN_ANY || pr.op_k < JN_EQ || pr.op_k > JN_ANY) return JN_ERR_INVALID;
    // columns, output and stream on the current device (whose scratch address
    // the call looks up): nothing may be staged, no other device's array used
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return JN_ERR_CUDA;
    }
    const void* cols[6] = {R->key, R->key2, R->payload, S->key, S->key2, S->payload};
    for (const void* c : cols)
        if (c && pointer_device(c) != dev) return JN_ERR_INVALID;
    if (capacity > 0 && pointer_device(out) != dev) return JN_ERR_INVALID;
    if (((uintptr_t)out & 7) != 0) return JN_ERR_INVALID;  // pairs are stored as 8-byte words
    if (stream) {
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return JN_ERR_INVALID;
        }
        if (sdev != dev) return JN_ERR_INVALID;
    }
    if (R->n == 0 || S->n == 0) {
        *n_out = 0;
        return JN_OK;
    }
    if ((R->n > 0 && !R->key) || (S->n > 0 && !S->key)) return JN_ERR_INVALID;
    const bool has2 = R->key2 && S->key2;
    cudaStream_t st = (cudaStream_t)stream;
    if (R->key_type == JN_KEY_I32)
        return has2 ? na_run<int32_t, true>(R, S, pr, out, capacity, n_out, st)
                    : na_run<int32_t, false>(R, S, pr, out, capacity, n_out, st);
    return has2 ? na_run<int64_t, true>(R, S, pr, out, capacity, n_out, st)
                : na_run<int64_t, false>(R, S, pr, out, capacity, n_out, st);
}
