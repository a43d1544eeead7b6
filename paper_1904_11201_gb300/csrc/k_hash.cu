// Partitioned equi hash join (Sec. 3.3.2) with Algorithm 1's pre-filter
// (Sec. 3.1) and an exact count pass in place of Eq. (rsize) (Sec. 3.3.3).
//
// Pipeline on one stream (R = build side, S = probe side):
//   1. presence: one read of each key column sets a bit per key in the
//      table's presence bitmap and counts first-pass digits.  A tuple is kept
//      only if its key's bit is set in the other table's bitmap (the common
//      key set of Algorithm 1's first Map-Reduce round).
//   2. partition pass 1 (b1 bits of the key hash), filtered; regions are
//      sized by the unfiltered counts and filled through atomic cursors.
//   3. partition pass 2 (b2 more bits), exact offsets from a histogram of
//      the pass-1 output.  Partition p = top (b1 + b2) hash bits; the pair of
//      passes plays the role of the shuffle on join_key / alpha.
//   4. work items (partition, R chunk, S chunk); count pass builds a
//      shared-memory hash table on the R chunk and probes with the S chunk;
//      exclusive scan of the per-item counts gives exact output offsets and
//      the total (one 8-byte read-back).
//   5. one exact allocation, then the emit pass repeats build and probe and
//      writes (R.payload, S.payload) pairs at the scanned offsets.
#include "jn_algos.h"
#include "jn_partition.cuh"

namespace jnx {

constexpr int HJ_T = 512;          // threads per join block
constexpr int HJ_CAP = 8192;       // R rows per shared-memory table
constexpr int HJ_SCH = 8192;       // S rows per work item
constexpr int HJ_LGNB_MAX = 11;    // at most 2048 buckets

// Items of partition p: ceil(nr / CAP) R chunks x ceil(ns / SCH) S chunks.
__global__ void k_items(const uint64_t* __restrict__ roff, const uint64_t* __restrict__ soff, int P,
                        uint64_t* __restrict__ items) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    uint64_t nr = roff[p + 1] - roff[p], ns = soff[p + 1] - soff[p];
    items[p] = (nr && ns) ? ((nr + HJ_CAP - 1) / HJ_CAP) * ((ns + HJ_SCH - 1) / HJ_SCH) : 0;
}

__device__ __forceinline__ int bucket_bits(int rn) {
    int lg = 0;
    while ((1 << lg) < rn) lg++;
    lg -= 1;  // about two rows per bucket
    return lg < 0 ? 0 : (lg > HJ_LGNB_MAX ? HJ_LGNB_MAX : lg);
}

__device__ __forceinline__ uint32_t bucket_of(uint32_t h, int bits, int lg) {
    return lg == 0 ? 0u : ((h << bits) >> (32 - lg));
}

// MODE_COUNT: item_val[it] = matches of the item.
// MODE_AGG:   as COUNT, and chk += sum over matches of f(r) * g(s).
// MODE_EMIT:  writes the item's pairs at out[item_off[it] ...].
template <typename K, int MODE>
__global__ void __launch_bounds__(HJ_T)
k_hash_join(const K* __restrict__ rk, const int32_t* __restrict__ rp, const uint64_t* __restrict__ roff,
            const K* __restrict__ sk, const int32_t* __restrict__ sp, const uint64_t* __restrict__ soff,
            const uint64_t* __restrict__ item_prefix, int P, int bits,
            unsigned long long* __restrict__ item_val, unsigned long long* __restrict__ chk,
            const uint64_t* __restrict__ item_off, jn_pair* __restrict__ out,
            unsigned int* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_key = reinterpret_cast<K*>(smem);
    int32_t* s_pay = reinterpret_cast<int32_t*>(s_key + HJ_CAP);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_pay + HJ_CAP);  // (1 << HJ_LGNB_MAX) words
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t tmp32[33];
    __shared__ unsigned int s_item;
    __shared__ uint32_t s_cursor;

    const uint64_t nitems = item_prefix[P];
    const int lane = threadIdx.x & 31;
    while (true) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(work, 1u);
            s_cursor = 0;
        }
        __syncthreads();
        const uint64_t it = s_item;
        if (it >= nitems) break;
        const int p = find_segment(item_prefix, P, it);
        const uint64_t nr = roff[p + 1] - roff[p], ns = soff[p + 1] - soff[p];
        const uint64_t nrc = (nr + HJ_CAP - 1) / HJ_CAP;
        const uint64_t local = it - item_prefix[p];
        const uint64_t rc = local % nrc, sc = local / nrc;
        const uint64_t rbeg = roff[p] + rc * HJ_CAP;
        const int rn = (int)min((uint64_t)HJ_CAP, nr - rc * HJ_CAP);
        const uint64_t sbeg = soff[p] + sc * HJ_SCH;
        const int sn = (int)min((uint64_t)HJ_SCH, ns - sc * HJ_SCH);
        const int lg = bucket_bits(rn);
        const int nb = 1 << lg;

        // ---- build: counting sort of the R chunk by bucket ----
        for (int i = threadIdx.x; i < nb; i += HJ_T) s_off[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < rn; i += HJ_T)
            atomicAdd(&s_off[bucket_of(khash(rk[rbeg + i]), bits, lg)], 1u);
        __syncthreads();
        {
            // exclusive scan of nb <= 2048 counters, 4 per thread
            uint32_t v[4];
            uint32_t sum = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                int i = threadIdx.x * 4 + j;
                v[j] = i < nb ? s_off[i] : 0u;
                sum += v[j];
            }
            uint32_t tot;
            uint32_t pre = block_excl_scan(sum, tmp32, &tot);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                int i = threadIdx.x * 4 + j;
                if (i < nb) s_off[i] = pre;
                pre += v[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < rn; i += HJ_T) {
            const K k = rk[rbeg + i];
            const uint32_t pos = atomicAdd(&s_off[bucket_of(khash(k), bits, lg)], 1u);
            s_key[pos] = k;
            s_pay[pos] = rp[rbeg + i];
        }
        __syncthreads();
        // now bucket b holds rows [b ? s_off[b-1] : 0, s_off[b])

        // ---- probe with the S chunk ----
        unsigned long long acc = 0, csum = 0;
        const int rounds = (sn + HJ_T - 1) / HJ_T;
        for (int r = 0; r < rounds; r++) {
            const int j = r * HJ_T + threadIdx.x;
            uint32_t lo = 0, hi = 0;
            K k = 0;
            int32_t pay = 0;
            if (j < sn) {
                k = __ldcs(sk + sbeg + j);
                pay = __ldcs(sp + sbeg + j);
                const uint32_t b = bucket_of(khash(k), bits, lg);
                lo = b ? s_off[b - 1] : 0u;
                hi = s_off[b];
            }
            uint32_t m = 0;
            unsigned long long fs = 0;
            for (uint32_t e = lo; e < hi; e++) {
                if (s_key[e] == k) {
                    m++;
                    if (MODE == MODE_AGG) fs += chk_f(s_pay[e]);
                }
            }
            if (MODE == MODE_EMIT) {
                const uint32_t incl = warp_incl_scan(m);
                const uint32_t wt = __shfl_sync(0xffffffffu, incl, 31);
                uint32_t base = 0;
                if (lane == 0 && wt) base = atomicAdd(&s_cursor, wt);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (m) {
                    uint64_t o = item_off[it] + base + (incl - m);
                    for (uint32_t e = lo; e < hi; e++) {
                        if (s_key[e] == k) {
                            jn_pair q;
                            q.r = s_pay[e];
                            q.s = pay;
                            out[o++] = q;
                        }
                    }
                }
            } else {
                acc += m;
                if (MODE == MODE_AGG && m) csum += fs * chk_g(pay);
            }
        }
        if (MODE != MODE_EMIT) {
            const unsigned long long tot = block_sum(acc, tmp64);
            if (MODE == MODE_AGG) {
                const unsigned long long ct = block_sum(csum, tmp64);
                if (threadIdx.x == 0 && ct) atomicAdd(chk, ct);
            }
            if (threadIdx.x == 0) item_val[it] = tot;
        }
        __syncthreads();
    }
}

template <typename K>
static size_t hash_smem() {
    return (size_t)HJ_CAP * (sizeof(K) + 4) + sizeof(uint32_t) * (1u << HJ_LGNB_MAX);
}

static int persistent_grid(jn_ctx* c, const void* fn, int threads, size_t smem) {
    int per = 0;
    if (smem > 48 * 1024) ensure_smem(fn, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    if (per < 1) per = 1;
    return per * c->num_sms;
}

// Partitions one table through both passes.  Outputs the partitioned key and
// payload columns and offsets[P + 1].
template <typename K>
struct Partitioned {
    K* key = nullptr;
    int32_t* pay = nullptr;
    uint64_t* off = nullptr;  // P + 1 exact offsets
};

template <typename K>
static jn_status partition_table(jn_ctx* c, Scratch& s, const Cols<K>& T, int b1, int b2,
                                 const uint32_t* other_bitmap, uint32_t fmask,
                                 const unsigned long long* hist1, Partitioned<K>* outp,
                                 uint64_t* d_survivors, unsigned int* work) {
    const int F1 = 1 << b1, F2 = 1 << b2, P = F1 * F2;
    const uint64_t n = (uint64_t)T.n;
    // ---- pass 1: regions sized by the unfiltered histogram ----
    uint64_t *start1, *seg_b, *seg_c, *tp;
    unsigned long long* cur1;
    K* k1;
    int32_t* p1;
    JN_TRY(s.get(&start1, F1 + 1));
    JN_TRY(s.get(&cur1, F1));
    JN_TRY(s.get(&seg_b, F1 + 1));
    JN_TRY(s.get(&seg_c, F1 + 1));
    JN_TRY(s.get(&tp, F1 + 2));
    JN_TRY(s.get(&k1, n));
    JN_TRY(s.get(&p1, n));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist1), start1, F1));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((F1 + 255) / 256), dim3(256), 0,
                  (const uint64_t*)start1, cur1, (int64_t)F1));
    JN_TRY(launch(c, K_SEGMENTS, k_one_segment, dim3(1), dim3(32), 0, seg_b, seg_c, tp, n));
    const size_t sm = scatter_smem<K>(false);
    auto kern1 = other_bitmap ? k_scatter<K, true, HashDigit> : k_scatter<K, false, HashDigit>;
    const int g1 = persistent_grid(c, (const void*)kern1, SC_T, sm);
    HashDigit d1{32 - b1, (uint32_t)(F1 - 1)};
    JN_TRY(zero(c, work, sizeof(unsigned int)));
    JN_TRY(launch(c, K_SCATTER, kern1, dim3(g1), dim3(SC_T), sm, T.key, (const K*)nullptr, T.pay,
                  (const uint64_t*)seg_b, (const uint64_t*)seg_c, (const uint64_t*)tp, 1, d1, F1,
                  other_bitmap, fmask, cur1, k1, (K*)nullptr, p1, work));
    // ---- pass 1 regions become the segments of pass 2 ----
    JN_TRY(launch(c, K_SEGMENTS, k_segments, dim3(1), dim3(1024), 0, (const unsigned long long*)cur1,
                  (const uint64_t*)start1, F1, seg_c, tp, d_survivors));
    unsigned long long* hist2;
    uint64_t* start2;
    unsigned long long* cur2;
    JN_TRY(s.get(&hist2, P));
    JN_TRY(s.get(&start2, P + 1));
    JN_TRY(s.get(&cur2, P));
    JN_TRY(zero(c, hist2, sizeof(unsigned long long) * P));
    HashDigit d2{32 - b1 - b2, (uint32_t)(F2 - 1)};
    auto kh = k_seg_hist<K, HashDigit>;
    const size_t smh = sizeof(uint32_t) * F2;
    const int gh = persistent_grid(c, (const void*)kh, SC_T, smh);
    JN_TRY(zero(c, work, sizeof(unsigned int)));
    JN_TRY(launch(c, K_HIST, kh, dim3(gh), dim3(SC_T), smh, (const K*)k1, (const uint64_t*)start1,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, F1, d2, F2, hist2, work));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist2), start2, P));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((P + 255) / 256), dim3(256), 0,
                  (const uint64_t*)start2, cur2, (int64_t)P));
    // ---- pass 2 ----
    K* k2;
    int32_t* p2;
    JN_TRY(s.get(&k2, n));
    JN_TRY(s.get(&p2, n));
    auto kern2 = k_scatter<K, false, HashDigit>;
    const int g2 = persistent_grid(c, (const void*)kern2, SC_T, sm);
    JN_TRY(zero(c, work, sizeof(unsigned int)));
    JN_TRY(launch(c, K_SCATTER, kern2, dim3(g2), dim3(SC_T), sm, (const K*)k1, (const K*)nullptr,
                  (const int32_t*)p1, (const uint64_t*)start1, (const uint64_t*)seg_c,
                  (const uint64_t*)tp, F1, d2, F2, (const uint32_t*)nullptr, 0u, cur2, k2,
                  (K*)nullptr, p2, work));
    outp->key = k2;
    outp->pay = p2;
    outp->off = start2;
    return JN_OK;
}

template <typename K>
jn_status run_hash(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int mode, OutPlan* plan,
                   RunResult* res) {
    const uint64_t nr = (uint64_t)R.n, ns = (uint64_t)S.n;
    jn_run_info& info = c->info;
    if (nr == 0 || ns == 0) {
        res->count = 0;
        res->checksum = 0;
        if (mode == MODE_EMIT) {
            Scratch s0(c);
            JN_TRY(out_prepare(c, s0, 0, *plan));
            JN_TRY(out_finish(c, 0, *plan));
        }
        return JN_OK;
    }
    const jn_tuning& tu = c->tune;
    // ---- parameters ----
    int b = tu.radix_bits;
    if (b == 0) {
        uint64_t target = HJ_CAP / 2;  // expected R rows per partition
        b = ceil_log2((nr + target - 1) / target);
        if (b > 16) b = 16;
    }
    int b1 = tu.radix_bits1 ? tu.radix_bits1 : (b + 1) / 2;
    if (b1 > b) b1 = b;
    if (b1 > 10) b1 = 10;
    if (b - b1 > 10) b1 = b - 10;
    const int b2 = b - b1;
    const int F1 = 1 << b1, P = 1 << b;
    bool pre = tu.prefilter == 1 || (tu.prefilter == -1 && nr + ns >= (1u << 22));
    int fb = tu.filter_bits ? tu.filter_bits : ceil_log2(nr + ns) + 1;
    if (fb < 10) fb = 10;
    if (fb > 28 && tu.filter_bits == 0) fb = 28;
    const uint64_t fwords = pre ? (uint64_t(1) << fb) / 32 : 0;
    const uint32_t fmask = (uint32_t)((uint64_t(1) << fb) - 1);

    Scratch s(c);
    unsigned int* work;
    uint64_t* d_small;  // [0] R survivors, [1] S survivors
    JN_TRY(s.get(&work, 4));
    JN_TRY(s.get(&d_small, 8));
    uint32_t *bmR = nullptr, *bmS = nullptr;
    unsigned long long *h1R, *h1S;
    JN_TRY(s.get(&h1R, F1));
    JN_TRY(s.get(&h1S, F1));
    JN_TRY(zero(c, h1R, sizeof(unsigned long long) * F1));
    JN_TRY(zero(c, h1S, sizeof(unsigned long long) * F1));
    if (pre) {
        JN_TRY(s.get(&bmR, fwords));
        JN_TRY(s.get(&bmS, fwords));
        JN_TRY(zero(c, bmR, fwords * 4));
        JN_TRY(zero(c, bmS, fwords * 4));
    }
    // ---- 1. presence bitmaps + first-pass histograms ----
    HashDigit d1{32 - b1, (uint32_t)(F1 - 1)};
    {
        auto kp = k_presence_hist<K>;
        const size_t smp = sizeof(uint32_t) * F1;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kp, 512, smp);
        if (per < 1) per = 1;
        const int g = per * c->num_sms;
        JN_TRY(launch(c, K_PRESENCE, kp, dim3(g), dim3(512), smp, R.key, R.n, bmR, fmask, d1, F1, h1R));
        JN_TRY(launch(c, K_PRESENCE, kp, dim3(g), dim3(512), smp, S.key, S.n, bmS, fmask, d1, F1, h1S));
    }
    // ---- 2-3. two partition passes per table (filtered by the other's bitmap) ----
    Partitioned<K> PR, PS;
    JN_TRY(partition_table<K>(c, s, R, b1, b2, bmS, fmask, h1R, &PR, d_small + 0, work));
    JN_TRY(partition_table<K>(c, s, S, b1, b2, bmR, fmask, h1S, &PS, d_small + 1, work));
    // ---- 4. work items and the count pass ----
    uint64_t *items, *iprefix;
    JN_TRY(s.get(&items, P));
    JN_TRY(s.get(&iprefix, P + 1));
    JN_TRY(launch(c, K_ITEMS, k_items, dim3((P + 255) / 256), dim3(256), 0, (const uint64_t*)PR.off,
                  (const uint64_t*)PS.off, P, items));
    JN_TRY(scan_u64(c, items, iprefix, P));
    uint64_t h[3];
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)(iprefix + P),
                  d_small + 2, 1));
    JN_TRY(read_back(c, d_small, h, 3));
    const uint64_t nitems = h[2];
    info.r_survivors = h[0];
    info.s_survivors = h[1];
    info.partitions = (uint64_t)P;
    info.work_items = nitems;
    info.prefilter = pre ? 1 : 0;
    info.radix_bits = b;
    info.radix_bits1 = b1;
    info.filter_bits = pre ? fb : 0;
    info.heavy_keys = 0;
    if (nitems == 0) {
        res->count = 0;
        res->checksum = 0;
        if (mode == MODE_EMIT) {
            JN_TRY(out_prepare(c, s, 0, *plan));
            JN_TRY(out_finish(c, 0, *plan));
        }
        return JN_OK;
    }
    unsigned long long *ival, *chk;
    uint64_t* ioff;
    JN_TRY(s.get(&ival, nitems));
    JN_TRY(s.get(&ioff, nitems + 1));
    JN_TRY(s.get(&chk, 1));
    JN_TRY(zero(c, chk, 8));
    const size_t smj = hash_smem<K>();
    auto kc = (mode == MODE_AGG) ? k_hash_join<K, MODE_AGG> : k_hash_join<K, MODE_COUNT>;
    const int gj = persistent_grid(c, (const void*)kc, HJ_T, smj);
    JN_TRY(zero(c, work, 4));
    JN_TRY(launch(c, K_HASH_COUNT, kc, dim3(gj), dim3(HJ_T), smj, (const K*)PR.key,
                  (const int32_t*)PR.pay, (const uint64_t*)PR.off, (const K*)PS.key,
                  (const int32_t*)PS.pay, (const uint64_t*)PS.off, (const uint64_t*)iprefix, P, b, ival,
                  chk, (const uint64_t*)nullptr, (jn_pair*)nullptr, work));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(ival), ioff, (int64_t)nitems));
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)(ioff + nitems),
                  d_small + 3, 1));
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)chk, d_small + 4, 1));
    uint64_t hc[2];
    JN_TRY(read_back(c, d_small + 3, hc, 2));
    res->count = hc[0];
    res->checksum = hc[1];
    info.result = hc[0];
    if (mode != MODE_EMIT) return JN_OK;
    // ---- 5. exact allocation and the emit pass ----
    JN_TRY(out_prepare(c, s, hc[0], *plan));
    if (hc[0] > 0) {
        auto ke = k_hash_join<K, MODE_EMIT>;
        const int ge = persistent_grid(c, (const void*)ke, HJ_T, smj);
        JN_TRY(zero(c, work, 4));
        JN_TRY(launch(c, K_HASH_EMIT, ke, dim3(ge), dim3(HJ_T), smj, (const K*)PR.key,
                      (const int32_t*)PR.pay, (const uint64_t*)PR.off, (const K*)PS.key,
                      (const int32_t*)PS.pay, (const uint64_t*)PS.off, (const uint64_t*)iprefix, P, b,
                      (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                      (const uint64_t*)ioff, plan->dev, work));
    }
    JN_TRY(out_finish(c, hc[0], *plan));
    return JN_OK;
}

template jn_status run_hash<int32_t>(jn_ctx*, const Cols<int32_t>&, const Cols<int32_t>&, int,
                                     OutPlan*, RunResult*);
template jn_status run_hash<int64_t>(jn_ctx*, const Cols<int64_t>&, const Cols<int64_t>&, int,
                                     OutPlan*, RunResult*);

}  // namespace jnx
