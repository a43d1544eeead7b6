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
constexpr int HJ_CAP = 4096;       // R rows per shared-memory table
constexpr int HJ_SCH = 4096;       // S rows per work item
constexpr int HJ_LGNB_MAX = 11;    // at most 2048 buckets
constexpr int HJ_PAD = 16;         // rows of slack for 16-byte widened copies

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

// One work item: rows [rbeg, rbeg + rn) of R and [sbeg, sbeg + sn) of S.
struct Item {
    unsigned long long rbeg, sbeg;
    int rn, sn;
};

// Writes the items of every partition (its R chunks x S chunks) at
// items[item_prefix[p] ...].
__global__ void k_item_desc(const uint64_t* __restrict__ roff, const uint64_t* __restrict__ soff,
                            const uint64_t* __restrict__ item_prefix, int P, Item* __restrict__ items) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const uint64_t i0 = item_prefix[p], i1 = item_prefix[p + 1];
    if (i0 == i1) return;
    const uint64_t nr = roff[p + 1] - roff[p], ns = soff[p + 1] - soff[p];
    const uint64_t nrc = (nr + HJ_CAP - 1) / HJ_CAP;
    for (uint64_t it = i0; it < i1; it++) {
        const uint64_t local = it - i0;
        const uint64_t rc = local % nrc, sc = local / nrc;
        Item d;
        d.rbeg = roff[p] + rc * HJ_CAP;
        d.rn = (int)min((uint64_t)HJ_CAP, nr - rc * HJ_CAP);
        d.sbeg = soff[p] + sc * HJ_SCH;
        d.sn = (int)min((uint64_t)HJ_SCH, ns - sc * HJ_SCH);
        items[it] = d;
    }
}

// Starts the copy of rows [beg, beg + n) into `g` (widened to 16 bytes);
// returns the byte offset of row `beg` inside the staged span.
template <typename R>
__device__ __forceinline__ uint32_t stage_span(const R* rows, uint64_t beg, int n, void* g, uint64_t* bar) {
    const uint64_t lo = (beg * sizeof(R)) & ~15ull;
    const uint64_t hi = ((beg + n) * sizeof(R) + 15) & ~15ull;
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, (uint32_t)(hi - lo));
    tma_load_1d(g, reinterpret_cast<const unsigned char*>(rows) + lo, (uint32_t)(hi - lo), bar);
    return (uint32_t)(beg * sizeof(R) - lo);
}

template <typename R>
__device__ __forceinline__ uint32_t span_off(uint64_t beg) {
    return (uint32_t)(beg * sizeof(R) - ((beg * sizeof(R)) & ~15ull));
}

// MODE_COUNT: item_val[it] = matches of the item.
// MODE_AGG:   as COUNT, and chk += sum over matches of f(r) * g(s).
// MODE_EMIT:  writes the item's pairs at out[item_off[it] ...].
// Items are dealt round-robin over the persistent blocks.  The R and S rows
// of an item are staged by TMA bulk copies: the next item's R rows load
// while this item probes, its S rows while it builds.  The partitioned rows
// are library scratch, 16-byte aligned and padded by HJ_PAD rows, so every
// widened copy stays inside its allocation.
template <typename K, int MODE>
__global__ void __launch_bounds__(HJ_T, 2)
k_hash_join(const Row<K, false>* __restrict__ rrows, const Row<K, false>* __restrict__ srows,
            const Item* __restrict__ items, uint64_t nitems, int bits, unsigned long long* __restrict__ item_val,
            unsigned long long* __restrict__ chk, const uint64_t* __restrict__ item_off,
            jn_pair* __restrict__ out, unsigned int* __restrict__ err) {
    using R = Row<K, false>;
    constexpr int GR = HJ_CAP + 32 / (int)sizeof(R) + 2;
    constexpr int GS = HJ_SCH + 32 / (int)sizeof(R) + 2;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* g_r = smem;                                  // GR rows
    unsigned char* g_s = g_r + GR * sizeof(R);                  // GS rows
    K* s_key = reinterpret_cast<K*>(g_s + GS * sizeof(R));      // HJ_CAP
    int32_t* s_pay = reinterpret_cast<int32_t*>(s_key + HJ_CAP);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_pay + HJ_CAP);  // 1 << HJ_LGNB_MAX
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t tmp32[33];
    __shared__ uint32_t s_cursor;
    __shared__ __align__(8) uint64_t bar_r, bar_s;

    const int lane = threadIdx.x & 31;
    uint64_t it = blockIdx.x;
    if (it >= nitems) return;
    Item d = items[it];
    if (threadIdx.x == 0) {
        mbar_init(&bar_r, 1);
        mbar_init(&bar_s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_span<R>(rrows, d.rbeg, d.rn, g_r, &bar_r);
        stage_span<R>(srows, d.sbeg, d.sn, g_s, &bar_s);
        s_cursor = 0;
    }
    __syncthreads();
    uint32_t phase = 0;
    while (true) {
        const uint64_t itn = it + gridDim.x;
        const bool has_next = itn < nitems;
        Item dn;
        if (has_next) dn = items[itn];  // used once this item's staging is free
        const int rn = d.rn, sn = d.sn;
        const int lg = bucket_bits(rn);
        const int nb = 1 << lg;
        for (int i = threadIdx.x; i < nb; i += HJ_T) s_off[i] = 0;
        bool ok = mbar_wait(&bar_r, phase, err);
        if (__syncthreads_or(!ok)) {
            mbar_wait(&bar_r, phase, nullptr);
            mbar_wait(&bar_s, phase, nullptr);
            break;
        }
        // ---- build: counting sort of the staged R chunk by bucket ----
        const R* rrow = reinterpret_cast<const R*>(g_r + span_off<R>(d.rbeg));
        for (int i = threadIdx.x; i < rn; i += HJ_T)
            atomicAdd(&s_off[bucket_of(khash(rrow[i].key), bits, lg)], 1u);
        __syncthreads();
        {
            uint32_t v[4];
            uint32_t sum = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = threadIdx.x * 4 + j;
                v[j] = i < nb ? s_off[i] : 0u;
                sum += v[j];
            }
            uint32_t tot;
            uint32_t pre = block_excl_scan(sum, tmp32, &tot);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = threadIdx.x * 4 + j;
                if (i < nb) s_off[i] = pre;
                pre += v[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < rn; i += HJ_T) {
            const R x = rrow[i];
            const uint32_t pos = atomicAdd(&s_off[bucket_of(khash(x.key), bits, lg)], 1u);
            s_key[pos] = x.key;
            s_pay[pos] = x.pay;
        }
        __syncthreads();
        // bucket b now holds rows [b ? s_off[b-1] : 0, s_off[b]); R staging is free
        if (threadIdx.x == 0 && has_next) stage_span<R>(rrows, dn.rbeg, dn.rn, g_r, &bar_r);
        ok = mbar_wait(&bar_s, phase, err);
        if (__syncthreads_or(!ok)) {
            mbar_wait(&bar_s, phase, nullptr);
            if (has_next) mbar_wait(&bar_r, phase ^ 1u, nullptr);
            break;
        }
        // ---- probe with the staged S chunk ----
        const R* srow = reinterpret_cast<const R*>(g_s + span_off<R>(d.sbeg));
        unsigned long long acc = 0, csum = 0;
        const int rounds = (sn + HJ_T - 1) / HJ_T;
        for (int r = 0; r < rounds; r++) {
            const int j = r * HJ_T + threadIdx.x;
            uint32_t lo = 0, hi = 0;
            R x;
            x.key = 0;
            x.pay = 0;
            if (j < sn) {
                x = srow[j];
                const uint32_t b = bucket_of(khash(x.key), bits, lg);
                lo = b ? s_off[b - 1] : 0u;
                hi = s_off[b];
            }
            uint32_t m = 0;
            unsigned long long fs = 0;
            for (uint32_t e = lo; e < hi; e++) {
                if (s_key[e] == x.key) {
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
                        if (s_key[e] == x.key) {
                            jn_pair q;
                            q.r = s_pay[e];
                            q.s = x.pay;
                            out[o++] = q;
                        }
                    }
                }
            } else {
                acc += m;
                if (MODE == MODE_AGG && m) csum += fs * chk_g(x.pay);
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
        __syncthreads();  // S staging and the table are free
        if (threadIdx.x == 0) {
            s_cursor = 0;
            if (has_next) stage_span<R>(srows, dn.sbeg, dn.sn, g_s, &bar_s);
        }
        if (!has_next) break;
        __syncthreads();
        phase ^= 1u;
        it = itn;
        d = dn;
    }
}

template <typename K>
static size_t hash_smem() {
    using R = Row<K, false>;
    const size_t gr = HJ_CAP + 32 / sizeof(R) + 2, gs = HJ_SCH + 32 / sizeof(R) + 2;
    return (gr + gs) * sizeof(R) + (size_t)HJ_CAP * (sizeof(K) + 4) + sizeof(uint32_t) * (1u << HJ_LGNB_MAX);
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

// Partitions one table through both passes.  Outputs the partitioned rows
// and offsets[P + 1].
template <typename K>
struct Partitioned {
    Row<K, false>* rows = nullptr;
    uint64_t* off = nullptr;  // P + 1 exact offsets
};

template <typename K>
static jn_status partition_table(jn_ctx* c, Scratch& s, const Cols<K>& T, int b1, int b2,
                                 const uint32_t* other_bitmap, uint32_t fmask,
                                 const unsigned long long* hist1, Partitioned<K>* outp,
                                 uint64_t* d_survivors, unsigned int* work) {
    using R = Row<K, false>;
    const int F1 = 1 << b1, F2 = 1 << b2, P = F1 * F2;
    const uint64_t n = (uint64_t)T.n;
    // ---- pass 1: regions sized by the unfiltered histogram ----
    uint64_t *start1, *seg_b, *seg_c, *tp;
    unsigned long long* cur1;
    R* r1;
    JN_TRY(s.get(&start1, F1 + 1));
    JN_TRY(s.get(&cur1, F1));
    JN_TRY(s.get(&seg_b, F1 + 1));
    JN_TRY(s.get(&seg_c, F1 + 1));
    JN_TRY(s.get(&tp, F1 + 2));
    JN_TRY(s.get(&r1, n + HJ_PAD));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist1), start1, F1));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((F1 + 255) / 256), dim3(256), 0,
                  (const uint64_t*)start1, cur1, (int64_t)F1));
    JN_TRY(launch(c, K_SEGMENTS, k_one_segment, dim3(1), dim3(32), 0, seg_b, seg_c, tp, n));
    const size_t sm = scatter_smem<K, false>();
    auto kern1 = other_bitmap ? k_scatter<K, false, true, HashDigit> : k_scatter<K, false, false, HashDigit>;
    const int g1 = persistent_grid(c, (const void*)kern1, SC_T, sm);
    HashDigit d1{32 - b1, (uint32_t)(F1 - 1)};
    PartIn<K, false> in1{T.key, nullptr, T.pay, nullptr, n};
    JN_TRY(launch(c, K_SCATTER, kern1, dim3(g1), dim3(SC_T), sm, in1, (const uint64_t*)seg_b,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, 1, d1, F1, other_bitmap, fmask, cur1, r1,
                  c->d_err));
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
    auto kh = k_seg_hist_rows<R, HashDigit>;
    const size_t smh = sizeof(uint32_t) * F2;
    const int gh = persistent_grid(c, (const void*)kh, SC_T, smh);
    JN_TRY(launch(c, K_HIST, kh, dim3(gh), dim3(SC_T), smh, (const R*)r1, (const uint64_t*)start1,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, F1, d2, F2, hist2));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist2), start2, P));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((P + 255) / 256), dim3(256), 0,
                  (const uint64_t*)start2, cur2, (int64_t)P));
    // ---- pass 2 ----
    R* r2;
    JN_TRY(s.get(&r2, n + HJ_PAD));
    auto kern2 = k_scatter<K, false, false, HashDigit>;
    const int g2 = persistent_grid(c, (const void*)kern2, SC_T, sm);
    PartIn<K, false> in2{nullptr, nullptr, nullptr, r1, n + HJ_PAD};
    JN_TRY(launch(c, K_SCATTER, kern2, dim3(g2), dim3(SC_T), sm, in2, (const uint64_t*)start1,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, F1, d2, F2, (const uint32_t*)nullptr, 0u, cur2,
                  r2, c->d_err));
    outp->rows = r2;
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
        if (b > 20) b = 20;
    }
    int b1 = tu.radix_bits1 ? tu.radix_bits1 : b / 2;
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
    // the join kernel stages rows with 16-byte bulk copies from these columns
    if ((((uintptr_t)PR.rows) | ((uintptr_t)PS.rows)) & 15)
        return fail(c, JN_ERR_CUDA, "partition scratch is not 16-byte aligned");
    Item* idesc;
    JN_TRY(s.get(&idesc, nitems));
    JN_TRY(launch(c, K_ITEMS, k_item_desc, dim3((P + 255) / 256), dim3(256), 0, (const uint64_t*)PR.off,
                  (const uint64_t*)PS.off, (const uint64_t*)iprefix, P, idesc));
    unsigned long long *ival, *chk;
    uint64_t* ioff;
    JN_TRY(s.get(&ival, nitems));
    JN_TRY(s.get(&ioff, nitems + 1));
    JN_TRY(s.get(&chk, 1));
    JN_TRY(zero(c, chk, 8));
    const size_t smj = hash_smem<K>();
    auto kc = (mode == MODE_AGG) ? k_hash_join<K, MODE_AGG> : k_hash_join<K, MODE_COUNT>;
    const int gj = (int)min((uint64_t)persistent_grid(c, (const void*)kc, HJ_T, smj), nitems);
    JN_TRY(launch(c, K_HASH_COUNT, kc, dim3(gj), dim3(HJ_T), smj, (const Row<K, false>*)PR.rows,
                  (const Row<K, false>*)PS.rows, (const Item*)idesc, nitems, b, ival, chk,
                  (const uint64_t*)nullptr, (jn_pair*)nullptr, c->d_err));
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
        const int ge = (int)min((uint64_t)persistent_grid(c, (const void*)ke, HJ_T, smj), nitems);
        JN_TRY(launch(c, K_HASH_EMIT, ke, dim3(ge), dim3(HJ_T), smj, (const Row<K, false>*)PR.rows,
                      (const Row<K, false>*)PS.rows, (const Item*)idesc, nitems, b,
                      (unsigned long long*)nullptr, (unsigned long long*)nullptr, (const uint64_t*)ioff,
                      plan->dev, c->d_err));
    }
    JN_TRY(out_finish(c, hc[0], *plan));
    return JN_OK;
}

template jn_status run_hash<int32_t>(jn_ctx*, const Cols<int32_t>&, const Cols<int32_t>&, int,
                                     OutPlan*, RunResult*);
template jn_status run_hash<int64_t>(jn_ctx*, const Cols<int64_t>&, const Cols<int64_t>&, int,
                                     OutPlan*, RunResult*);

}  // namespace jnx
