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
#include <vector>

#include "jn_algos.h"
#include "jn_heavy.cuh"
#include "jn_partition.cuh"
#include "jn_region.cuh"
#include "jn_sortjoin.cuh"

namespace jnx {

// Join block shape (build-time knobs): threads, R rows per table, S rows per
// staged chunk, and blocks per SM the register budget allows.
#ifndef JN_HJ_T
#define JN_HJ_T 512
#endif
#ifndef JN_HJ_CAP
#define JN_HJ_CAP 4096
#endif
#ifndef JN_HJ_SCH
#define JN_HJ_SCH 1536
#endif
#ifndef JN_HJ_MINB
#define JN_HJ_MINB 2
#endif
constexpr int HJ_T = JN_HJ_T;        // threads per join block
constexpr int HJ_CAP = JN_HJ_CAP;    // R rows per shared-memory table (int32 keys)
constexpr int HJ_SCH = JN_HJ_SCH;    // S rows per staged chunk
#ifndef JN_HJ_PU
#define JN_HJ_PU 3  // a 1536-row chunk is three rounds of 512 threads
#endif
constexpr int HJ_PU = JN_HJ_PU;      // S rows a thread probes per round in the emit pass

#ifndef JN_SLICE_PAIRS
#define JN_SLICE_PAIRS (1ull << 24)  // host outputs of at least this many pairs are copied back in slices
#endif
constexpr int HJ_PAD = 16;         // rows of slack for 16-byte widened copies
// the sort-merge kernels hold a chunk as 8 words per thread, index its rows in
// 15 bits and sort it as a power-of-two network of at least 256 rows, in shared
// memory sized for the chunk itself (int64 chunks are HJ_CAP / 2 rows)
static_assert(HJ_CAP <= 8 * SJ_T && HJ_CAP < 0x8000, "R chunk larger than the sort-merge kernels hold");
static_assert((HJ_CAP & (HJ_CAP - 1)) == 0 && HJ_CAP >= 512,
              "R chunk must be a power of two of at least 512 rows (the sort network's size)");
constexpr uint64_t CE_PAIRS = 1u << 16;  // cross-product pairs per work chunk

// The partitions of one table: either P + 1 offsets (partition p = rows
// [off[p], off[p + 1])) or a first row and a row count per partition.
struct PartView {
    const uint64_t* off;
    const uint32_t* beg;
    const uint32_t* cnt;
    __device__ __forceinline__ uint64_t first(int p) const { return off ? off[p] : (uint64_t)beg[p]; }
    __device__ __forceinline__ uint64_t rows(int p) const { return off ? off[p + 1] - off[p] : (uint64_t)cnt[p]; }
};

// Items of partition p: one per chunk of HJ_CAP R rows; each item probes
// every S row of the partition, HJ_SCH rows at a time.  With `bound`, adds
// sum_p |R_p| * |S_p| to it: Eq. (rsize)'s allocation for these partitions.
__global__ void k_items(PartView rv, PartView sv, int P, int cap, uint64_t* __restrict__ items,
                        unsigned long long* __restrict__ bound) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t nr = 0, ns = 0;
    if (p < P) {
        nr = rv.rows(p);
        ns = sv.rows(p);
        items[p] = (nr && ns) ? (nr + cap - 1) / cap : 0;
    }
    if (bound) warp_add_to(bound, nr * ns);  // < |R| * |S| < 2^62: no overflow
}

// R rows per shared-memory table: 4096 for int32 keys, 2048 for int64.
template <typename K>
__host__ __device__ constexpr int cap_of() {
    return sizeof(K) == 4 ? HJ_CAP : HJ_CAP / 2;
}


// items[it] for every item: its partition is the last p with item_prefix[p] <= it.
__global__ void k_item_desc(PartView rv, PartView sv, const uint64_t* __restrict__ item_prefix, int P, int cap,
                            Item* __restrict__ items) {
    const uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= item_prefix[P]) return;
    const int p = find_segment(item_prefix, P, it);
    const uint64_t rc = it - item_prefix[p];
    const uint64_t nr = rv.rows(p);
    Item d;
    d.rbeg = rv.first(p) + rc * cap;
    d.rn = (int)min((uint64_t)cap, nr - rc * cap);
    d.sbeg = sv.first(p);
    d.sn = (int)sv.rows(p);
    items[it] = d;
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

// Emit-mode slot of the open-addressing table: a key and, packed in one
// word, its multiplicity (high half) and the cursor of its payload run (low
// half), so one load gives the key, the count and where its payloads sit.
template <typename K>
struct alignas(2 * sizeof(K)) RunSlot {
    K key;
    uint32_t packed;
};

// Shared-memory layout of the join kernel (bytes), shared by host and device,
// for a table of CAP_ R rows.
template <typename K, int MODE, int CAP_ = cap_of<K>()>
struct JoinSmem {
    using R = Row<K, false>;
    static constexpr int CAP = CAP_;
    static constexpr int GR = CAP + 32 / (int)sizeof(R) + 2;     // staged R rows (widened span)
    static constexpr int GS = HJ_SCH + 32 / (int)sizeof(R) + 2;  // staged S rows per buffer
    static constexpr int TS = (CAP * 5) / 4;                     // open-addressing slots
    static constexpr size_t STAGE = (size_t)(GR + 2 * GS) * sizeof(R);
    // emit: TS slots and one for the sentinel key, then the payloads grouped by slot
    static constexpr size_t TABLE =
        MODE == MODE_EMIT ? (size_t)(TS + 1) * sizeof(RunSlot<K>) + (size_t)CAP * 4
                          : (size_t)TS * (sizeof(K) + 4) + (MODE == MODE_AGG ? (size_t)TS * 8 : 0);
    static constexpr size_t BYTES = STAGE + TABLE;
};
static_assert(cap_of<int32_t>() < (1 << 16), "run cursors and counts fit half a word");

// Slot of a key in the open-addressing table of a partition: the hash bits
// below the partition bits, spread over TS slots.
__device__ __forceinline__ uint32_t oa_slot(uint32_t h, int bits, int ts) {
    const uint32_t x = (h << bits) * 0x9E3779B1u;
    return (uint32_t)(((uint64_t)x * (uint64_t)ts) >> 32);
}

// MODE_COUNT: item_val[it] = matches of the item.
// MODE_AGG:   as COUNT, and chk += sum over matches of f(r) * g(s).
// MODE_EMIT:  writes the item's pairs at out[item_off[it] ...].
//
// Items (a chunk of R rows of one partition against all S rows of that
// partition) are dealt round-robin over the persistent blocks.  R rows and S
// chunks are staged in shared memory by TMA bulk copies: the next item's R
// rows load while this item probes, and S chunks stream through two buffers,
// the next chunk loading while the current one is probed.
//   emit:         each distinct R key gets one slot holding its multiplicity
//                 and the run of its payloads in a slot-grouped array, so a
//                 match is one lookup and a contiguous copy;
//   count / agg:  equal R keys are folded into one open-addressing slot
//                 (key, multiplicity [, sum of f]), so a probe costs one
//                 lookup however many rows share the key.
// The partitioned rows are library scratch, 16-byte aligned and padded by
// HJ_PAD rows, so every widened copy stays inside its allocation.
// PU: S rows a thread probes per round.  The emit pass overlaps HJ_PU rows'
// lookups and reserves their output once; the count pass, with no output to
// reserve, measured fastest with one.
template <typename K, int MODE, bool MERGE = false, int CAP = cap_of<K>(), int PU = (MODE == MODE_EMIT ? HJ_PU : 1)>
__global__ void __launch_bounds__(HJ_T, (CAP < cap_of<K>() && MODE != MODE_EMIT) ? 3 : JN_HJ_MINB)
k_hash_join(const Row<K, false>* __restrict__ rrows, const Row<K, false>* __restrict__ srows,
            const Item* __restrict__ items, const uint64_t* __restrict__ nitems_p, int bits,
            unsigned long long* __restrict__ item_val,
            unsigned long long* __restrict__ chk, const uint64_t* __restrict__ item_off,
            jn_pair* __restrict__ out, unsigned int* __restrict__ err, uint64_t item_lo = 0,
            uint64_t item_hi = ~0ull) {
    using R = Row<K, false>;
    using L = JoinSmem<K, MODE, CAP>;
    constexpr int TS = L::TS;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* g_r = smem;
    unsigned char* g_s0 = g_r + L::GR * sizeof(R);
    unsigned char* g_s1 = g_s0 + L::GS * sizeof(R);
    unsigned char* tab = g_s1 + L::GS * sizeof(R);
    // emit table: slots (slot TS holds the sentinel key) and slot-grouped payloads
    RunSlot<K>* e_tab = reinterpret_cast<RunSlot<K>*>(tab);
    int32_t* s_pay = reinterpret_cast<int32_t*>(e_tab + TS + 1);
    constexpr int PER = (TS + 1 + HJ_T - 1) / HJ_T;  // slots per thread in the run-start scan
    // count-mode table
    K* o_key = reinterpret_cast<K*>(tab);
    uint32_t* o_cnt = reinterpret_cast<uint32_t*>(o_key + TS);
    unsigned long long* o_f = reinterpret_cast<unsigned long long*>(o_cnt + TS);
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t tmp32[33];
    __shared__ uint32_t s_cursor, s_mincnt;
    __shared__ unsigned long long s_minf;
    __shared__ __align__(8) uint64_t bar_r, bar_s[2];
    const K KMIN = key_sentinel<K>();

    const int lane = threadIdx.x & 31;
    // items [item_lo, min(*nitems_p, item_hi)) of the queue
    const uint64_t nitems = min(*nitems_p, item_hi);
    uint64_t it = item_lo + blockIdx.x;
    if (it >= nitems) return;
    Item d = items[it];
    // S-chunk stream: chunk q of this block sits in buffer q & 1; thread 0
    // stages chunks ahead (producer), every thread consumes them in order.
    uint64_t p_it = it;  // producer: item and chunk of the next chunk to stage
    int p_sc = 0, p_nsc = (d.sn + HJ_SCH - 1) / HJ_SCH;
    uint64_t p_sbeg = d.sbeg;
    int p_sn = d.sn;
    bool p_valid = true;
    uint32_t qp = 0, qc = 0;  // chunks staged / consumed
    auto stage_next_chunk = [&]() {  // thread 0 only
        if (!p_valid) return;
        const int n = min(HJ_SCH, p_sn - p_sc * HJ_SCH);
        stage_span<R>(srows, p_sbeg + (uint64_t)p_sc * HJ_SCH, n, (qp & 1) ? g_s1 : g_s0, &bar_s[qp & 1]);
        qp++;
        if (++p_sc == p_nsc) {
            p_it += gridDim.x;
            p_valid = p_it < nitems;
            if (p_valid) {
                const Item x = items[p_it];
                p_sbeg = x.sbeg;
                p_sn = x.sn;
                p_nsc = (x.sn + HJ_SCH - 1) / HJ_SCH;
                p_sc = 0;
            }
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar_r, 1);
        mbar_init(&bar_s[0], 1);
        mbar_init(&bar_s[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_span<R>(rrows, d.rbeg, d.rn, g_r, &bar_r);
        stage_next_chunk();
        stage_next_chunk();
        s_cursor = 0;
    }
    __syncthreads();
    uint32_t pr = 0;  // phase of bar_r
    bool r_pending = true;
    bool failed = false;
    while (true) {
        const uint64_t itn = it + gridDim.x;
        const bool has_next = itn < nitems;
        Item dn;
        if (has_next) dn = items[itn];  // its R rows load once this item's R staging is free
        const int rn = d.rn;
        // slots this item uses: four times its R rows (at most the table) -- a
        // slot is picked by multiply-shift, so any count works.  At a load of
        // a quarter, a lookup that misses (most of them in a selective join)
        // scans about 1.4 slots; at a half, 2.5.  The skewed variant keeps the
        // whole table
        const int ts = (MERGE || MODE == MODE_EMIT) ? TS : min(TS, max(64, 4 * rn));
        if (MODE == MODE_EMIT) {
            for (int i = threadIdx.x; i <= TS; i += HJ_T) {
                e_tab[i].key = KMIN;
                e_tab[i].packed = 0;
            }
        } else {
            for (int i = threadIdx.x; i < ts; i += HJ_T) {
                o_key[i] = KMIN;
                o_cnt[i] = 0;
                if (MODE == MODE_AGG) o_f[i] = 0;
            }
            if (threadIdx.x == 0) {
                s_mincnt = 0;
                s_minf = 0;
            }
        }
        if (__syncthreads_or(!mbar_wait(&bar_r, pr, err))) {
            failed = true;
            break;
        }
        pr ^= 1u;
        r_pending = false;
        const R* rrow = reinterpret_cast<const R*>(g_r + span_off<R>(d.rbeg));
        if (MODE == MODE_EMIT) {
            // ---- build: one slot per distinct key, then its payloads as one run ----
            // MERGE (skewed input): lanes of a warp holding the same key update
            // their slot once, to spare contended shared atomics
            const int rnw = MERGE ? (rn + 31) & ~31 : rn;
            for (int i = threadIdx.x; i < rnw; i += HJ_T) {
                const bool in = i < rn;
                R x;
                x.key = KMIN;
                x.pay = 0;
                if (in) x = rrow[i];
                uint32_t cnt = 1;
                if (MERGE) {
                    const unsigned act = __ballot_sync(0xffffffffu, in);
                    if (!in) continue;
                    const unsigned peers = __match_any_sync(act, x.key);
                    if (lane != __ffs(peers) - 1) continue;
                    cnt = __popc(peers);
                }
                uint32_t h = TS;  // the sentinel key keeps its own slot
                if (x.key != KMIN) {
                    h = oa_slot(khash(x.key), bits, TS);
                    for (int probe = 0; probe < TS; probe++) {
                        K old;
                        if (sizeof(K) == 4)
                            old = (K)atomicCAS(reinterpret_cast<int*>(&e_tab[h].key), (int)KMIN, (int)x.key);
                        else
                            old = (K)atomicCAS(reinterpret_cast<unsigned long long*>(&e_tab[h].key),
                                               (unsigned long long)KMIN, (unsigned long long)x.key);
                        if (old == KMIN || old == x.key) break;
                        h = (h + 1 == (uint32_t)TS) ? 0u : h + 1;
                    }
                }
                atomicAdd(&e_tab[h].packed, cnt << 16);
            }
            __syncthreads();
            // run starts: exclusive scan of the slot counts into the low halves
            {
                const int i0 = threadIdx.x * PER;
                uint32_t sum = 0;
#pragma unroll
                for (int k = 0; k < PER; k++)
                    if (i0 + k <= TS) sum += e_tab[i0 + k].packed >> 16;
                uint32_t tot;
                uint32_t pre = block_excl_scan(sum, tmp32, &tot);
#pragma unroll
                for (int k = 0; k < PER; k++)
                    if (i0 + k <= TS) {
                        const uint32_t p = e_tab[i0 + k].packed;
                        e_tab[i0 + k].packed = p + pre;
                        pre += p >> 16;
                    }
            }
            __syncthreads();
            // payloads into their runs; each cursor ends at its run's end
            for (int i = threadIdx.x; i < rnw; i += HJ_T) {
                const bool in = i < rn;
                R x;
                x.key = KMIN;
                x.pay = 0;
                if (in) x = rrow[i];
                uint32_t h = TS;
                if (in && x.key != KMIN) {
                    h = oa_slot(khash(x.key), bits, TS);
                    for (int probe = 0; probe < TS && e_tab[h].key != x.key; probe++)
                        h = (h + 1 == (uint32_t)TS) ? 0u : h + 1;
                }
                uint32_t pos;
                if (MERGE) {
                    const unsigned act = __ballot_sync(0xffffffffu, in);
                    if (!in) continue;
                    const unsigned peers = __match_any_sync(act, x.key);
                    const int leader = __ffs(peers) - 1;
                    uint32_t b0 = 0;
                    if (lane == leader) b0 = atomicAdd(&e_tab[h].packed, (uint32_t)__popc(peers));
                    b0 = __shfl_sync(peers, b0, leader);
                    pos = (b0 & 0xffffu) + __popc(peers & ((1u << lane) - 1));
                } else {
                    if (!in) continue;
                    pos = atomicAdd(&e_tab[h].packed, 1u) & 0xffffu;
                }
                s_pay[pos] = x.pay;
            }
        } else {
            // ---- build: fold equal keys into one slot (key, count [, sum f]) ----
            // MERGE (skewed input): lanes of a warp holding the same key insert
            // once, with their count, to spare contended shared atomics
            const int rnw = MERGE ? (rn + 31) & ~31 : rn;
            for (int i = threadIdx.x; i < rnw; i += HJ_T) {
                const bool in = i < rn;
                R x;
                x.key = KMIN;
                x.pay = 0;
                if (in) x = rrow[i];
                uint32_t cnt = 1;
                unsigned long long fv = 0;
                if (MERGE) {
                    const unsigned act = __ballot_sync(0xffffffffu, in);
                    if (!in) continue;
                    const unsigned peers = __match_any_sync(act, x.key);
                    if (MODE == MODE_AGG) {
                        // sum f over the peer group, gathered by its leader
                        const unsigned long long mine = chk_f(x.pay);
                        for (unsigned m = peers; m; m &= m - 1) fv += __shfl_sync(peers, mine, __ffs(m) - 1);
                    }
                    if ((threadIdx.x & 31) != (unsigned)(__ffs(peers) - 1)) continue;
                    cnt = __popc(peers);
                } else if (MODE == MODE_AGG) {
                    fv = chk_f(x.pay);
                }
                if (x.key == KMIN) {  // the empty-slot marker itself: kept aside
                    atomicAdd(&s_mincnt, cnt);
                    if (MODE == MODE_AGG) atomicAdd(&s_minf, fv);
                    continue;
                }
                uint32_t h = oa_slot(khash(x.key), bits, ts);
                for (int probe = 0; probe < ts; probe++) {
                    K old;
                    if (sizeof(K) == 4)
                        old = (K)atomicCAS(reinterpret_cast<int*>(o_key) + h, (int)KMIN, (int)x.key);
                    else
                        old = (K)atomicCAS(reinterpret_cast<unsigned long long*>(o_key) + h,
                                           (unsigned long long)KMIN, (unsigned long long)x.key);
                    if (old == KMIN || old == x.key) {
                        atomicAdd(&o_cnt[h], cnt);
                        if (MODE == MODE_AGG) atomicAdd(&o_f[h], fv);
                        break;
                    }
                    h = (h + 1 == (uint32_t)ts) ? 0u : h + 1;
                }
            }
        }
        __syncthreads();
        // R staging is free: stage the next item's R rows
        if (threadIdx.x == 0 && has_next) stage_span<R>(rrows, dn.rbeg, dn.rn, g_r, &bar_r);
        r_pending = has_next;
        // ---- probe with every S chunk of the partition ----
        unsigned long long acc = 0, csum = 0;
        const uint64_t ibase = MODE == MODE_EMIT ? item_off[it] : 0;
        const int nsc = (d.sn + HJ_SCH - 1) / HJ_SCH;
        for (int sc = 0; sc < nsc; sc++) {
            const uint32_t b = qc & 1, ph = (qc >> 1) & 1;
            if (__syncthreads_or(!mbar_wait(&bar_s[b], ph, err))) {
                failed = true;
                break;
            }
            const uint64_t sbeg = d.sbeg + (uint64_t)sc * HJ_SCH;
            const int sn = min(HJ_SCH, d.sn - sc * HJ_SCH);
            const R* srow = reinterpret_cast<const R*>((b ? g_s1 : g_s0) + span_off<R>(sbeg));
            const int rounds = (sn + HJ_T - 1) / HJ_T;
            // PU S rows per thread per round: their lookups and warp scans
            // overlap and one cursor reservation serves them all, while each
            // row's pairs still go out as one coalesced run per warp
            for (int r = 0; r < rounds; r += PU) {
                R x[PU];
                uint32_t m[PU], beg[PU];
                unsigned long long fs[PU];
#pragma unroll
                for (int u = 0; u < PU; u++) {
                    const int j = (r + u) * HJ_T + threadIdx.x;
                    x[u].key = 0;
                    x[u].pay = 0;
                    m[u] = 0;
                    beg[u] = 0;
                    fs[u] = 0;
                    if (j < sn) x[u] = srow[j];
                }
#pragma unroll
                for (int u = 0; u < PU; u++) {
                    const int j = (r + u) * HJ_T + threadIdx.x;
                    if (j >= sn) continue;
                    if (MODE == MODE_EMIT) {
                        uint32_t p = 0;
                        if (x[u].key == KMIN) {
                            p = e_tab[TS].packed;
                        } else {
                            uint32_t h = oa_slot(khash(x[u].key), bits, TS);
                            for (int probe = 0; probe < TS; probe++) {
                                const RunSlot<K> t = e_tab[h];
                                if (t.key == x[u].key) {
                                    p = t.packed;
                                    break;
                                }
                                if (t.key == KMIN) break;
                                h = (h + 1 == (uint32_t)TS) ? 0u : h + 1;
                            }
                        }
                        m[u] = p >> 16;
                        beg[u] = (p & 0xffffu) - m[u];
                    } else if (x[u].key == KMIN) {
                        m[u] = s_mincnt;
                        if (MODE == MODE_AGG) fs[u] = s_minf;
                    } else {
                        uint32_t h = oa_slot(khash(x[u].key), bits, ts);
                        for (int probe = 0; probe < ts; probe++) {
                            const K kk = o_key[h];
                            if (kk == x[u].key) {
                                m[u] = o_cnt[h];
                                if (MODE == MODE_AGG) fs[u] = o_f[h];
                                break;
                            }
                            if (kk == KMIN) break;
                            h = (h + 1 == (uint32_t)ts) ? 0u : h + 1;
                        }
                    }
                }
                if (MODE == MODE_EMIT) {
                    uint32_t incl[PU], wt[PU], wsum = 0;
#pragma unroll
                    for (int u = 0; u < PU; u++) {
                        incl[u] = warp_incl_scan(m[u]);
                        wt[u] = __shfl_sync(0xffffffffu, incl[u], 31);
                        wsum += wt[u];
                    }
                    uint32_t base = 0;
                    if (lane == 0 && wsum) base = atomicAdd(&s_cursor, wsum);
                    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
                    for (int u = 0; u < PU; u++) {
                        const uint64_t o = ibase + base + (incl[u] - m[u]);
                        base += wt[u];
                        // a short run is written by its lane (the lanes' first pairs
                        // are neighbours and go out together); a long run by the
                        // whole warp, 32 pairs at a time
                        const bool longr = m[u] > 4;
                        if (!longr)
                            for (uint32_t i = 0; i < m[u]; i++) st_pair(out + o + i, s_pay[beg[u] + i], x[u].pay);
                        for (unsigned lanes = __ballot_sync(0xffffffffu, longr); lanes; lanes &= lanes - 1) {
                            const int src = __ffs(lanes) - 1;
                            const uint32_t bm = __shfl_sync(0xffffffffu, m[u], src);
                            const uint32_t bb = __shfl_sync(0xffffffffu, beg[u], src);
                            const int32_t bp = __shfl_sync(0xffffffffu, x[u].pay, src);
                            const uint64_t bo = __shfl_sync(0xffffffffu, o, src);
                            for (uint32_t i = lane; i < bm; i += 32) st_pair(out + bo + i, s_pay[bb + i], bp);
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < PU; u++) {
                        acc += m[u];
                        if (MODE == MODE_AGG && m[u]) csum += fs[u] * chk_g(x[u].pay);
                    }
                }
            }
            __syncthreads();  // this S buffer is free: stage the chunk after next
            qc++;
            if (threadIdx.x == 0) stage_next_chunk();
        }
        if (failed) break;
        if (MODE != MODE_EMIT) {
            const unsigned long long tot = block_sum(acc, tmp64);
            if (MODE == MODE_AGG) {
                const unsigned long long ct = block_sum(csum, tmp64);
                if (threadIdx.x == 0 && ct) atomicAdd(chk, ct);
            }
            if (threadIdx.x == 0) item_val[it] = tot;
        }
        if (!has_next) break;
        __syncthreads();
        if (threadIdx.x == 0) s_cursor = 0;
        it = itn;
        d = dn;
    }
    if (failed) {
        // let copies in flight land before the block exits (thread 0 knows qp)
        __shared__ uint32_t s_qp;
        if (threadIdx.x == 0) s_qp = qp;
        __syncthreads();
        if (r_pending) mbar_wait(&bar_r, pr, nullptr);
        for (uint32_t q = qc; q < s_qp; q++) mbar_wait(&bar_s[q & 1], (q >> 1) & 1, nullptr);
    }
}

template <typename K>
static size_t hash_smem(int mode, int cap = cap_of<K>()) {
    constexpr int C = cap_of<K>(), H = C / 2;
    if (mode == MODE_EMIT) return cap == C ? JoinSmem<K, MODE_EMIT>::BYTES : JoinSmem<K, MODE_EMIT, H>::BYTES;
    if (mode == MODE_AGG) return cap == C ? JoinSmem<K, MODE_AGG>::BYTES : JoinSmem<K, MODE_AGG, H>::BYTES;
    return cap == C ? JoinSmem<K, MODE_COUNT>::BYTES : JoinSmem<K, MODE_COUNT, H>::BYTES;
}

// The join kernel for a table of `cap` R rows (the full table or half of it),
// with or without the skewed-input build.
template <typename K, int MODE>
static auto hash_join_kernel(bool merge, int cap) {
    constexpr int C = cap_of<K>(), H = C / 2;
    if (cap == C) return merge ? k_hash_join<K, MODE, true, C> : k_hash_join<K, MODE, false, C>;
    return merge ? k_hash_join<K, MODE, true, H> : k_hash_join<K, MODE, false, H>;
}

static int persistent_grid(jn_ctx* c, const void* fn, int threads, size_t smem) {
    int per = 0;
    if (smem > 0) ensure_smem(fn, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    if (per < 1) per = 1;
    return per * c->num_sms;
}

// Partitions one table through both passes.  Outputs the partitioned rows
// and offsets[P + 1]; with heavy keys, also the heavy rows grouped by key and
// their offsets[HV_MAX + 1].
template <typename K>
struct Partitioned {
    Row<K, false>* rows = nullptr;
    uint64_t* off = nullptr;        // P + 1 exact offsets (two radix passes), or
    uint32_t* pbeg = nullptr;       // first row and row count per partition (region path)
    uint32_t* pcnt = nullptr;
    Row<K, false>* hrows = nullptr; // heavy rows grouped by heavy key
    uint64_t* hoff = nullptr;       // HV_MAX + 1 offsets
    PartView view() const { return off ? PartView{off, nullptr, nullptr} : PartView{nullptr, pbeg, pcnt}; }
};

template <typename K, typename D1>
static jn_status partition_table(jn_ctx* c, Scratch& s, const Cols<K>& T, int b1, int b2, D1 d1,
                                 const HeavySet<K>* hs, const uint32_t* other_bitmap, uint32_t fmask,
                                 const unsigned long long* hist1, Partitioned<K>* outp, uint64_t* d_survivors) {
    using R = Row<K, false>;
    const int F1 = 1 << b1, F2 = 1 << b2, P = F1 * F2;
    const int nd1 = F1 + (hs ? 1 : 0);  // heavy rows get the extra digit F1
    const uint64_t n = (uint64_t)T.n;
    // ---- pass 1: regions sized by the unfiltered histogram ----
    uint64_t *start1, *seg_b, *seg_c, *tp;
    unsigned long long* cur1;
    R* r1;
    JN_TRY(s.get(&start1, nd1 + 1));
    JN_TRY(s.get(&cur1, nd1));
    JN_TRY(s.get(&seg_b, F1 + 1));
    JN_TRY(s.get(&seg_c, F1 + 1));
    JN_TRY(s.get(&tp, F1 + 2));
    JN_TRY(s.get(&r1, n + HJ_PAD));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hist1), start1, nd1));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((nd1 + 255) / 256), dim3(256), 0,
                  (const uint64_t*)start1, cur1, (int64_t)nd1));
    JN_TRY(launch(c, K_SEGMENTS, k_one_segment, dim3(1), dim3(32), 0, seg_b, seg_c, tp, n));
    const size_t sm = scatter_smem<K, false>();
    auto kern1 = other_bitmap ? k_scatter<K, false, true, D1> : k_scatter<K, false, false, D1>;
    const int g1 = persistent_grid(c, (const void*)kern1, SC_T, sm);
    PartIn<K, false> in1{T.key, nullptr, T.pay, nullptr, n, nullptr, nullptr, T.host};
    JN_TRY(launch(c, K_SCATTER, kern1, dim3(g1), dim3(SC_T), sm, in1, (const uint64_t*)seg_b,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, 1, d1, nd1, other_bitmap, fmask, cur1, r1,
                  c->d_err));
    // ---- pass 1 regions (without the heavy one) become the segments of pass 2 ----
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
    PartIn<K, false> in2{nullptr, nullptr, nullptr, r1, n + HJ_PAD, nullptr, nullptr};
    JN_TRY(launch(c, K_SCATTER, kern2, dim3(g2), dim3(SC_T), sm, in2, (const uint64_t*)start1,
                  (const uint64_t*)seg_c, (const uint64_t*)tp, F1, d2, F2, (const uint32_t*)nullptr, 0u, cur2,
                  r2, c->d_err));
    outp->rows = r2;
    outp->off = start2;
    if (!hs) return JN_OK;
    // ---- heavy rows (region F1) grouped by heavy key ----
    uint64_t *hseg_c, *htp, *hstart;
    unsigned long long *hhist, *hcur;
    R* hr;
    JN_TRY(s.get(&hseg_c, 2));
    JN_TRY(s.get(&htp, 3));
    JN_TRY(s.get(&hhist, HV_MAX));
    JN_TRY(s.get(&hstart, HV_MAX + 1));
    JN_TRY(s.get(&hcur, HV_MAX));
    JN_TRY(s.get(&hr, n + HJ_PAD));
    JN_TRY(zero(c, hhist, sizeof(unsigned long long) * HV_MAX));
    JN_TRY(launch(c, K_SEGMENTS, k_segments, dim3(1), dim3(32), 0, (const unsigned long long*)(cur1 + F1),
                  (const uint64_t*)(start1 + F1), 1, hseg_c, htp, (uint64_t*)nullptr));
    HeavyIdxDigit<K> dh{*hs};
    auto khh = k_seg_hist_rows<R, HeavyIdxDigit<K>>;
    const int ghh = persistent_grid(c, (const void*)khh, SC_T, sizeof(uint32_t) * HV_MAX);
    JN_TRY(launch(c, K_HIST, khh, dim3(ghh), dim3(SC_T), sizeof(uint32_t) * HV_MAX, (const R*)r1,
                  (const uint64_t*)(start1 + F1), (const uint64_t*)hseg_c, (const uint64_t*)htp, 1, dh, HV_MAX,
                  hhist));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hhist), hstart, HV_MAX));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((HV_MAX + 255) / 256), dim3(256), 0, (const uint64_t*)hstart,
                  hcur, (int64_t)HV_MAX));
    auto kern3 = k_scatter<K, false, false, HeavyIdxDigit<K>>;
    const int g3 = persistent_grid(c, (const void*)kern3, SC_T, sm);
    JN_TRY(launch(c, K_SCATTER, kern3, dim3(g3), dim3(SC_T), sm, in2, (const uint64_t*)(start1 + F1),
                  (const uint64_t*)hseg_c, (const uint64_t*)htp, 1, dh, HV_MAX, (const uint32_t*)nullptr, 0u,
                  hcur, hr, c->d_err));
    outp->hrows = hr;
    outp->hoff = hstart;
    return JN_OK;
}

// Heavy rows of a table (rows [seg[0], seg[1]) of `rows`) grouped by heavy
// key: rows and HV_MAX + 1 offsets.
template <typename K>
static jn_status group_heavy(jn_ctx* c, Scratch& s, const Row<K, false>* rows, uint64_t rows_ok, const uint64_t* seg,
                             const HeavySet<K>& hs, Partitioned<K>* outp) {
    using R = Row<K, false>;
    uint64_t *hseg_c, *htp, *hstart;
    unsigned long long *hhist, *hcur;
    R* hr;
    JN_TRY(s.get(&hseg_c, 2));
    JN_TRY(s.get(&htp, 3));
    JN_TRY(s.get(&hhist, HV_MAX));
    JN_TRY(s.get(&hstart, HV_MAX + 1));
    JN_TRY(s.get(&hcur, HV_MAX));
    JN_TRY(s.get(&hr, rows_ok));
    JN_TRY(zero(c, hhist, sizeof(unsigned long long) * HV_MAX));
    JN_TRY(launch(c, K_SEGMENTS, k_segments, dim3(1), dim3(32), 0, reinterpret_cast<const unsigned long long*>(seg + 1),
                  seg, 1, hseg_c, htp, (uint64_t*)nullptr));
    HeavyIdxDigit<K> dh{hs};
    auto kh = k_seg_hist_rows<R, HeavyIdxDigit<K>>;
    const int gh = persistent_grid(c, (const void*)kh, SC_T, sizeof(uint32_t) * HV_MAX);
    JN_TRY(launch(c, K_HIST, kh, dim3(gh), dim3(SC_T), sizeof(uint32_t) * HV_MAX, rows, seg, (const uint64_t*)hseg_c,
                  (const uint64_t*)htp, 1, dh, HV_MAX, hhist));
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(hhist), hstart, HV_MAX));
    JN_TRY(launch(c, K_MISC, k_init_cursor, dim3((HV_MAX + 255) / 256), dim3(256), 0, (const uint64_t*)hstart, hcur,
                  (int64_t)HV_MAX));
    auto ks = k_scatter<K, false, false, HeavyIdxDigit<K>>;
    const size_t sm = scatter_smem<K, false>();
    const int gs = persistent_grid(c, (const void*)ks, SC_T, sm);
    PartIn<K, false> in{nullptr, nullptr, nullptr, rows, rows_ok, nullptr, nullptr};
    JN_TRY(launch(c, K_SCATTER, ks, dim3(gs), dim3(SC_T), sm, in, seg, (const uint64_t*)hseg_c, (const uint64_t*)htp,
                  1, dh, HV_MAX, (const uint32_t*)nullptr, 0u, hcur, hr, c->d_err));
    outp->hrows = hr;
    outp->hoff = hstart;
    return JN_OK;
}

// Region path (jn_region.cuh): level-1 regions of both tables (b1 bits of
// the key hash, plus the heavy digit F1), then one block per region splits it
// into 2^b2 partitions of rows.  With `filter`, table `first` builds the
// key-presence slices and the other table is thinned by them (Algorithm 1's
// pre-filter, one side).  d_small[0] / [1] receive R's / S's rows kept.
template <typename K, typename D1>
static jn_status region_partition(jn_ctx* c, Scratch& s, const Cols<K>& R, const Cols<K>& S, int b1, int b2, D1 d1,
                                  const HeavySet<K>* hs, bool filter, int first, int fb, Partitioned<K>* PR,
                                  Partitioned<K>* PS, uint64_t* d_small) {
    using RW = Row<K, false>;
    using SH = RgShape<K>;
    const int F1 = 1 << b1, F2 = 1 << b2;
    const int nd1 = F1 + (hs ? 1 : 0);
    const int G = c->num_sms;
    const Cols<K>* T[2] = {&R, &S};
    Partitioned<K>* P[2] = {PR, PS};
    RW* rows1[2];
    uint64_t* start1[2];
    uint32_t* choff[2];
    int64_t chunk[2], nch[2];
    // level-1 histograms of both key columns (the keys land before the payloads)
    for (int t = 0; t < 2; t++) {
        const int64_t n = T[t]->n;
        const int64_t tiles = (int64_t)ceil_div((uint64_t)n, SH::T1);
        // about eight chunks per block, so blocks finish together
        const int64_t ct = max((int64_t)1, (int64_t)ceil_div((uint64_t)tiles, 8 * (uint64_t)G));
        chunk[t] = ct * SH::T1;
        nch[t] = (int64_t)ceil_div((uint64_t)n, (uint64_t)chunk[t]);
        uint32_t* hist;
        uint64_t* tot;
        JN_TRY(s.get(&hist, (size_t)nch[t] * nd1));
        JN_TRY(s.get(&choff[t], (size_t)nch[t] * nd1));
        JN_TRY(s.get(&tot, nd1));
        JN_TRY(s.get(&start1[t], nd1 + 1));
        auto kh = k_chunk_hist<K, D1>;
        JN_TRY(launch(c, K_CHUNK_HIST, kh, dim3((unsigned)min(nch[t], (int64_t)4 * G)), dim3(512), sizeof(uint32_t) * nd1,
                      T[t]->key, n, chunk[t], d1, nd1, hist));
        JN_TRY(launch(c, K_CHUNK_HIST, k_chunk_scan, dim3((nd1 + 31) / 32), dim3(32, 32), 0, (const uint32_t*)hist, nch[t],
                      nd1, choff[t], tot));
        JN_TRY(scan_u64(c, tot, start1[t], nd1));
    }
    const bool keep = !RecomputeDigit<D1>::value;
    for (int t = 0; t < 2; t++) {
        JN_TRY(t == 0 ? wait_copies_r(c) : wait_copies(c, true));
        const int64_t n = T[t]->n;
        JN_TRY(s.get(&rows1[t], (size_t)n + HJ_PAD));
        auto k1 = k_region1_scatter<K, D1>;
        JN_TRY(launch(c, K_REGION1, k1, dim3((unsigned)min(nch[t], (int64_t)G)), dim3(RG_T),
                      Region1Smem<K>::bytes(keep), T[t]->key, T[t]->pay, n, chunk[t], d1, nd1,
                      (const uint32_t*)choff[t], (const uint64_t*)start1[t], rows1[t], c->d_err));
    }
    // level 2: the building table first, then the thinned one
    uint32_t* bitmap = nullptr;
    const int swords = fb - b1 >= 5 ? 1 << (fb - b1 - 5) : 1;
    if (filter) JN_TRY(s.get(&bitmap, (size_t)F1 * swords));
    for (int q = 0; q < 2; q++) {
        const int t = q == 0 ? first : 1 - first;
        const int64_t n = T[t]->n;
        RW* rows;
        uint32_t *pb, *pc;
        JN_TRY(s.get(&rows, (size_t)n + HJ_PAD));
        JN_TRY(s.get(&pb, (size_t)F1 * F2));
        JN_TRY(s.get(&pc, (size_t)F1 * F2));
        auto k2 = !filter ? k_region2<K, false, false> : q == 0 ? k_region2<K, true, false> : k_region2<K, false, true>;
        JN_TRY(launch(c, K_REGION2, k2, dim3((unsigned)min(F1, G)), dim3(RG_T), Region2Smem<K>::bytes(),
                      (const RW*)rows1[t], (uint64_t)n + HJ_PAD, (const uint64_t*)start1[t], F1, b1, b2, bitmap, fb,
                      rows, pb, pc, reinterpret_cast<unsigned long long*>(d_small + t), c->d_err));
        P[t]->rows = rows;
        P[t]->pbeg = pb;
        P[t]->pcnt = pc;
        if (hs) JN_TRY(group_heavy<K>(c, s, (const RW*)rows1[t], (uint64_t)n + HJ_PAD, start1[t] + F1, *hs, P[t]));
    }
    return JN_OK;
}

template <typename K>
jn_status run_hash(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int mode, OutPlan* plan,
                   RunResult* res, bool sort_merge) {
    using RW = Row<K, false>;
    const uint64_t nr = (uint64_t)R.n, ns = (uint64_t)S.n;
    jn_run_info& info = c->info;
    JN_TRY(wait_copies(c, false));  // key columns (payloads may still be on their way)
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
    // R rows per shared-memory table: the full table or half of it (a smaller
    // table doubles the partitions for the same rows per partition); a size
    // outside the key type's two is taken as the nearer one, so one context
    // serves both key types
    const int cap = tu.table_rows == 0 || tu.table_rows >= cap_of<K>() ? cap_of<K>() : cap_of<K>() / 2;
    bool heavy = tu.heavy >= 1 || (tu.heavy == -1 && nr + ns >= (1u << 20));
    const int64_t heavy_rows = tu.heavy >= 2 ? tu.heavy : cap_of<K>() / 4;  // rows that make a key heavy
    // which tables the pre-filter thins: bit 0 S (by R's keys), bit 1 R (by S's keys)
    int fside = 0;
    if (tu.prefilter == -1 && nr + ns >= (1u << 22))
        // with one table twice the other or larger, only the large one is
        // filtered: building the large table's bitmap costs more than thinning
        // the small table saves
        fside = 2 * nr <= ns ? 1 : 2 * ns <= nr ? 2 : 3;
    else if (tu.prefilter == 1)
        fside = 3;
    else if (tu.prefilter == 2)
        fside = 1;
    else if (tu.prefilter == 3)
        fside = 2;
    // partition path: regions (one level-1 pass, one block per region for the
    // second level, the filter built per region in shared memory) unless two
    // radix passes are asked for or the columns are read in place from host
    // memory.  The region path thins one table: the one the pre-filter names,
    // the larger one (S on a tie) when both are asked for.
    bool region = tu.hash_path != 1 && !R.host && !S.host;
    const int fside_rg = fside == 3 ? (ns >= nr ? 1 : 2) : fside;
    auto radix_bits_for = [&](int fs) {
        int bb = tu.radix_bits;
        if (bb == 0) {
            // expected R rows per partition: the table capacity when the filter
            // will thin R's rows out, half of it otherwise
            uint64_t target = (fs & 2) ? cap : cap / 2;
            bb = ceil_log2((nr + target - 1) / target);
            if (bb > 20) bb = 20;
        }
        return bb;
    };
    int b = radix_bits_for(region ? fside_rg : fside);
    int b1 = 0;
    if (region) {
        // 512 level-1 regions at most unless the second level would need more
        // than 8 bits: the level-1 scatter runs at 1.0 ms per 256M rows with
        // 512 digits and 1.4 ms with 1024 (GB300)
        b1 = tu.radix_bits1 ? tu.radix_bits1 : max(min(b, 9), b - 8);
        if (b1 > b) b1 = b;
        if (b1 > 10 || b - b1 > 8) region = false;  // beyond the region kernels' digit tables
        else fside = fside_rg;
        if (!region) b = radix_bits_for(fside);
    }
    if (!region) {
        b1 = tu.radix_bits1 ? tu.radix_bits1 : b / 2;
        if (b1 > b) b1 = b;
        const int b1max = heavy ? 9 : 10;  // pass 1 needs F1 (+1 heavy) <= 1024 digits
        if (b1 > b1max) b1 = b1max;
        if (b - b1 > 10) b1 = b - 10;
        if (b1 > b1max) return fail(c, JN_ERR_UNSUPPORTED, "radix bits too large for two passes");
    }
    const bool pre = !region && fside != 0;  // presence bitmaps of the two-pass path
    const int b2 = b - b1;
    const int F1 = 1 << b1, P = 1 << b;
    const int nd1 = F1 + (heavy ? 1 : 0);
    int fb = tu.filter_bits ? tu.filter_bits : ceil_log2(nr + ns) + 1;
    if (region) {
        // bitmap bits: the building table's key count, rounded up, in slices of
        // 2^5 .. 2^RG_SLICE_LOG bits per region
        const uint64_t nb = (fside & 1) ? nr : ns;
        if (tu.filter_bits == 0) fb = ceil_log2(nb) + 1;
        if (fb < b1 + 5) fb = b1 + 5;
        if (fb > b1 + RG_SLICE_LOG) fb = b1 + RG_SLICE_LOG;
        if (fb > 32) fb = 32;
    } else {
        if (fb < 10) fb = 10;
        if (fb > 28 && tu.filter_bits == 0) fb = 28;
    }
    const uint64_t fwords = pre ? (uint64_t(1) << fb) / 32 : 0;
    const uint32_t fmask = (uint32_t)((uint64_t(1) << fb) - 1);

    Scratch s(c);
    uint64_t* d_small;  // [0] R survivors, [1] S survivors, [2] items, [3] count, [4] checksum, [5] heavy
    JN_TRY(s.get(&d_small, 16));  // [8 ..] output offsets of emit slices
    JN_TRY(zero(c, d_small, 128));
    uint32_t *bmR = nullptr, *bmS = nullptr;
    unsigned long long *h1R, *h1S;
    JN_TRY(s.get(&h1R, nd1));
    JN_TRY(s.get(&h1S, nd1));
    if (!region) {
        JN_TRY(zero(c, h1R, sizeof(unsigned long long) * nd1));
        JN_TRY(zero(c, h1S, sizeof(unsigned long long) * nd1));
    }
    if (pre && (fside & 1)) {  // R's keys, filtering S
        JN_TRY(s.get(&bmR, fwords));
        JN_TRY(zero(c, bmR, fwords * 4));
    }
    if (pre && (fside & 2)) {  // S's keys, filtering R
        JN_TRY(s.get(&bmS, fwords));
        JN_TRY(zero(c, bmS, fwords * 4));
    }
    // ---- 0. heavy keys from a strided sample of both key columns ----
    HeavySet<K> hs{};
    int* d_hcount = nullptr;
    if (heavy) {
        K *tk, *hkeys, *htk;
        unsigned int* tc;
        int* htidx;
        const int slots = 1 << HV_SAMPLE_LOG;
        JN_TRY(s.get(&tk, slots));
        JN_TRY(s.get(&tc, 2 * slots));
        JN_TRY(s.get(&hkeys, HV_MAX));
        JN_TRY(s.get(&htk, HV_SLOTS));
        JN_TRY(s.get(&htidx, HV_SLOTS));
        JN_TRY(s.get(&d_hcount, 2));
        const int64_t target = 1 << 19;  // samples per table
        const int64_t sr = max((int64_t)1, (int64_t)nr / target), ss = max((int64_t)1, (int64_t)ns / target);
        // a key is heavy when about heavy_rows rows of one table carry it
        // (at least 8 sampled rows when sampling, so chance repeats do not qualify)
        const unsigned thr_r = (unsigned)max((int64_t)(sr > 1 ? 8 : 1), heavy_rows / sr);
        const unsigned thr_s = (unsigned)max((int64_t)(ss > 1 ? 8 : 1), heavy_rows / ss);
        const unsigned thr = thr_r < thr_s ? thr_r : thr_s;
        JN_TRY(launch(c, K_HEAVY_SAMPLE, k_sample_init<K>, dim3(256), dim3(256), 0, tk, tc, slots));
        JN_TRY(launch(c, K_HEAVY_SAMPLE, k_sample<K>, dim3(256), dim3(256), 0, R.key, R.n, sr, 0, tk, tc));
        JN_TRY(launch(c, K_HEAVY_SAMPLE, k_sample<K>, dim3(256), dim3(256), 0, S.key, S.n, ss, 1, tk, tc));
        unsigned int *chist, *d_thr;
        JN_TRY(s.get(&chist, HV_CBINS));
        JN_TRY(s.get(&d_thr, 1));
        JN_TRY(zero(c, chist, sizeof(unsigned int) * HV_CBINS));
        JN_TRY(zero(c, d_hcount, 2 * sizeof(int)));
        JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_hist<K>, dim3(c->num_sms), dim3(1024), 0, (const K*)tk,
                      (const unsigned int*)tc, thr, chist));
        JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_thr, dim3(1), dim3(32), 0, (const unsigned int*)chist, thr, d_thr));
        JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_collect<K>, dim3(2 * c->num_sms), dim3(256), 0, (const K*)tk,
                      (const unsigned int*)tc, (const unsigned int*)d_thr, hkeys, d_hcount));
        JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_table<K>, dim3(1), dim3(1024), 0, (const K*)hkeys, htk, htidx,
                      d_hcount));
        hs = HeavySet<K>{htk, htidx, hkeys, d_hcount};
        uint64_t hcw = 0;
        JN_TRY(read_back(c, reinterpret_cast<const uint64_t*>(d_hcount), &hcw, 1));
        if ((hcw & 0xffffffffu) == 0) {
            heavy = false;  // no frequent key: the plain path
        } else if (pre) {
            JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_bits<K>, dim3(1), dim3(1024), 0, hs, bmR, bmS, fmask));
        }
    }
    // ---- 1. presence bitmaps + first-pass histograms ----
    Partitioned<K> PR, PS;
    auto pass_all = [&](auto d1) -> jn_status {
        using D1 = decltype(d1);
        auto kp = k_presence_hist<K, D1>;
        const size_t smp = sizeof(uint32_t) * nd1;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kp, 512, smp);
        if (per < 1) per = 1;
        const int g = per * c->num_sms;
        JN_TRY(launch(c, K_PRESENCE, kp, dim3(g), dim3(512), smp, R.key, R.n, bmR, fmask, d1, nd1, h1R));
        JN_TRY(launch(c, K_PRESENCE, kp, dim3(g), dim3(512), smp, S.key, S.n, bmS, fmask, d1, nd1, h1S));
        // ---- 2-3. two partition passes per table (filtered by the other's bitmap) ----
        JN_TRY(wait_copies_r(c));
        JN_TRY((partition_table<K, D1>(c, s, R, b1, b2, d1, heavy ? &hs : nullptr, bmS, fmask, h1R, &PR,
                                       d_small + 0)));
        JN_TRY(wait_copies(c, true));
        JN_TRY((partition_table<K, D1>(c, s, S, b1, b2, d1, heavy ? &hs : nullptr, bmR, fmask, h1S, &PS,
                                       d_small + 1)));
        return JN_OK;
    };
    auto region_all = [&](auto d1) -> jn_status {
        return region_partition<K, decltype(d1)>(c, s, R, S, b1, b2, d1, heavy ? &hs : nullptr, fside != 0,
                                                 (fside & 1) ? 0 : 1, fb, &PR, &PS, d_small);
    };
    if (heavy) {
        HeavyHashDigit<K> d1{32 - b1, (uint32_t)(F1 - 1), (uint32_t)F1, hs, nullptr};
        JN_TRY(region ? region_all(d1) : pass_all(d1));
    } else {
        HashDigit d1{32 - b1, (uint32_t)(F1 - 1)};
        JN_TRY(region ? region_all(d1) : pass_all(d1));
    }
    // ---- 4. work items and the count pass ----
    uint64_t *items, *iprefix;
    JN_TRY(s.get(&items, P));
    JN_TRY(s.get(&iprefix, P + 1));
    JN_TRY(launch(c, K_ITEMS, k_items, dim3((P + 255) / 256), dim3(256), 0, PR.view(), PS.view(), P, cap,
                  items, (unsigned long long*)(d_small + 15)));
    JN_TRY(scan_u64(c, items, iprefix, P));
    uint64_t h[16];
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)(iprefix + P),
                  d_small + 2, 1));
    if (heavy) JN_CUDA(c, cudaMemcpyAsync(d_small + 7, d_hcount, 4, cudaMemcpyDeviceToDevice, c->stream));
    JN_TRY(read_back(c, d_small, h, 16));
    // many frequent keys in the sample: expect duplicate-heavy partitions too
    const bool skewed = heavy && (h[7] & 0xffffffffu) >= 64;
    const uint64_t nitems = h[2];
    info.r_survivors = h[0];
    info.s_survivors = h[1];
    info.partitions = (uint64_t)P;
    info.work_items = nitems;
    info.prefilter = fside == 3 ? 1 : fside == 1 ? 2 : fside == 2 ? 3 : 0;
    info.radix_bits = b;
    info.radix_bits1 = b1;
    info.filter_bits = fside ? fb : 0;
    info.hash_path = region ? 2 : 1;
    info.table_rows = (uint64_t)cap;
    info.heavy_keys = 0;
    // the join kernel stages rows with 16-byte bulk copies from these arrays
    if ((((uintptr_t)PR.rows) | ((uintptr_t)PS.rows)) & 15)
        return fail(c, JN_ERR_CUDA, "partition scratch is not 16-byte aligned");
    Item* idesc;
    unsigned long long *ival, *chk;
    uint64_t* ioff;
    JN_TRY(s.get(&idesc, nitems + 1));
    JN_TRY(s.get(&ival, nitems + 1));
    RW* rsorted = nullptr;  // sort-merge: the R chunks sorted by key
    JN_TRY(s.get(&ioff, nitems + 1));
    JN_TRY(s.get(&chk, 1));
    JN_TRY(zero(c, chk, 8));
    if (nitems) {
        JN_TRY(launch(c, K_ITEMS, k_item_desc, dim3((unsigned)ceil_div(nitems, 256)), dim3(256), 0, PR.view(),
                      PS.view(), (const uint64_t*)iprefix, P, cap, idesc));
        const int cm = mode == MODE_AGG ? MODE_AGG : MODE_COUNT;
        if (sort_merge) {
            // every R chunk sorted by key once, into a copy the count and emit passes read
            JN_TRY(s.get(&rsorted, (size_t)R.n + HJ_PAD));
            auto kso = k_sort_chunks<K>;
            const size_t sms = SortJoinSmem<K>::sort_bytes(cap);
            const int gs = (int)min((uint64_t)persistent_grid(c, (const void*)kso, SJ_T, sms), nitems);
            JN_TRY(launch(c, K_SORT_CHUNKS, kso, dim3(gs), dim3(SJ_T), sms, (const RW*)PR.rows, rsorted,
                          (const Item*)idesc, (const uint64_t*)(iprefix + P), cap));
            auto kc = cm == MODE_AGG ? k_sort_join<K, MODE_AGG> : k_sort_join<K, MODE_COUNT>;
            const size_t smc = SortJoinSmem<K>::bytes(cap, cm);
            const int gj = (int)min((uint64_t)persistent_grid(c, (const void*)kc, SJ_T, smc), nitems);
            JN_TRY(launch(c, K_SORT_COUNT, kc, dim3(gj), dim3(SJ_T), smc, (const RW*)rsorted, (const RW*)PS.rows,
                          (const Item*)idesc, (const uint64_t*)(iprefix + P), cap, ival, chk,
                          (const uint64_t*)nullptr, (jn_pair*)nullptr, (uint64_t)0, ~0ull));
        } else {
            const size_t smc = hash_smem<K>(cm, cap);
            auto kc = cm == MODE_AGG ? hash_join_kernel<K, MODE_AGG>(skewed, cap)
                                     : hash_join_kernel<K, MODE_COUNT>(skewed, cap);
            const int gj = (int)min((uint64_t)persistent_grid(c, (const void*)kc, HJ_T, smc), nitems);
            JN_TRY(launch(c, K_HASH_COUNT, kc, dim3(gj), dim3(HJ_T), smc, (const RW*)PR.rows, (const RW*)PS.rows,
                          (const Item*)idesc, (const uint64_t*)(iprefix + P), b, ival, chk,
                          (const uint64_t*)nullptr, (jn_pair*)nullptr, c->d_err, (uint64_t)0, ~0ull));
        }
    }
    JN_TRY(scan_u64(c, reinterpret_cast<const uint64_t*>(ival), ioff, (int64_t)nitems));
    // ---- heavy keys: c_R(h) * c_S(h) pairs each ----
    uint64_t *hp = nullptr, *hpoff = nullptr, *hch = nullptr, *hchp = nullptr;
    if (heavy) {
        JN_TRY(s.get(&hp, HV_MAX));
        JN_TRY(s.get(&hpoff, HV_MAX + 1));
        JN_TRY(s.get(&hch, HV_MAX));
        JN_TRY(s.get(&hchp, HV_MAX + 1));
        unsigned long long *fsum, *gsum;
        JN_TRY(s.get(&fsum, HV_MAX));
        JN_TRY(s.get(&gsum, HV_MAX));
        JN_TRY(zero(c, fsum, 8 * HV_MAX));
        JN_TRY(zero(c, gsum, 8 * HV_MAX));
        JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_pairs<RW>, dim3(mode == MODE_AGG ? 64 : 1, HV_MAX), dim3(256), 0,
                      (const RW*)PR.hrows, (const uint64_t*)PR.hoff, (const RW*)PS.hrows, (const uint64_t*)PS.hoff,
                      (const int*)d_hcount, hp, hch, fsum, gsum, mode == MODE_AGG ? 1 : 0, (uint64_t)CE_PAIRS));
        if (mode == MODE_AGG)
            JN_TRY(launch(c, K_HEAVY_SELECT, k_heavy_chk, dim3(1), dim3(1024), 0, (const unsigned long long*)fsum,
                          (const unsigned long long*)gsum, chk));
        JN_TRY(scan_u64(c, hp, hpoff, HV_MAX));
        JN_TRY(scan_u64(c, hch, hchp, HV_MAX));
        JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)(hpoff + HV_MAX),
                      d_small + 5, 1));
        JN_CUDA(c, cudaMemcpyAsync(d_small + 6, d_hcount, 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)(ioff + nitems),
                  d_small + 3, 1));
    JN_TRY(launch(c, K_MISC, k_copy_words, dim3(1), dim3(32), 0, (const uint64_t*)chk, d_small + 4, 1));
    uint64_t hc[4];
    JN_TRY(read_back(c, d_small + 3, hc, 4));
    const uint64_t normal = hc[0], heavy_pairs = heavy ? hc[2] : 0;
    const uint64_t total = normal + heavy_pairs;
    res->count = total;
    res->checksum = hc[1];
    info.result = total;
    info.heavy_keys = heavy ? (hc[3] & 0xffffffffu) : 0;
    info.heavy_pairs = heavy_pairs;
    info.cartesian_bound = h[15] + heavy_pairs;  // the frequent keys' cross products are exact
    if (mode != MODE_EMIT) return JN_OK;
    // ---- 5. exact allocation and the emit pass ----
    JN_TRY(out_prepare(c, s, total, *plan));
    // A host output is copied back slice by slice (on the copy stream) while
    // the later slices of the work queue emit: slice k's pairs are the
    // contiguous range [ioff[ib[k]], ioff[ib[k + 1]]).
    const int nsl = (plan->host_copy && normal >= (uint64_t)JN_SLICE_PAIRS && nitems >= 64) ? 4 : 1;
    uint64_t ib[5], ob[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k <= nsl; k++) ib[k] = nitems * (uint64_t)k / (uint64_t)nsl;
    if (nsl > 1) {
        for (int k = 0; k <= nsl; k++)
            JN_CUDA(c, cudaMemcpyAsync(d_small + 8 + k, ioff + ib[k], 8, cudaMemcpyDeviceToDevice, c->stream));
        JN_TRY(read_back(c, d_small + 8, ob, nsl + 1));
        if (!c->copy_stream) JN_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    }
    auto copy_back = [&](uint64_t lo, uint64_t hi) -> jn_status {  // pairs [lo, hi) to the caller's buffer
        if (hi <= lo) return JN_OK;
        cudaEvent_t e;
        JN_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, c->stream);
        cudaStreamWaitEvent(c->copy_stream, e, 0);
        cudaEventDestroy(e);
        JN_CUDA(c, cudaMemcpyAsync(*plan->user_out + lo, plan->dev + lo, (hi - lo) * sizeof(jn_pair),
                                   cudaMemcpyDefault, c->copy_stream));
        return JN_OK;
    };
    if (normal > 0) {
        auto ke = hash_join_kernel<K, MODE_EMIT>(skewed, cap);
        auto kse = k_sort_join<K, MODE_EMIT>;
        const size_t sme = sort_merge ? SortJoinSmem<K>::bytes(cap, MODE_EMIT) : hash_smem<K>(MODE_EMIT, cap);
        const uint64_t pg = sort_merge ? (uint64_t)persistent_grid(c, (const void*)kse, SJ_T, sme)
                                       : (uint64_t)persistent_grid(c, (const void*)ke, HJ_T, sme);
        for (int k = 0; k < nsl; k++) {
            if (ib[k + 1] == ib[k]) continue;
            const int ge = (int)min(pg, ib[k + 1] - ib[k]);
            if (sort_merge)
                JN_TRY(launch(c, K_SORT_EMIT, kse, dim3(ge), dim3(SJ_T), sme, (const RW*)rsorted,
                              (const RW*)PS.rows, (const Item*)idesc, (const uint64_t*)(iprefix + P), cap,
                              (unsigned long long*)nullptr, (unsigned long long*)nullptr, (const uint64_t*)ioff,
                              plan->dev, ib[k], ib[k + 1]));
            else
                JN_TRY(launch(c, K_HASH_EMIT, ke, dim3(ge), dim3(HJ_T), sme, (const RW*)PR.rows,
                              (const RW*)PS.rows, (const Item*)idesc, (const uint64_t*)(iprefix + P), b,
                              (unsigned long long*)nullptr, (unsigned long long*)nullptr, (const uint64_t*)ioff,
                              plan->dev, c->d_err, ib[k], ib[k + 1]));
            if (nsl > 1) JN_TRY(copy_back(ob[k], ob[k + 1]));
        }
    }
    if (heavy_pairs > 0) {
        JN_TRY(launch(c, K_CROSS_EMIT, k_cartesian<RW>, dim3(8 * c->num_sms), dim3(256), 0, (const RW*)PR.hrows,
                      (const uint64_t*)PR.hoff, (const RW*)PS.hrows, (const uint64_t*)PS.hoff,
                      (const uint64_t*)hpoff, (const uint64_t*)hchp, HV_MAX, (uint64_t)CE_PAIRS, normal,
                      plan->dev));
    }
    if (nsl > 1) {
        JN_TRY(copy_back(normal, total));
        cudaEvent_t e;  // the run ends when its last copy has landed
        JN_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, c->copy_stream);
        cudaStreamWaitEvent(c->stream, e, 0);
        cudaEventDestroy(e);
        plan->copied = true;
    }
    JN_TRY(out_finish(c, total, *plan));
    return JN_OK;
}

// ------------------------------------------------------------------ batch --
// Histogram of per-segment digits over a tile list: hist[seg * 1024 + d].
template <typename K>
__global__ void __launch_bounds__(SC_T)
k_batch_hist(const SegCols<K>* __restrict__ segs, const TileRef* __restrict__ tiles,
             const uint64_t* __restrict__ ntiles_p, SegHashDigit dg, unsigned long long* __restrict__ hist) {
    __shared__ uint32_t s_h[SC_FMAX];
    const uint64_t ntiles = *ntiles_p;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileRef x = tiles[t];
        dg.set_seg(x.seg);
        const int nd = 1 << dg.b;
        for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
        __syncthreads();
        const K* k = segs[x.seg].key;
        for (int i = threadIdx.x; i < x.cnt; i += blockDim.x) atomicAdd(&s_h[dg(k[x.beg + i])], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < nd; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(uint64_t)x.seg * SC_FMAX + i], (unsigned long long)s_h[i]);
        __syncthreads();
    }
}

// out_off[i] = output offset of join i: the offset of its first item.
__global__ void k_batch_offsets(const uint64_t* __restrict__ item_prefix, const uint64_t* __restrict__ ioff,
                                int count, uint64_t* __restrict__ out_off) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > count) return;
    out_off[i] = ioff[item_prefix[(uint64_t)i * SC_FMAX]];
}

// A batch of equi-joins run as one: every table of every join is a segment
// of one radix pass (segment i = R of join i, segment n + i = S of join i),
// partition (i, d) has the global id i * 1024 + d, and the count and emit
// passes run over one work queue of (partition, R chunk) items of all joins.
// Each phase is one launch for the whole batch; with graphs on, the phases up
// to the count read-back and the emit phase are each replayed as a CUDA graph.
template <typename K>
struct HashBatchRun : BatchRun {
    using RW = Row<K, false>;
    std::unique_ptr<Scratch> s;
    int n = 0;
    uint64_t P = 0, item_bound = 0;
    RW* prow = nullptr;
    Item* idesc = nullptr;
    uint64_t *iprefix = nullptr, *ioff = nullptr;

    jn_status prepare(jn_ctx* c, const Cols<K>* Rs, const Cols<K>* Ss) {
        const int cap = cap_of<K>();
        s.reset(new Scratch(c));
        // ---- host plan: per-join fan-out, segment table and tile list ----
        std::vector<SegCols<K>> segs(2 * (size_t)n);
        std::vector<int> bits(2 * (size_t)n);
        std::vector<TileRef> tiles;
        uint64_t rows = 0, rrows = 0;
        const uint64_t part_rows = c->tune.part_rows > 0 ? (uint64_t)c->tune.part_rows : (uint64_t)cap / 2;
        for (int i = 0; i < n; i++) {
            int b = ceil_log2(ceil_div((uint64_t)Rs[i].n, part_rows));
            if (b > 10) b = 10;
            bits[i] = bits[n + i] = b;
            segs[i] = SegCols<K>{Rs[i].key, nullptr, Rs[i].pay, (uint64_t)Rs[i].n};
            segs[n + i] = SegCols<K>{Ss[i].key, nullptr, Ss[i].pay, (uint64_t)Ss[i].n};
            rows += (uint64_t)Rs[i].n + (uint64_t)Ss[i].n;
            rrows += (uint64_t)Rs[i].n;
        }
        for (int sgi = 0; sgi < 2 * n; sgi++)
            for (uint64_t b = 0; b < segs[sgi].n; b += SC_TILE)
                tiles.push_back(TileRef{b, sgi, (int)min((uint64_t)SC_TILE, segs[sgi].n - b)});
        const uint64_t ntiles = tiles.size();
        P = (uint64_t)n * SC_FMAX;
        item_bound = P + rrows / (uint64_t)cap + 1;  // items <= P + sum nr / cap
        SegCols<K>* d_segs;
        int* d_bits;
        TileRef* d_tiles;
        uint64_t *d_ntiles, *start, *items, *d_off;
        unsigned long long *hist, *cur, *ival, *chk;
        JN_TRY(s->get(&d_segs, 2 * (size_t)n));
        JN_TRY(s->get(&d_bits, 2 * (size_t)n));
        JN_TRY(s->get(&d_tiles, ntiles + 1));
        JN_TRY(s->get(&d_ntiles, 1));
        JN_TRY(s->get(&hist, 2 * P));
        JN_TRY(s->get(&start, 2 * P + 1));
        JN_TRY(s->get(&cur, 2 * P));
        JN_TRY(s->get(&prow, rows + HJ_PAD));
        JN_TRY(s->get(&items, P));
        JN_TRY(s->get(&iprefix, P + 1));
        JN_TRY(s->get(&idesc, item_bound));
        JN_TRY(s->get(&ival, item_bound));
        JN_TRY(s->get(&ioff, item_bound + 1));
        JN_TRY(s->get(&chk, 1));
        JN_TRY(s->get(&d_off, (size_t)n + 1));
        JN_CUDA(c, cudaMemcpyAsync(d_segs, segs.data(), sizeof(SegCols<K>) * segs.size(), cudaMemcpyHostToDevice,
                                   c->stream));
        JN_CUDA(c, cudaMemcpyAsync(d_bits, bits.data(), sizeof(int) * bits.size(), cudaMemcpyHostToDevice,
                                   c->stream));
        if (ntiles)
            JN_CUDA(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TileRef) * ntiles, cudaMemcpyHostToDevice,
                                       c->stream));
        JN_CUDA(c, cudaMemcpyAsync(d_ntiles, &ntiles, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream));
        JN_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vectors go out of scope below

        GraphPhase gp(c, c->tune.graphs != 0 && !c->profiling);
        JN_TRY(gp.begin());
        jn_status st = JN_OK;
        do {
            SegHashDigit dg{d_bits, 0};
            if ((st = zero(c, hist, sizeof(unsigned long long) * 2 * P)) != JN_OK) break;
            if ((st = zero(c, chk, 8)) != JN_OK) break;
            if ((st = zero(c, ival, sizeof(unsigned long long) * item_bound)) != JN_OK) break;
            if ((st = launch(c, K_HIST, k_batch_hist<K>, dim3(4 * c->num_sms), dim3(SC_T), 0,
                             (const SegCols<K>*)d_segs, (const TileRef*)d_tiles, (const uint64_t*)d_ntiles, dg,
                             hist)) != JN_OK)
                break;
            if ((st = scan_u64(c, reinterpret_cast<const uint64_t*>(hist), start, (int64_t)(2 * P))) != JN_OK) break;
            if ((st = launch(c, K_MISC, k_init_cursor, dim3((unsigned)ceil_div(2 * P, 256)), dim3(256), 0,
                             (const uint64_t*)start, cur, (int64_t)(2 * P))) != JN_OK)
                break;
            auto ks = k_scatter<K, false, false, SegHashDigit>;
            const size_t sm = scatter_smem<K, false>();
            PartIn<K, false> in{nullptr, nullptr, nullptr, nullptr, 0, d_segs, d_tiles};
            if ((st = launch(c, K_SCATTER, ks, dim3(persistent_grid(c, (const void*)ks, SC_T, sm)), dim3(SC_T), sm,
                             in, (const uint64_t*)nullptr, (const uint64_t*)nullptr, (const uint64_t*)d_ntiles, 0,
                             dg, SC_FMAX, (const uint32_t*)nullptr, 0u, cur, prow, c->d_err)) != JN_OK)
                break;
            const uint64_t* roff = start;
            const uint64_t* soff = start + P;
            if ((st = launch(c, K_ITEMS, k_items, dim3((unsigned)ceil_div(P, 256)), dim3(256), 0,
                             PartView{roff, nullptr, nullptr}, PartView{soff, nullptr, nullptr}, (int)P, cap, items,
                             (unsigned long long*)nullptr)) != JN_OK)
                break;
            if ((st = scan_u64(c, items, iprefix, (int64_t)P)) != JN_OK) break;
            if ((st = launch(c, K_ITEMS, k_item_desc, dim3((unsigned)ceil_div(item_bound, 256)), dim3(256), 0,
                             PartView{roff, nullptr, nullptr}, PartView{soff, nullptr, nullptr},
                             (const uint64_t*)iprefix, (int)P, cap, idesc)) != JN_OK)
                break;
            auto kc = k_hash_join<K, MODE_COUNT, false>;
            const size_t smc = hash_smem<K>(MODE_COUNT);
            if ((st = launch(c, K_HASH_COUNT, kc, dim3(persistent_grid(c, (const void*)kc, HJ_T, smc)), dim3(HJ_T),
                             smc, (const RW*)prow, (const RW*)prow, (const Item*)idesc,
                             (const uint64_t*)(iprefix + P), 10, ival, chk, (const uint64_t*)nullptr,
                             (jn_pair*)nullptr, c->d_err, (uint64_t)0, ~0ull)) != JN_OK)
                break;
            // items past the real count keep zero counts: scan the whole bound
            if ((st = scan_u64(c, reinterpret_cast<const uint64_t*>(ival), ioff, (int64_t)item_bound)) != JN_OK) break;
            if ((st = launch(c, K_MISC, k_batch_offsets, dim3((unsigned)ceil_div((uint64_t)n + 1, 256)), dim3(256), 0,
                             (const uint64_t*)iprefix, (const uint64_t*)ioff, n, d_off)) != JN_OK)
                break;
        } while (0);
        if (st != JN_OK) {
            gp.abort();
            return st;
        }
        JN_TRY(gp.end_and_run());
        offsets.assign((size_t)n + 1, 0);
        JN_CUDA(c, cudaMemcpyAsync(offsets.data(), d_off, sizeof(uint64_t) * (n + 1), cudaMemcpyDeviceToHost,
                                   c->stream));
        uint64_t dummy;
        JN_TRY(read_back(c, d_off, &dummy, 0));
        total = offsets[n];
        return JN_OK;
    }

    jn_status emit(jn_ctx* c, jn_pair* out) override {
        if (total == 0) return JN_OK;
        GraphPhase gp(c, c->tune.graphs != 0 && !c->profiling);
        JN_TRY(gp.begin());
        auto ke = k_hash_join<K, MODE_EMIT>;
        const size_t sme = hash_smem<K>(MODE_EMIT);
        jn_status st = launch(c, K_HASH_EMIT, ke, dim3(persistent_grid(c, (const void*)ke, HJ_T, sme)), dim3(HJ_T),
                              sme, (const RW*)prow, (const RW*)prow, (const Item*)idesc, (const uint64_t*)(iprefix + P),
                              10, (unsigned long long*)nullptr, (unsigned long long*)nullptr, (const uint64_t*)ioff,
                              out, c->d_err, (uint64_t)0, ~0ull);
        if (st != JN_OK) {
            gp.abort();
            return st;
        }
        JN_TRY(gp.end_and_run());
        return JN_OK;
    }
};

template <typename K>
jn_status batch_hash_prepare(jn_ctx* c, int n, const Cols<K>* Rs, const Cols<K>* Ss, std::unique_ptr<BatchRun>* run) {
    std::unique_ptr<HashBatchRun<K>> r(new HashBatchRun<K>());
    r->n = n;
    JN_TRY(r->prepare(c, Rs, Ss));
    c->info.partitions += r->P;
    c->info.work_items += r->item_bound;
    run->reset(r.release());
    return JN_OK;
}

template jn_status batch_hash_prepare<int32_t>(jn_ctx*, int, const Cols<int32_t>*, const Cols<int32_t>*,
                                               std::unique_ptr<BatchRun>*);
template jn_status batch_hash_prepare<int64_t>(jn_ctx*, int, const Cols<int64_t>*, const Cols<int64_t>*,
                                               std::unique_ptr<BatchRun>*);

int hash_cap(int32_t key_type) { return key_type == JN_KEY_I32 ? cap_of<int32_t>() : cap_of<int64_t>(); }

template jn_status run_hash<int32_t>(jn_ctx*, const Cols<int32_t>&, const Cols<int32_t>&, int,
                                     OutPlan*, RunResult*, bool);
template jn_status run_hash<int64_t>(jn_ctx*, const Cols<int64_t>&, const Cols<int64_t>&, int,
                                     OutPlan*, RunResult*, bool);

}  // namespace jnx
