// Two-level radix partitioning of the equi hash join, built for one GPU
// with no global atomics on the data path: the shuffle of Algorithm 1 (rows
// regrouped by a function of the join key, Sec. 3.1) split into the two
// levels of the Reducer hierarchy (Eq. 9, Sec. 3.3.4).
//
// Level 1 (regions).  The key column is cut into chunks.  k_chunk_hist
// counts every chunk's first-level digits; k_chunk_scan turns the counts into
// the output position of every (chunk, digit) run; k_region1_scatter streams
// each chunk through shared memory (TMA bulk copies, two stages), orders a
// tile's rows by digit and writes them to those positions.  Output: rows
// (key, payload) grouped by digit ("regions").  Rows rather than two columns,
// because a tile holds only a few rows of each digit and a 4-byte column run
// of that length leaves partly written 32-byte sectors that cost DRAM
// read-modify-writes (measured on GB300: 2.7 ms against 1.5 ms per 256M rows
// at 1024 digits).
//
// Level 2 (partitions).  k_region2 gives every region to one block.  The
// block counts the region's second-level digits, then moves its rows into
// (region, digit) partitions stored as rows (key, payload) -- the layout the
// join kernels stage.  Holding a whole region lets the block keep the
// key-presence filter of Algorithm 1 for that region in shared memory: the
// first table's block sets a bit per key in its region's slice of the bitmap
// (BUILD) and writes the slice out; the second table's block loads the slice
// and drops every row whose bit is clear (FILTER).  No bitmap bit is set with
// a global atomic.
//
// The bitmap is indexed by the top `fb` bits of the key hash, so region i
// (the top b1 bits) owns the contiguous slice [i << (fb - b1), (i + 1) <<
// (fb - b1)).  A bit shared by two keys only weakens the filter; the join
// compares keys, so the result never depends on it.
#pragma once

#include "jn_async.cuh"
#include "jn_heavy.cuh"
#include "jn_partition.cuh"

namespace jnx {

constexpr int RG_T = 512;               // threads of the region kernels (16 rows each per int32 tile)
constexpr int RG_STAGE = 65536 + 64;    // bytes per staging buffer (a tile and its 16-byte widening)
constexpr int RG_NDMAX = 1026;          // level-1 digits at most (1024 + the heavy digit, even)
constexpr int RG_F2MAX = 256;           // level-2 digits at most
constexpr int RG_SLICE_LOG = 19;        // bitmap bits per region at most (2^19 bits = 64 KB)

// Tile shapes: a staged tile fills one 64 KB stage.
template <typename K>
struct RgShape {
    using RW = Row<K, false>;
    static constexpr int T1 = sizeof(K) == 4 ? 8192 : 4096;   // level-1 rows per tile (key + payload columns)
    static constexpr int T2 = 65536 / (int)sizeof(RW);        // level-2 rows per tile (staged rows)
    static constexpr int KB = T1 * (int)sizeof(K) + 32;      // staged keys of a level-1 tile
    static_assert(KB + T1 * 4 + 32 <= RG_STAGE, "level-1 tile fits a stage");
    static_assert(T1 * (int)sizeof(RW) <= RG_STAGE, "level-1 tile rows fit a stage");
    static_assert(T2 * (int)sizeof(RW) + 32 <= RG_STAGE, "level-2 tile fits a stage");
    static_assert(T1 % (4 * RG_T) == 0 && T2 % RG_T == 0, "whole rows per thread");
};

// Digit functors whose digit is cheap to recompute from the key (HashDigit)
// are recomputed at write-out; the others (a heavy-key lookup) are kept in
// shared memory next to the row.
template <typename D>
struct RecomputeDigit {
    static constexpr bool value = false;
};
template <>
struct RecomputeDigit<HashDigit> {
    static constexpr bool value = true;
};

template <typename K>
struct Region1Smem {
    __host__ __device__ static constexpr size_t bytes(bool keep_digit) {
        return 2 * (size_t)RG_STAGE + (keep_digit ? (size_t)RgShape<K>::T1 * 2 : 0) + 4 * (size_t)RG_NDMAX * 4;
    }
};

// ----------------------------------------------------------- level 1 --

// Chunk c covers rows [c * chunk, min(n, (c + 1) * chunk)).
// hist[c * nd + d] = rows of chunk c whose digit is d.
template <typename K, typename Digit>
__global__ void __launch_bounds__(512)
k_chunk_hist(const K* __restrict__ keys, int64_t n, int64_t chunk, Digit dg0, int nd, uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t s_h[];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);
    constexpr int V = 16 / (int)sizeof(K);
    const int64_t nch = (n + chunk - 1) / chunk;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
        __syncthreads();
        const int64_t b = c * chunk;
        const int64_t cnt = min(n - b, chunk);
        const K* p = keys + b;
        // scalar head up to a 16-byte boundary, vector body, scalar tail
        int64_t head = (int64_t)(((16 - ((uintptr_t)p & 15)) & 15) / sizeof(K));
        if (head > cnt) head = cnt;
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x) atomicAdd(&s_h[dg(p[i])], 1u);
        const int64_t nv = (cnt - head) / V;
        const int4* pv = reinterpret_cast<const int4*>(p + head);
        for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) {
            const int4 q = __ldcs(pv + i);
            const K* kv = reinterpret_cast<const K*>(&q);
#pragma unroll
            for (int j = 0; j < V; j++) atomicAdd(&s_h[dg(kv[j])], 1u);
        }
        for (int64_t i = head + nv * V + threadIdx.x; i < cnt; i += blockDim.x) atomicAdd(&s_h[dg(p[i])], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < nd; i += blockDim.x) hist[c * nd + i] = s_h[i];
        __syncthreads();
    }
}

// Column scans of the chunk histograms: off[c * nd + d] = sum over c' < c of
// hist[c' * nd + d] (the run of chunk c inside digit d's region), tot[d] = the
// digit's rows.  Block (32, 32): x = digit in a group of 32, y = slice of the
// chunks; each slice is summed, the 32 slice sums are scanned in shared
// memory, then each slice writes its prefixes.
__global__ void __launch_bounds__(1024)
k_chunk_scan(const uint32_t* __restrict__ hist, int64_t nch, int nd, uint32_t* __restrict__ off,
             uint64_t* __restrict__ tot) {
    __shared__ uint32_t s_part[32][33];
    const int d = blockIdx.x * 32 + threadIdx.x;
    const int64_t per = (nch + 31) / 32;
    const int64_t c0 = threadIdx.y * per, c1 = min(nch, c0 + per);
    uint32_t sum = 0;
    if (d < nd)
        for (int64_t c = c0; c < c1; c++) sum += hist[c * nd + d];
    s_part[threadIdx.y][threadIdx.x] = sum;
    __syncthreads();
    uint32_t pre = 0;
    for (int y = 0; y < (int)threadIdx.y; y++) pre += s_part[y][threadIdx.x];
    if (d < nd) {
        for (int64_t c = c0; c < c1; c++) {
            const uint32_t v = hist[c * nd + d];
            off[c * nd + d] = pre;
            pre += v;
        }
        if (threadIdx.y == 31) tot[d] = pre;
    }
}

// Row `i` of a staged column, or of the column itself when the tile was not
// staged (an unaligned base, or a widened span past the column's end).
struct StageTile {
    long long beg;
    int cnt;    // rows; -1 = no tile
    int tma;    // staged by a bulk copy
    int koff;   // element offset of row `beg` in the staged keys
    int poff;   // element offset of row `beg` in the staged payloads
};

// Starts the bulk copies of rows [beg, beg + cnt) of (key, pay) into `stage`
// (keys at 0, payloads at `kbytes`); thread 0 only.
template <typename K>
__device__ __forceinline__ void stage_columns(StageTile* t, const K* key, const int32_t* pay, uint64_t rows_ok,
                                              unsigned char* stage, int kbytes, uint64_t* bar) {
    t->tma = 0;
    uint64_t bk = 0, bp = 0;
    uint32_t nk = 0, np = 0;
    bool ok = byte_span(key, t->beg, t->cnt, sizeof(K), rows_ok, &bk, &nk) && nk <= (uint32_t)kbytes;
    if (ok && pay) ok = byte_span(pay, t->beg, t->cnt, 4, rows_ok, &bp, &np) && kbytes + np <= (uint32_t)RG_STAGE;
    if (!ok) return;
    t->tma = 1;
    t->koff = (int)(t->beg - (long long)(bk / sizeof(K)));
    t->poff = pay ? (int)(t->beg - (long long)(bp / 4)) : 0;
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, nk + np);
    tma_load_1d(stage, reinterpret_cast<const unsigned char*>(key) + bk, nk, bar);
    if (pay) tma_load_1d(stage + kbytes, reinterpret_cast<const unsigned char*>(pay) + bp, np, bar);
}

// Exclusive scan of cnt[0 .. nd) (nd <= RG_NDMAX) by the block, RG_DPT
// consecutive digits per thread: fills start[], sets base[d] = cur[d] -
// start[d] (modulo 2^32) and advances cur[d] by cnt[d]; clears cnt[];
// *total (when given) receives the sum.  Ends with a barrier.
constexpr int RG_DPT = (RG_NDMAX + RG_T - 1) / RG_T;
__device__ __forceinline__ void rg_scan_digits(uint32_t* cnt, uint32_t* start, uint32_t* base, uint32_t* cur, int nd,
                                               uint32_t* s_wsum, uint32_t* total = nullptr) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t c[RG_DPT];
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < RG_DPT; q++) {
        const int d = t * RG_DPT + q;
        c[q] = d < nd ? cnt[d] : 0u;
        v += c[q];
    }
    const uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    const uint32_t ws = lane < RG_T / 32 ? s_wsum[lane] : 0u;
    const uint32_t wi = warp_incl_scan(ws);
    uint32_t pre = __shfl_sync(0xffffffffu, wi - ws, warp) + inc - v;
#pragma unroll
    for (int q = 0; q < RG_DPT; q++) {
        const int d = t * RG_DPT + q;
        if (d < nd) {
            const uint32_t cu = cur[d];
            start[d] = pre;
            base[d] = cu - pre;
            cur[d] = cu + c[q];
            cnt[d] = 0;
        }
        pre += c[q];
    }
    if (total && t == RG_T - 1) *total = pre;
    __syncthreads();
}

// Level-1 scatter.  Block b takes chunks b, b + grid, ...; the rows of chunk
// c with digit d go to out[dstart[d] + off[c * nd + d] ...] in input order of
// tiles.  Tiles are staged by TMA into two stages: a tile is read into
// registers, its stage is reused to order the tile by digit, and once every
// thread has written its rows out (the next tile's first barrier) the stage
// receives the tile after next.
template <typename K, typename Digit>
__global__ void __launch_bounds__(RG_T, 1)
k_region1_scatter(const K* __restrict__ key, const int32_t* __restrict__ pay, int64_t n, int64_t chunk, Digit dg0,
                  int nd, const uint32_t* __restrict__ choff, const uint64_t* __restrict__ dstart,
                  Row<K, false>* __restrict__ out, unsigned int* __restrict__ err) {
    using S = RgShape<K>;
    using RW = Row<K, false>;
    constexpr int T = S::T1, IPT = T / RG_T;
    constexpr bool KEEP = !RecomputeDigit<Digit>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage0 = smem;
    uint16_t* s_d = reinterpret_cast<uint16_t*>(smem + 2 * (size_t)RG_STAGE);  // digits (KEEP only)
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + 2 * (size_t)RG_STAGE + (KEEP ? (size_t)T * 2 : 0));
    uint32_t* s_ts = s_cnt + RG_NDMAX;
    uint32_t* s_gb = s_ts + RG_NDMAX;
    uint32_t* s_cur = s_gb + RG_NDMAX;
    __shared__ uint32_t s_wsum[32];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ StageTile tile[2];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);
    const int tid = threadIdx.x;
    const int64_t nch = (n + chunk - 1) / chunk;
    for (int i = tid; i < RG_NDMAX; i += RG_T) s_cnt[i] = 0;
    // producer (thread 0): the next tile to stage
    int64_t pc = blockIdx.x, pt = 0;
    auto issue = [&](int s) {
        StageTile x;
        x.cnt = -1;
        x.tma = 0;
        x.beg = 0;
        if (pc < nch) {
            const int64_t cb = pc * chunk, ce = min(n, cb + chunk);
            x.beg = (long long)(cb + pt * T);
            x.cnt = (int)min((int64_t)T, ce - (int64_t)x.beg);
            stage_columns<K>(&x, key, pay, (uint64_t)n, stage0 + (size_t)s * RG_STAGE, S::KB, &bar[s]);
            if (x.beg + T >= ce) {
                pc += gridDim.x;
                pt = 0;
            } else {
                pt++;
            }
        }
        tile[s] = x;
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(0);
        issue(1);
    }
    __syncthreads();
    int64_t held = -1;  // chunk whose cursors are in s_cur
    uint32_t ph0 = 0, ph1 = 0;
    bool refill = false;  // the other stage is free and waits for the tile after next
    for (int s = 0;; s ^= 1) {
        const StageTile x = tile[s];
        if (x.cnt < 0) break;
        const int64_t c = x.beg / chunk;
        if (c != held) {
            for (int i = tid; i < nd; i += RG_T) s_cur[i] = (uint32_t)(dstart[i] + choff[c * nd + i]);
            held = c;
        }
        unsigned char* st = stage0 + (size_t)s * RG_STAGE;
        bool ok = true;
        if (x.tma) ok = mbar_wait(&bar[s], s ? ph1 : ph0, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {  // let the copies in flight land before leaving
                if (x.tma) mbar_wait(&bar[s], s ? ph1 : ph0, nullptr);
                if (!refill && tile[s ^ 1].cnt >= 0 && tile[s ^ 1].tma) mbar_wait(&bar[s ^ 1], s ? ph0 : ph1, nullptr);
            }
            break;
        }
        // every thread is past the previous tile's write-out: its stage is free
        if (refill && tid == 0) issue(s ^ 1);
        refill = true;
        if (x.tma) {
            if (s) ph1 ^= 1u; else ph0 ^= 1u;
        }
        const K* gk = reinterpret_cast<const K*>(st);
        const int32_t* gp = reinterpret_cast<const int32_t*>(st + S::KB);
        K kv[IPT];
        int32_t pv[IPT];
        uint32_t dv[IPT], rv[IPT];
        if (x.tma && x.koff == 0 && (!pay || x.poff == 0)) {
            // aligned tile: thread t holds rows 4 (t + RG_T q) .. + 3, read as 16-byte vectors
#pragma unroll
            for (int q = 0; q < IPT / 4; q++) {
                const int r0 = 4 * (tid + RG_T * q);
                K kk[4];
                if (sizeof(K) == 4) {
                    const int4 v = *reinterpret_cast<const int4*>(gk + r0);
                    kk[0] = (K)v.x; kk[1] = (K)v.y; kk[2] = (K)v.z; kk[3] = (K)v.w;
                } else {
                    const longlong2 a = *reinterpret_cast<const longlong2*>(gk + r0);
                    const longlong2 b = *reinterpret_cast<const longlong2*>(gk + r0 + 2);
                    kk[0] = (K)a.x; kk[1] = (K)a.y; kk[2] = (K)b.x; kk[3] = (K)b.y;
                }
                int32_t pp[4];
                if (pay) {
                    const int4 v = *reinterpret_cast<const int4*>(gp + r0);
                    pp[0] = v.x; pp[1] = v.y; pp[2] = v.z; pp[3] = v.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) pp[e] = (int32_t)(x.beg + r0 + e);
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int j = 4 * q + e;
                    dv[j] = 0xffffffffu;
                    if (r0 + e < x.cnt) {
                        kv[j] = kk[e];
                        pv[j] = pp[e];
                        dv[j] = dg(kv[j]);
                        rv[j] = atomicAdd(&s_cnt[dv[j]], 1u);
                    }
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < IPT; j++) {
                const int i = j * RG_T + tid;
                dv[j] = 0xffffffffu;
                if (i < x.cnt) {
                    kv[j] = x.tma ? gk[x.koff + i] : key[x.beg + i];
                    pv[j] = pay ? (x.tma ? gp[x.poff + i] : pay[x.beg + i]) : (int32_t)(x.beg + i);
                    dv[j] = dg(kv[j]);
                    rv[j] = atomicAdd(&s_cnt[dv[j]], 1u);
                }
            }
        }
        __syncthreads();  // counts complete; the stage is free to reorder into
        rg_scan_digits(s_cnt, s_ts, s_gb, s_cur, nd, s_wsum);
        RW* rr = reinterpret_cast<RW*>(st);
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            if (dv[j] != 0xffffffffu) {
                const uint32_t pos = s_ts[dv[j]] + rv[j];
                RW w;
                w.key = kv[j];
                w.pay = pv[j];
                rr[pos] = w;
                if (KEEP) s_d[pos] = (uint16_t)dv[j];
            }
        }
        __syncthreads();
        for (int pos = tid; pos < x.cnt; pos += RG_T) {
            const RW w = rr[pos];
            const uint32_t d = KEEP ? (uint32_t)s_d[pos] : dg(w.key);
            out[s_gb[d] + (uint32_t)pos] = w;
        }
    }
}

// ----------------------------------------------------------- level 2 --

// Bit of key hash h in the filter slice of its region (fb - b1 bits).
__device__ __forceinline__ uint32_t rg_slice_bit(uint32_t h, int fb, uint32_t smask) {
    return (h >> (32 - fb)) & smask;
}

template <typename K>
struct Region2Smem {
    __host__ __device__ static constexpr size_t bytes() {
        return 2 * (size_t)RG_STAGE + ((size_t)1 << RG_SLICE_LOG) / 8 + 5 * (size_t)RG_F2MAX * 4;
    }
};

// Starts the bulk copy of rows [beg, beg + cnt) into `stage`; thread 0 only.
// koff = rows between the widened start and row `beg`.
template <typename RW>
__device__ __forceinline__ void stage_rows(StageTile* t, const RW* rows, uint64_t rows_ok, unsigned char* stage,
                                           uint64_t* bar) {
    t->tma = 0;
    uint64_t b0 = 0;
    uint32_t nb = 0;
    if (!byte_span(rows, t->beg, t->cnt, sizeof(RW), rows_ok, &b0, &nb) || nb > (uint32_t)RG_STAGE) return;
    if ((t->beg * sizeof(RW) - b0) % sizeof(RW)) return;  // a row straddles the widened start
    t->tma = 1;
    t->koff = (int)((t->beg * sizeof(RW) - b0) / sizeof(RW));
    t->poff = 0;
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, nb);
    tma_load_1d(stage, reinterpret_cast<const unsigned char*>(rows) + b0, nb, bar);
}

// Level-2 pass.  Block b takes regions b, b + grid, ... of [0, F1).  For a
// region (rows [start1[i], start1[i + 1]) of the level-1 rows) it
//   1. streams the rows once: counts second-level digits of the rows it
//      keeps (FILTER: the key's bit is set in the region's slice of `bitmap`),
//      and with BUILD sets each key's bit in the slice;
//   2. records partition p = i * F2 + j as rows [pbeg[p], pbeg[p] + pcnt[p])
//      of `out` (kept rows are packed at the front of the region's range);
//   3. streams the rows again and writes the kept rows to their partitions, a
//      tile at a time ordered by digit in shared memory.
// `survivors` receives the rows kept.
template <typename K, bool BUILD, bool FILTER>
__global__ void __launch_bounds__(RG_T, 1)
k_region2(const Row<K, false>* __restrict__ in, uint64_t rows_ok, const uint64_t* __restrict__ start1, int F1, int b1,
          int b2, uint32_t* __restrict__ bitmap, int fb, Row<K, false>* __restrict__ out, uint32_t* __restrict__ pbeg,
          uint32_t* __restrict__ pcnt, unsigned long long* __restrict__ survivors, unsigned int* __restrict__ err) {
    using S = RgShape<K>;
    using RW = Row<K, false>;
    constexpr int T = S::T2, IPT = T / RG_T;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage0 = smem;
    uint32_t* s_slice = reinterpret_cast<uint32_t*>(smem + 2 * (size_t)RG_STAGE);
    uint32_t* s_hc = s_slice + (1u << RG_SLICE_LOG) / 32;  // region digit counts
    uint32_t* s_cnt = s_hc + RG_F2MAX;                     // tile digit counts
    uint32_t* s_ts = s_cnt + RG_F2MAX;                     // tile digit starts
    uint32_t* s_gb = s_ts + RG_F2MAX;                      // tile digit global bases
    uint32_t* s_cur = s_gb + RG_F2MAX;                     // digit cursors
    __shared__ uint32_t s_wsum[32];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ StageTile tile[2];
    __shared__ int tphase[2];   // 0 = histogram tile, 1 = row tile
    __shared__ int tregion[2];
    __shared__ uint32_t s_tot;
    const int tid = threadIdx.x;
    const int F2 = 1 << b2;
    const int sbits = fb - b1;
    const uint32_t smask = (1u << sbits) - 1u;
    const int swords = sbits >= 5 ? 1 << (sbits - 5) : 1;
    const int shift2 = 32 - b1 - b2;
    const uint32_t mask2 = (uint32_t)F2 - 1u;
    for (int i = tid; i < RG_F2MAX; i += RG_T) s_cnt[i] = 0;
    // producer (thread 0): region, phase and first row of the next tile
    int pr = blockIdx.x, pphase = 0;
    int64_t prow = pr < F1 ? (int64_t)start1[pr] : 0;
    auto issue = [&](int s) {
        StageTile x;
        x.cnt = -1;
        x.tma = 0;
        x.beg = 0;
        while (pr < F1) {
            const int64_t e = (int64_t)start1[pr + 1];
            if (prow < e) break;
            if (pphase == 0) {  // the row pass of this region follows its histogram pass
                pphase = 1;
                prow = (int64_t)start1[pr];
                if (prow < e) break;
            }
            pr += gridDim.x;
            pphase = 0;
            if (pr < F1) prow = (int64_t)start1[pr];
        }
        if (pr < F1) {
            const int64_t e = (int64_t)start1[pr + 1];
            x.beg = prow;
            x.cnt = (int)min((int64_t)T, (int64_t)(e - prow));
            stage_rows<RW>(&x, in, rows_ok, stage0 + (size_t)s * RG_STAGE, &bar[s]);
            prow += x.cnt;
        }
        tile[s] = x;
        tphase[s] = pphase;
        tregion[s] = pr;
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(0);
        issue(1);
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    bool refill = false;   // the other stage is free and waits for the tile after next
    int cur_region = -1;   // region being processed
    int next_region = blockIdx.x;  // the block's next region not yet opened
    auto open_region = [&](int i) {  // all threads; ends with a barrier
        for (int w = tid; w < swords; w += RG_T) {
            if (FILTER) s_slice[w] = bitmap[(size_t)i * swords + w];
            if (BUILD) s_slice[w] = 0;
        }
        for (int j = tid; j < RG_F2MAX; j += RG_T) s_hc[j] = 0;
        __syncthreads();
    };
    auto close_histogram = [&](int i) {  // all threads: partitions of region i, cursors; ends with a barrier
        const uint32_t rb = (uint32_t)start1[i];
        // exclusive scan of s_hc over F2 <= 256 digits by the first 8 warps
        if (tid < 256) {
            const int lane = tid & 31, warp = tid >> 5;
            const uint32_t v = tid < F2 ? s_hc[tid] : 0u;
            const uint32_t inc = warp_incl_scan(v);
            if (lane == 31) s_wsum[warp] = inc;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            const uint32_t ws = lane < 8 ? s_wsum[lane] : 0u;
            const uint32_t wi = warp_incl_scan(ws);
            const uint32_t wpre = __shfl_sync(0xffffffffu, wi - ws, warp);
            const uint32_t pre = wpre + inc - v;
            if (tid < F2) {
                pbeg[(size_t)i * F2 + tid] = rb + pre;
                pcnt[(size_t)i * F2 + tid] = v;
                s_cur[tid] = rb + pre;
            }
            if (tid == 255) s_tot = wpre + inc;
        }
        __syncthreads();
        if (tid == 0 && s_tot) atomicAdd(survivors, (unsigned long long)s_tot);
        if (BUILD)
            for (int w = tid; w < swords; w += RG_T) bitmap[(size_t)i * swords + w] = s_slice[w];
    };
    for (int s = 0;; s ^= 1) {
        const StageTile x = tile[s];
        const int xr = tregion[s], xph = tphase[s];
        // regions the producer skipped (no rows) before this tile's region
        while (next_region < F1 && (x.cnt < 0 || next_region < xr)) {
            open_region(next_region);
            close_histogram(next_region);
            next_region += gridDim.x;
        }
        if (x.cnt < 0) break;
        if (xr != cur_region) {
            open_region(xr);
            cur_region = xr;
            next_region = xr + gridDim.x;
        }
        unsigned char* st = stage0 + (size_t)s * RG_STAGE;
        bool ok = true;
        if (x.tma) ok = mbar_wait(&bar[s], s ? ph1 : ph0, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (x.tma) mbar_wait(&bar[s], s ? ph1 : ph0, nullptr);
                if (!refill && tile[s ^ 1].cnt >= 0 && tile[s ^ 1].tma) mbar_wait(&bar[s ^ 1], s ? ph0 : ph1, nullptr);
            }
            break;
        }
        // every thread is past the previous tile: its stage is free
        if (refill && tid == 0) issue(s ^ 1);
        refill = true;
        if (x.tma) {
            if (s) ph1 ^= 1u; else ph0 ^= 1u;
        }
        const RW* gr = reinterpret_cast<const RW*>(st) + x.koff;
        if (xph == 0) {
            // ---- histogram tile ----
            for (int i = tid; i < x.cnt; i += RG_T) {
                const K k = x.tma ? gr[i].key : in[x.beg + i].key;
                const uint32_t h = khash(k);
                if (FILTER || BUILD) {
                    const uint32_t bit = rg_slice_bit(h, fb, smask);
                    if (FILTER && !((s_slice[bit >> 5] >> (bit & 31)) & 1u)) continue;
                    if (BUILD) atomicOr(&s_slice[bit >> 5], 1u << (bit & 31));
                }
                atomicAdd(&s_hc[b2 ? (h >> shift2) & mask2 : 0u], 1u);
            }
            __syncthreads();
            if (x.beg + x.cnt >= (int64_t)start1[xr + 1]) close_histogram(xr);
            continue;
        }
        // ---- row tile ----
        RW rw[IPT];
        uint32_t dv[IPT], rv[IPT];
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const int i = j * RG_T + tid;
            dv[j] = 0xffffffffu;
            if (i < x.cnt) {
                rw[j] = x.tma ? gr[i] : in[x.beg + i];
                const uint32_t h = khash(rw[j].key);
                bool keep = true;
                if (FILTER) {
                    const uint32_t bit = rg_slice_bit(h, fb, smask);
                    keep = (s_slice[bit >> 5] >> (bit & 31)) & 1u;
                }
                if (keep) {
                    dv[j] = b2 ? (h >> shift2) & mask2 : 0u;
                    rv[j] = atomicAdd(&s_cnt[dv[j]], 1u);
                }
            }
        }
        __syncthreads();  // counts complete; the stage is free to reorder into
        rg_scan_digits(s_cnt, s_ts, s_gb, s_cur, F2 < 2 ? 2 : F2, s_wsum, &s_tot);
        RW* rr = reinterpret_cast<RW*>(st);
#pragma unroll
        for (int j = 0; j < IPT; j++)
            if (dv[j] != 0xffffffffu) rr[s_ts[dv[j]] + rv[j]] = rw[j];
        __syncthreads();
        const uint32_t total = s_tot;
        for (uint32_t pos = tid; pos < total; pos += RG_T) {
            const RW w = rr[pos];
            const uint32_t d = b2 ? (khash(w.key) >> shift2) & mask2 : 0u;
            out[s_gb[d] + pos] = w;
        }
    }
}

}  // namespace jnx
