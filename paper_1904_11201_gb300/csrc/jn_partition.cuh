// Radix / range partitioning on the device: the Map-Reduce shuffle of
// Algorithm 1 (tuples regrouped by a function of the join key, Sec. 3.1 and
// Sec. 3.3.4) done as histogram -> exclusive scan -> scatter.
//
// Layout: a table is SoA (key column, optional second column, int32
// payload).  A partition pass reads "segments" (contiguous row ranges) in
// tiles of SC_TILE rows, sorts each tile by digit in shared memory, reserves
// one contiguous run per (segment, digit) with a single atomic on a global
// cursor, and writes the runs out coalesced.  Runs of the same digit from
// consecutive tiles land next to each other, so partial lines merge in L2.
#pragma once

#include "jn_async.cuh"
#include "jn_common.cuh"

namespace jnx {

// Partition block shape (build-time knobs): threads per block, rows per
// thread per tile, and blocks per SM the scatter is compiled for.
#ifndef JN_SC_T
#define JN_SC_T 512
#endif
#ifndef JN_SC_IPT
#define JN_SC_IPT 8
#endif
#ifndef JN_SC_MINB
#define JN_SC_MINB 2
#endif
constexpr int SC_T = JN_SC_T;            // threads per scatter block
constexpr int SC_IPT = JN_SC_IPT;        // rows per thread per tile
constexpr int SC_TILE = SC_T * SC_IPT;   // rows per tile
constexpr int SC_FMAX = 1024;            // digits per pass
constexpr int SC_DPT = SC_FMAX / SC_T;   // digits per thread in a tile's digit scan
static_assert(SC_FMAX % SC_T == 0, "the digit scan gives every thread the same number of digits");
constexpr uint32_t SC_DROP = 0xFFFFu;    // digit of a filtered row

// Digit = bits of the multiplicative key hash: (khash(k) >> shift) & mask.
struct HashDigit {
    static constexpr int kFilterWords = 0;
    int shift;
    uint32_t mask;
    __device__ __forceinline__ void bind(uint32_t*) {}
    __device__ __forceinline__ void set_seg(int) {}
    __device__ __forceinline__ bool is_special(uint32_t) const { return false; }
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return (khash(k) >> shift) & mask;
    }
};

// Per-segment hash digit for batches of joins: segment s takes the top
// bits[s] bits of the key hash (0 bits: a single partition).
struct SegHashDigit {
    static constexpr int kFilterWords = 0;
    const int* bits;
    int b;
    __device__ __forceinline__ void bind(uint32_t*) {}
    __device__ __forceinline__ void set_seg(int s) { b = bits[s]; }
    __device__ __forceinline__ bool is_special(uint32_t) const { return false; }
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return b ? (khash(k) >> (32 - b)) : 0u;
    }
};

// Range parameters shared by both tables of a theta join: group of value v
// is (v - lo) >> shift, with lo and shift computed on the device.
struct RangeParams {
    long long lo;
    long long hi;
    int shift;      // group shift
    int groups;     // number of groups in use
    int fshift;     // fine-bucket shift inside a group window
    int pad;
};

struct RangeDigit {
    static constexpr int kFilterWords = 0;
    const RangeParams* p;
    __device__ __forceinline__ void bind(uint32_t*) {}
    __device__ __forceinline__ void set_seg(int) {}
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return (uint32_t)(((uint64_t)((int64_t)k - (int64_t)p->lo)) >> p->shift);
    }
};

// One join work item: rows [rbeg, rbeg + rn) of R against all rows
// [sbeg, sbeg + sn) of S of the same partition.
struct Item {
    unsigned long long rbeg, sbeg;
    int rn, sn;
};

// ---------------------------------------------------------------- rows --
// Partitioned intermediates are stored as rows (array of structs): the key,
// an optional second column and the payload of one tuple sit together, so a
// tuple moves with one load and one store and a tile with one bulk copy.
template <typename K, bool HB>
struct Row;
template <>
struct __align__(8) Row<int32_t, false> {
    int32_t key;
    int32_t pay;
};
template <>
struct __align__(16) Row<int64_t, false> {
    int64_t key;
    int32_t pay;
    int32_t pad;
};
template <>
struct __align__(16) Row<int32_t, true> {
    int32_t key;
    int32_t b;
    int32_t pay;
    int32_t pad;
};
template <>
struct __align__(8) Row<int64_t, true> {
    int64_t key;
    int64_t b;
    int32_t pay;
    int32_t pad;
};

// ------------------------------------------------------ presence + hist --
// One read of a key column: sets the key's bit in the presence bitmap
// (Algorithm 1's Map1/Reduce1 key set, as a bitmap) and counts first-pass
// digits (unfiltered, an upper bound of each region's survivors).
template <typename K, typename Digit>
__global__ void __launch_bounds__(512)
k_presence_hist(const K* __restrict__ keys, int64_t n, uint32_t* __restrict__ bitmap,
                uint32_t fmask, Digit dg0, int nd, unsigned long long* __restrict__ hist) {
    extern __shared__ uint32_t s_h[];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);
    if (hist)
        for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vec = sizeof(K) == 4 && (((uintptr_t)keys) & 15) == 0;
    int64_t start = 0;
    if (vec) {
        const int64_t nv = n / 4;
        const int4* kv = reinterpret_cast<const int4*>(keys);
        const int64_t nvw = (nv + 31) & ~(int64_t)31;  // warps stay converged for the merge
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvw; i += stride) {
            const bool in = i < nv;
            int4 q = in ? __ldcs(kv + i) : make_int4(0, 0, 0, 0);
            int32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t d = in ? dg((K)v[j]) : 0u;
                if (bitmap && in && !dg.is_special(d)) {
                    const uint32_t b = fbits((K)v[j]) & fmask;
                    atomicOr(&bitmap[b >> 5], 1u << (b & 31));
                }
                if (hist && in) atomicAdd(&s_h[d], 1u);
            }
        }
        start = nv * 4;
    }
    const int64_t rem = n - start;
    const int64_t remw = (rem + 31) & ~(int64_t)31;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < remw; t += stride) {
        const bool in = t < rem;
        const K k = in ? keys[start + t] : (K)0;
        const uint32_t d = in ? dg(k) : 0u;
        if (bitmap && in && !dg.is_special(d)) {
            const uint32_t b = fbits(k) & fmask;
            atomicOr(&bitmap[b >> 5], 1u << (b & 31));
        }
        if (hist && in) atomicAdd(&s_h[d], 1u);
    }
    __syncthreads();
    if (hist)
        for (int i = threadIdx.x; i < nd; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[i], (unsigned long long)s_h[i]);
}

// -------------------------------------------------------------- segments --
// One block: segment i covers [seg_begin[i], seg_begin[i] + cnt[i]) where
// cnt[i] = cursor[i] - seg_begin[i] (rows a pass actually wrote); writes the
// tile prefix (SC_TILE rows per tile) and the total row count.
static __global__ void k_segments(const unsigned long long* __restrict__ cursor,
                           const uint64_t* __restrict__ seg_begin, int nseg,
                           uint64_t* __restrict__ seg_count, uint64_t* __restrict__ tile_prefix,
                           uint64_t* __restrict__ total_rows) {
    __shared__ uint64_t tmp[33];
    uint64_t carry_t = 0, carry_r = 0;
    for (int base = 0; base < nseg; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint64_t cnt = 0, nt = 0;
        if (i < nseg) {
            cnt = cursor[i] - seg_begin[i];
            seg_count[i] = cnt;
            nt = (cnt + SC_TILE - 1) / SC_TILE;
        }
        uint64_t tt, tr;
        uint64_t pre = block_excl_scan(nt, tmp, &tt);
        if (i < nseg) tile_prefix[i] = carry_t + pre;
        block_excl_scan(cnt, tmp, &tr);
        carry_t += tt;
        carry_r += tr;
    }
    if (threadIdx.x == 0) {
        tile_prefix[nseg] = carry_t;
        if (total_rows) *total_rows = carry_r;
    }
}

// Finds the segment holding tile t: the last i with tile_prefix[i] <= t.
__device__ __forceinline__ int find_segment(const uint64_t* tp, int nseg, uint64_t t) {
    int lo = 0, hi = nseg;  // answer in [lo, hi)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (tp[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// --------------------------------------------------- per-segment hist --
// Digit histogram of every segment: hist[seg * nd + digit].  Persistent
// blocks take tiles round-robin; the tile prefix is held in shared memory.
template <typename K, typename Digit>
__global__ void __launch_bounds__(SC_T)
k_seg_hist(const K* __restrict__ keys, const uint64_t* __restrict__ seg_begin,
           const uint64_t* __restrict__ seg_count, const uint64_t* __restrict__ tile_prefix,
           int nseg, Digit dg0, int nd, unsigned long long* __restrict__ hist,
           unsigned int* __restrict__ work) {
    extern __shared__ uint32_t s_h[];
    __shared__ uint64_t s_tp[SC_FMAX + 1];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);
    for (int i = threadIdx.x; i <= nseg; i += blockDim.x) s_tp[i] = tile_prefix[i];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const uint64_t ntiles = s_tp[nseg];
    int seg_held = -1;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int seg = find_segment(s_tp, nseg, t);
        if (seg != seg_held) {
            // flush the counts of the previous segment before switching
            if (seg_held >= 0) {
                __syncthreads();
                for (int i = threadIdx.x; i < nd; i += blockDim.x) {
                    if (s_h[i]) atomicAdd(&hist[(uint64_t)seg_held * nd + i], (unsigned long long)s_h[i]);
                    s_h[i] = 0;
                }
                __syncthreads();
            }
            seg_held = seg;
        }
        const uint64_t off = (t - s_tp[seg]) * SC_TILE;
        const uint64_t beg = seg_begin[seg] + off;
        const int cnt = (int)min((uint64_t)SC_TILE, seg_count[seg] - off);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) atomicAdd(&s_h[dg(keys[beg + i])], 1u);
    }
    __syncthreads();
    if (seg_held >= 0)
        for (int i = threadIdx.x; i < nd; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(uint64_t)seg_held * nd + i], (unsigned long long)s_h[i]);
}

// Input of a partition pass: column buffers (the caller's table) or rows
// (the output of an earlier pass).
// Columns of one segment of a batch (a table of one join of the batch).
template <typename K>
struct SegCols {
    const K* key;
    const K* key_b;      // second column carried along (band joins), or NULL
    const int32_t* pay;  // NULL = row index
    uint64_t n;
};

// A tile of a batch: rows [beg, beg + cnt) of segment seg.
struct TileRef {
    unsigned long long beg;
    int seg;
    int cnt;
};

template <typename K, bool HB>
struct PartIn {
    const K* key;           // columns (when rows == NULL)
    const K* key_b;
    const int32_t* pay;     // NULL = row index
    const Row<K, HB>* rows; // rows (when not NULL)
    uint64_t rows_ok;       // rows that may be read (allocation size)
    const SegCols<K>* segs; // batches: per-segment columns (key, pay), else NULL
    const TileRef* tiles;   // batches: tile list, else NULL (tiles from the segment prefix)
    bool plain = false;     // columns in page-locked host memory: plain loads, no bulk copies
};

// Digit histogram of every segment of a row array (see k_seg_hist).
template <typename R, typename Digit>
__global__ void __launch_bounds__(SC_T)
k_seg_hist_rows(const R* __restrict__ rows, const uint64_t* __restrict__ seg_begin,
                const uint64_t* __restrict__ seg_count, const uint64_t* __restrict__ tile_prefix, int nseg,
                Digit dg0, int nd, unsigned long long* __restrict__ hist) {
    extern __shared__ uint32_t s_h[];
    __shared__ uint64_t s_tp[SC_FMAX + 1];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);
    for (int i = threadIdx.x; i <= nseg; i += blockDim.x) s_tp[i] = tile_prefix[i];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const uint64_t ntiles = s_tp[nseg];
    int seg_held = -1;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int seg = find_segment(s_tp, nseg, t);
        if (seg != seg_held) {
            if (seg_held >= 0) {
                __syncthreads();
                for (int i = threadIdx.x; i < nd; i += blockDim.x) {
                    if (s_h[i]) atomicAdd(&hist[(uint64_t)seg_held * nd + i], (unsigned long long)s_h[i]);
                    s_h[i] = 0;
                }
                __syncthreads();
            }
            seg_held = seg;
        }
        const uint64_t off = (t - s_tp[seg]) * SC_TILE;
        const uint64_t beg = seg_begin[seg] + off;
        const int cnt = (int)min((uint64_t)SC_TILE, seg_count[seg] - off);
        // all of a thread's keys of the tile are loaded before the first count,
        // so their loads are in flight together
        constexpr int PER = SC_TILE / SC_T;
        decltype(rows[0].key) k[PER];
#pragma unroll
        for (int j = 0; j < PER; j++) {
            const int i = j * SC_T + threadIdx.x;
            if (i < cnt) k[j] = rows[beg + i].key;
        }
#pragma unroll
        for (int j = 0; j < PER; j++)
            if (j * SC_T + (int)threadIdx.x < cnt) atomicAdd(&s_h[dg(k[j])], 1u);
    }
    __syncthreads();
    if (seg_held >= 0)
        for (int i = threadIdx.x; i < nd; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(uint64_t)seg_held * nd + i], (unsigned long long)s_h[i]);
}

// ---------------------------------------------------------------- scatter --
// Moves the rows of every segment into digit order.  `cursor[seg * nd + d]`
// holds the next free output row of (segment, digit) and is advanced by one
// atomic per tile and digit.  With FILTER, a row is dropped unless its key's
// bit is set in `other` (the presence bitmap of the other table).
//
// Input tiles are staged in shared memory by 1-D TMA bulk copies: as soon as
// a tile has been read into registers, thread 0 starts the copy of the block's
// next tile, so its load overlaps the digit sort and write-out of this one.
// Tiles whose widened 16-byte span would pass `rows_ok` (or whose base is not
// 16-byte aligned) are read with plain loads instead.
struct TileDesc {
    unsigned long long beg;
    int cnt;
    int seg;
    int valid;
    int tma;
    int koff;  // element offset of row `beg` in the staged key column / rows
    int boff;
    int poff;
};

template <typename K, bool HB>
struct ScatterSmem {
    using R = Row<K, HB>;
    static constexpr int GK = SC_TILE + 32 / (int)sizeof(K);  // staged key column (and b column)
    static constexpr int GP = SC_TILE + 8;                    // staged payload column
    static constexpr int GR = SC_TILE + 16;                   // staged rows (widened)
    __host__ __device__ static constexpr size_t staging_bytes() {
        return ((((size_t)GK * sizeof(K) * (HB ? 2 : 1) + (size_t)GP * 4) > (size_t)GR * sizeof(R)
                     ? ((size_t)GK * sizeof(K) * (HB ? 2 : 1) + (size_t)GP * 4)
                     : (size_t)GR * sizeof(R)) +
                127) &
               ~(size_t)127;
    }
    __host__ __device__ static constexpr size_t bytes() {
        return staging_bytes() + (size_t)SC_TILE * sizeof(R) + (size_t)SC_FMAX * 16;
    }
};

// Rows of tile t: segment, first row and row count.  `tp` is the tile
// prefix held in shared memory.
__device__ __forceinline__ void tile_rows(const uint64_t* tp, int nseg, uint64_t t,
                                          const uint64_t* __restrict__ seg_begin,
                                          const uint64_t* __restrict__ seg_count, TileDesc* d,
                                          const TileRef* tiles = nullptr) {
    if (tiles) {
        const TileRef x = tiles[t];
        d->seg = x.seg;
        d->beg = x.beg;
        d->cnt = x.cnt;
        return;
    }
    const int seg = find_segment(tp, nseg, t);
    const uint64_t off = (t - tp[seg]) * SC_TILE;
    d->seg = seg;
    d->beg = seg_begin[seg] + off;
    d->cnt = (int)min((uint64_t)SC_TILE, seg_count[seg] - off);
}

// Byte span [beg*E, (beg+cnt)*E) widened to 16-byte boundaries; false when
// the base is unaligned or the widened end passes the readable bytes.
__device__ __forceinline__ bool byte_span(const void* base, uint64_t beg, uint64_t cnt, uint64_t e,
                                          uint64_t rows_ok, uint64_t* b0, uint32_t* bytes) {
    const uint64_t lo = (beg * e) & ~15ull;
    const uint64_t hi = ((beg + cnt) * e + 15) & ~15ull;
    if ((((uintptr_t)base) & 15) != 0 || hi > rows_ok * e) return false;
    *b0 = lo;
    *bytes = (uint32_t)(hi - lo);
    return true;
}

// Starts the bulk copy of a tile into the staging buffer (thread 0 only).
template <typename K, bool HB>
__device__ __forceinline__ void scatter_issue(TileDesc* d, const PartIn<K, HB>& in, unsigned char* stage,
                                              uint64_t* bar) {
    using SM = ScatterSmem<K, HB>;
    d->tma = 0;
    if (in.rows) {
        uint64_t b0;
        uint32_t nb;
        if (!byte_span(in.rows, d->beg, d->cnt, sizeof(Row<K, HB>), in.rows_ok, &b0, &nb)) return;
        d->tma = 1;
        d->koff = (int)((d->beg * sizeof(Row<K, HB>) - b0));  // byte offset
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, nb);
        tma_load_1d(stage, reinterpret_cast<const unsigned char*>(in.rows) + b0, nb, bar);
        return;
    }
    if (in.plain) return;
    const K* ikey = in.segs ? in.segs[d->seg].key : in.key;
    const K* ikb = in.segs ? in.segs[d->seg].key_b : in.key_b;
    const int32_t* ipay = in.segs ? in.segs[d->seg].pay : in.pay;
    const uint64_t iok = in.segs ? in.segs[d->seg].n : in.rows_ok;
    uint64_t bk = 0, bb = 0, bp = 0;
    uint32_t nk = 0, nbb = 0, np = 0;
    bool ok = byte_span(ikey, d->beg, d->cnt, sizeof(K), iok, &bk, &nk);
    if (ok && HB) ok = byte_span(ikb, d->beg, d->cnt, sizeof(K), iok, &bb, &nbb);
    if (ok && ipay) ok = byte_span(ipay, d->beg, d->cnt, 4, iok, &bp, &np);
    if (!ok) return;
    d->tma = 1;
    d->koff = (int)(d->beg - bk / sizeof(K));
    d->boff = (int)(d->beg - bb / sizeof(K));
    d->poff = (int)(d->beg - bp / 4);
    K* gk = reinterpret_cast<K*>(stage);
    K* gb = gk + SM::GK;
    int32_t* gp = reinterpret_cast<int32_t*>(gb + (HB ? SM::GK : 0));
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, nk + nbb + np);
    tma_load_1d(gk, reinterpret_cast<const unsigned char*>(ikey) + bk, nk, bar);
    if (HB) tma_load_1d(gb, reinterpret_cast<const unsigned char*>(ikb) + bb, nbb, bar);
    if (ipay) tma_load_1d(gp, reinterpret_cast<const unsigned char*>(ipay) + bp, np, bar);
}

template <typename K, bool HB, bool FILTER, typename Digit>
__global__ void __launch_bounds__(SC_T, JN_SC_MINB)
k_scatter(PartIn<K, HB> in, const uint64_t* __restrict__ seg_begin, const uint64_t* __restrict__ seg_count,
          const uint64_t* __restrict__ tile_prefix, int nseg, Digit dg0, int nd,
          const uint32_t* __restrict__ other, uint32_t fmask, unsigned long long* __restrict__ cursor,
          Row<K, HB>* __restrict__ out, unsigned int* __restrict__ err) {
    using SM = ScatterSmem<K, HB>;
    using R = Row<K, HB>;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage = smem;
    R* s_row = reinterpret_cast<R*>(smem + SM::staging_bytes());
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_row + SC_TILE);
    uint32_t* s_start = s_cnt + SC_FMAX;
    unsigned long long* s_delta = reinterpret_cast<unsigned long long*>(s_start + SC_FMAX);
    __shared__ uint32_t tmp[33];
    __shared__ TileDesc desc[2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint64_t s_tp[SC_FMAX + 1];
    __shared__ uint32_t s_dgf[Digit::kFilterWords > 0 ? Digit::kFilterWords : 1];
    Digit dg = dg0;
    dg.bind(s_dgf);

    // Tiles are dealt round-robin: block b takes tiles b, b + grid, ...
    // batches pass a tile list (tile_prefix[0] = tile count) instead of segments
    if (!in.tiles)
        for (int i = threadIdx.x; i <= nseg; i += SC_T) s_tp[i] = tile_prefix[i];
    for (int i = threadIdx.x; i < nd; i += SC_T) s_cnt[i] = 0;
    __syncthreads();
    const uint64_t ntiles = in.tiles ? tile_prefix[0] : s_tp[nseg];
    uint64_t t = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        desc[0].valid = t < ntiles;
        if (t < ntiles) {
            tile_rows(s_tp, nseg, t, seg_begin, seg_count, &desc[0], in.tiles);
            scatter_issue<K, HB>(&desc[0], in, stage, &bar);
        }
    }
    __syncthreads();
    int cur = 0;
    uint32_t phase = 0;
    const K* gk = reinterpret_cast<const K*>(stage);
    const K* gb = gk + SM::GK;
    const int32_t* gp = reinterpret_cast<const int32_t*>(gb + (HB ? SM::GK : 0));
    while (true) {
        const TileDesc d = desc[cur];
        if (!d.valid) break;
        // look up the next tile now; its copy starts once the staging is free
        const uint64_t tn = t + gridDim.x;
        TileDesc dn;
        dn.valid = tn < ntiles;
        if (threadIdx.x == 0 && dn.valid) tile_rows(s_tp, nseg, tn, seg_begin, seg_count, &dn, in.tiles);
        bool ok = true;
        if (d.tma) ok = mbar_wait(&bar, phase, err);
        if (__syncthreads_or(!ok)) {
            if (d.tma) mbar_wait(&bar, phase, nullptr);  // let the copy in flight land before exiting
            break;
        }
        if (d.tma) phase ^= 1u;
        const uint64_t beg = d.beg;
        const int cnt = d.cnt;
        dg.set_seg(d.seg);
        const K* ikey = in.segs ? in.segs[d.seg].key : in.key;
        const K* ikb = in.segs ? in.segs[d.seg].key_b : in.key_b;
        const int32_t* ipay = in.segs ? in.segs[d.seg].pay : in.pay;

        R v[SC_IPT];
        uint32_t dd[SC_IPT];
        uint32_t rk[SC_IPT];
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) {
            const int i = j * SC_T + threadIdx.x;
            dd[j] = SC_DROP;
            if (i < cnt) {
                if (in.rows) {
                    v[j] = d.tma ? *reinterpret_cast<const R*>(stage + d.koff + (size_t)i * sizeof(R))
                                 : in.rows[beg + i];
                } else if (d.tma) {
                    v[j].key = gk[d.koff + i];
                    if constexpr (HB) v[j].b = gb[d.boff + i];
                    v[j].pay = ipay ? gp[d.poff + i] : (int32_t)(beg + i);
                } else {
                    v[j].key = ikey[beg + i];
                    if constexpr (HB) v[j].b = ikb[beg + i];
                    v[j].pay = ipay ? ipay[beg + i] : (int32_t)(beg + i);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) {
            const int i = j * SC_T + threadIdx.x;
            if (i < cnt) {
                bool keep = true;
                if (FILTER) {
                    const uint32_t b = fbits(v[j].key) & fmask;
                    keep = (__ldg(other + (b >> 5)) >> (b & 31)) & 1u;
                }
                if (keep) dd[j] = dg(v[j].key);
            }
        }
        __syncthreads();  // the staging buffer is free: start the next tile's copy
        if (threadIdx.x == 0) {
            if (dn.valid) scatter_issue<K, HB>(&dn, in, stage, &bar);
            desc[cur ^ 1] = dn;
        }
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) rk[j] = (dd[j] != SC_DROP) ? atomicAdd(&s_cnt[dd[j]], 1u) : 0u;
        __syncthreads();
        // exclusive scan of the digit counts; nd <= SC_FMAX = SC_DPT * SC_T
        uint32_t cc[SC_DPT];
        uint32_t csum = 0;
        const int i0 = SC_DPT * threadIdx.x;
#pragma unroll
        for (int q = 0; q < SC_DPT; q++) {
            cc[q] = i0 + q < nd ? s_cnt[i0 + q] : 0u;
            csum += cc[q];
        }
        uint32_t total;
        uint32_t pre = block_excl_scan(csum, tmp, &total);
#pragma unroll
        for (int q = 0; q < SC_DPT; q++) {
            const int i = i0 + q;
            if (i < nd) {
                s_start[i] = pre;
                if (cc[q]) s_delta[i] = atomicAdd(&cursor[(uint64_t)d.seg * nd + i], (unsigned long long)cc[q]) - pre;
            }
            pre += cc[q];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) {
            if (dd[j] != SC_DROP) {
                const uint32_t pos = s_start[dd[j]] + rk[j];
                s_row[pos] = v[j];
            }
        }
        __syncthreads();
        // a staged row's digit is recomputed from its key (cheaper than
        // keeping it in shared memory next to the row)
        for (uint32_t pos = threadIdx.x; pos < total; pos += SC_T) {
            const R x = s_row[pos];
            out[s_delta[dg(x.key)] + pos] = x;
        }
        for (int i = threadIdx.x; i < nd; i += SC_T) s_cnt[i] = 0;
        __syncthreads();
        cur ^= 1;
        t = tn;
    }
}

template <typename K, bool HB>
inline size_t scatter_smem() {
    return ScatterSmem<K, HB>::bytes();
}

// Single-block setup for one-segment passes: seg_begin = 0, count = n.
static __global__ void k_one_segment(uint64_t* seg_begin, uint64_t* seg_count, uint64_t* tile_prefix,
                              uint64_t n) {
    if (threadIdx.x == 0) {
        seg_begin[0] = 0;
        seg_count[0] = n;
        tile_prefix[0] = 0;
        tile_prefix[1] = (n + SC_TILE - 1) / SC_TILE;
    }
}

// cursor[i] = start[i] (u64 -> unsigned long long copy of scan offsets).
static __global__ void k_init_cursor(const uint64_t* __restrict__ start, unsigned long long* __restrict__ cur,
                              int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cur[i] = start[i];
}

}  // namespace jnx

namespace jnx {
// dst[i] = src[i] for i < n (tiny device-to-device word copies on the stream).
static __global__ void k_copy_words(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst, int n) {
    int i = threadIdx.x;
    if (i < n) dst[i] = src[i];
}
}  // namespace jnx
