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

#include "jn_common.cuh"

namespace jnx {

constexpr int SC_T = 512;                // threads per scatter block
constexpr int SC_IPT = 8;                // rows per thread per tile
constexpr int SC_TILE = SC_T * SC_IPT;   // rows per tile
constexpr int SC_FMAX = 1024;            // digits per pass
constexpr uint32_t SC_DROP = 0xFFFFu;    // digit of a filtered row

// Digit = bits of the multiplicative key hash: (khash(k) >> shift) & mask.
struct HashDigit {
    int shift;
    uint32_t mask;
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return (khash(k) >> shift) & mask;
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
    const RangeParams* p;
    template <typename K>
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return (uint32_t)(((uint64_t)((int64_t)k - (int64_t)p->lo)) >> p->shift);
    }
};

// ------------------------------------------------------ presence + hist --
// One read of a key column: sets the key's bit in the presence bitmap
// (Algorithm 1's Map1/Reduce1 key set, as a bitmap) and counts first-pass
// digits (unfiltered, an upper bound of each region's survivors).
template <typename K>
__global__ void __launch_bounds__(512)
k_presence_hist(const K* __restrict__ keys, int64_t n, uint32_t* __restrict__ bitmap,
                uint32_t fmask, HashDigit dg, int nd, unsigned long long* __restrict__ hist) {
    extern __shared__ uint32_t s_h[];
    if (hist)
        for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vec = sizeof(K) == 4 && (((uintptr_t)keys) & 15) == 0;
    int64_t start = 0;
    if (vec) {
        const int64_t nv = n / 4;
        const int4* kv = reinterpret_cast<const int4*>(keys);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
            int4 q = __ldcs(kv + i);
            int32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (bitmap) {
                    uint32_t b = fbits((K)v[j]) & fmask;
                    atomicOr(&bitmap[b >> 5], 1u << (b & 31));
                }
                if (hist) atomicAdd(&s_h[dg((K)v[j])], 1u);
            }
        }
        start = nv * 4;
    }
    for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        K k = keys[i];
        if (bitmap) {
            uint32_t b = fbits(k) & fmask;
            atomicOr(&bitmap[b >> 5], 1u << (b & 31));
        }
        if (hist) atomicAdd(&s_h[dg(k)], 1u);
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
// blocks claim tiles from *work.
template <typename K, typename Digit>
__global__ void __launch_bounds__(SC_T)
k_seg_hist(const K* __restrict__ keys, const uint64_t* __restrict__ seg_begin,
           const uint64_t* __restrict__ seg_count, const uint64_t* __restrict__ tile_prefix,
           int nseg, Digit dg, int nd, unsigned long long* __restrict__ hist,
           unsigned int* __restrict__ work) {
    extern __shared__ uint32_t s_h[];
    __shared__ unsigned int s_tile;
    const uint64_t ntiles = tile_prefix[nseg];
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(work, 1u);
        for (int i = threadIdx.x; i < nd; i += blockDim.x) s_h[i] = 0;
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= ntiles) break;
        const int seg = find_segment(tile_prefix, nseg, t);
        const uint64_t off = (t - tile_prefix[seg]) * SC_TILE;
        const uint64_t beg = seg_begin[seg] + off;
        const int cnt = (int)min((uint64_t)SC_TILE, seg_count[seg] - off);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) atomicAdd(&s_h[dg(keys[beg + i])], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < nd; i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(uint64_t)seg * nd + i], (unsigned long long)s_h[i]);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- scatter --
// Moves the rows of every segment into digit order.  `cursor[seg * nd + d]`
// holds the next free output row of (segment, digit) and is advanced by one
// atomic per tile and digit.  With FILTER, a row is dropped unless its key's
// bit is set in `other` (the presence bitmap of the other table).  With
// key_b, a second column is carried along.  A NULL payload means "row
// index" (the input row number).
template <typename K, bool FILTER, typename Digit>
__global__ void __launch_bounds__(SC_T)
k_scatter(const K* __restrict__ keys, const K* __restrict__ key_b, const int32_t* __restrict__ pays,
          const uint64_t* __restrict__ seg_begin, const uint64_t* __restrict__ seg_count,
          const uint64_t* __restrict__ tile_prefix, int nseg, Digit dg, int nd,
          const uint32_t* __restrict__ other, uint32_t fmask,
          unsigned long long* __restrict__ cursor, K* __restrict__ out_keys,
          K* __restrict__ out_key_b, int32_t* __restrict__ out_pays, unsigned int* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_key = reinterpret_cast<K*>(smem);
    K* s_kb = s_key + SC_TILE;                                   // used only with key_b
    int32_t* s_pay = reinterpret_cast<int32_t*>(s_kb + (key_b ? SC_TILE : 0));
    uint16_t* s_dig = reinterpret_cast<uint16_t*>(s_pay + SC_TILE);
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_dig + SC_TILE);
    uint32_t* s_start = s_cnt + SC_FMAX;
    unsigned long long* s_base = reinterpret_cast<unsigned long long*>(s_start + SC_FMAX);
    __shared__ uint32_t tmp[33];
    __shared__ unsigned int s_tile;

    const uint64_t ntiles = tile_prefix[nseg];
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(work, 1u);
        for (int i = threadIdx.x; i < nd; i += SC_T) s_cnt[i] = 0;
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= ntiles) break;
        const int seg = find_segment(tile_prefix, nseg, t);
        const uint64_t off = (t - tile_prefix[seg]) * SC_TILE;
        const uint64_t beg = seg_begin[seg] + off;
        const int cnt = (int)min((uint64_t)SC_TILE, seg_count[seg] - off);

        K k[SC_IPT];
        K kb[SC_IPT];
        int32_t p[SC_IPT];
        uint32_t d[SC_IPT];
        uint32_t r[SC_IPT];
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) {
            const int i = j * SC_T + threadIdx.x;
            d[j] = SC_DROP;
            if (i < cnt) {
                k[j] = __ldcs(keys + beg + i);
                if (key_b) kb[j] = __ldcs(key_b + beg + i);
                p[j] = pays ? __ldcs(pays + beg + i) : (int32_t)(beg + i);
                bool keep = true;
                if (FILTER) {
                    const uint32_t b = fbits(k[j]) & fmask;
                    keep = (__ldg(other + (b >> 5)) >> (b & 31)) & 1u;
                }
                if (keep) d[j] = dg(k[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < SC_IPT; j++)
            r[j] = (d[j] != SC_DROP) ? atomicAdd(&s_cnt[d[j]], 1u) : 0u;
        __syncthreads();
        // exclusive scan of the digit counts; nd <= SC_FMAX = 2 * SC_T
        uint32_t c0 = 0, c1 = 0;
        const int i0 = 2 * threadIdx.x, i1 = i0 + 1;
        if (i0 < nd) c0 = s_cnt[i0];
        if (i1 < nd) c1 = s_cnt[i1];
        uint32_t total;
        uint32_t pre = block_excl_scan(c0 + c1, tmp, &total);
        if (i0 < nd) {
            s_start[i0] = pre;
            if (c0) s_base[i0] = atomicAdd(&cursor[(uint64_t)seg * nd + i0], (unsigned long long)c0);
        }
        if (i1 < nd) {
            s_start[i1] = pre + c0;
            if (c1) s_base[i1] = atomicAdd(&cursor[(uint64_t)seg * nd + i1], (unsigned long long)c1);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SC_IPT; j++) {
            if (d[j] != SC_DROP) {
                const uint32_t pos = s_start[d[j]] + r[j];
                s_key[pos] = k[j];
                if (key_b) s_kb[pos] = kb[j];
                s_pay[pos] = p[j];
                s_dig[pos] = (uint16_t)d[j];
            }
        }
        __syncthreads();
        for (uint32_t pos = threadIdx.x; pos < total; pos += SC_T) {
            const uint32_t dd = s_dig[pos];
            const unsigned long long o = s_base[dd] + (pos - s_start[dd]);
            out_keys[o] = s_key[pos];
            if (key_b) out_key_b[o] = s_kb[pos];
            out_pays[o] = s_pay[pos];
        }
        __syncthreads();
    }
}

template <typename K>
inline size_t scatter_smem(bool with_b) {
    return (size_t)SC_TILE * (sizeof(K) * (with_b ? 2 : 1) + 4 + 2) + SC_FMAX * 8 + SC_FMAX * 8;
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
