// Frequent ("heavy") join keys of the hash join.
//
// Under a skewed key distribution a few keys carry millions of rows; their
// join is the full cross product of their R rows and S rows, so it needs no
// hash table at all: its size is c_R(k) * c_S(k) and its pairs are written as
// a Cartesian product (the always-true region of Algorithm 3, Sec. 4.2,
// applied to a single key).  Heavy keys are picked from a strided sample of
// both key columns; rows with a heavy key are set aside in the first
// partition pass (digit F1) and grouped by key afterwards.  Which keys are
// picked never changes the result: a key left out simply stays on the
// partitioned path.
#pragma once

#include "jn_partition.cuh"

namespace jnx {

constexpr int HV_MAX = 1024;         // heavy keys at most (digits of the heavy grouping pass)
constexpr int HV_SLOTS = 4096;       // open-addressing table of heavy keys
constexpr int HV_FBITS = 16;         // shared-memory filter of 2^16 bits over khash
constexpr int HV_SAMPLE_LOG = 21;    // sample table slots (log2)

template <typename K>
__device__ __forceinline__ K key_sentinel() {
    return sizeof(K) == 4 ? (K)INT32_MIN : (K)INT64_MIN;
}

// Heavy key set: keys[i], i < *count, and a table mapping key -> index.
template <typename K>
struct HeavySet {
    const K* tab_key;        // HV_SLOTS keys
    const int* tab_idx;      // HV_SLOTS indices, -1 = empty
    const K* keys;           // HV_MAX keys in index order
    const int* count;        // number of heavy keys
};

__device__ __forceinline__ uint32_t hv_slot(uint32_t h) { return (h * 0x85EBCA6Bu) >> (32 - 12); }

template <typename K>
__device__ __forceinline__ int hv_lookup(const HeavySet<K>& hs, K k) {
    uint32_t s = hv_slot(khash(k));
    for (int probe = 0; probe < HV_SLOTS; probe++) {
        const int idx = hs.tab_idx[s];
        if (idx < 0) return -1;
        if (hs.tab_key[s] == k) return idx;
        s = (s + 1) & (HV_SLOTS - 1);
    }
    return -1;
}

// Fills the shared-memory filter (2^HV_FBITS bits, HV_FBITS / 8 KB) from the
// heavy list; all threads of the block call it, followed by __syncthreads.
template <typename K>
__device__ __forceinline__ void hv_filter_fill(uint32_t* f, const HeavySet<K>& hs) {
    for (int i = threadIdx.x; i < (1 << HV_FBITS) / 32; i += blockDim.x) f[i] = 0;
    __syncthreads();
    const int h = *hs.count;
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const uint32_t b = khash(hs.keys[i]) >> (32 - HV_FBITS);
        atomicOr(&f[b >> 5], 1u << (b & 31));
    }
}

// Index of k in the heavy set, or -1; the filter answers most misses.
template <typename K>
__device__ __forceinline__ int hv_find(const uint32_t* f, const HeavySet<K>& hs, K k) {
    const uint32_t b = khash(k) >> (32 - HV_FBITS);
    if (!((f[b >> 5] >> (b & 31)) & 1u)) return -1;
    return hv_lookup(hs, k);
}

// ------------------------------------------------------------- sampling --
template <typename K>
__global__ void k_sample_init(K* tk, unsigned int* tc, int slots) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x) {
        tk[i] = key_sentinel<K>();
        tc[2 * i] = 0;
        tc[2 * i + 1] = 0;
    }
}

// Counts every `stride`-th key of a column into the sample table (side 0 = R,
// 1 = S).  The sentinel key is never counted (it stays on the normal path).
template <typename K>
__global__ void k_sample(const K* __restrict__ keys, int64_t n, int64_t stride, int side, K* tk,
                         unsigned int* tc) {
    const int slots = 1 << HV_SAMPLE_LOG;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j * stride < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const K k = keys[j * stride];
        if (k == key_sentinel<K>()) continue;
        uint32_t s = (khash(k) * 0x27D4EB2Fu) >> (32 - HV_SAMPLE_LOG);
        for (int probe = 0; probe < 64; probe++) {
            K old;
            if (sizeof(K) == 4)
                old = (K)atomicCAS(reinterpret_cast<int*>(tk) + s, (int)key_sentinel<K>(), (int)k);
            else
                old = (K)atomicCAS(reinterpret_cast<unsigned long long*>(tk) + s,
                                   (unsigned long long)key_sentinel<K>(), (unsigned long long)k);
            if (old == key_sentinel<K>() || old == k) {
                atomicAdd(&tc[2 * s + side], 1u);
                break;
            }
            s = (s + 1) & (slots - 1);
        }
    }
}

// Sampled counts are binned exactly below HV_CBINS - 1; the top bin holds
// every larger count.
constexpr int HV_CBINS = 4096;

// Histogram of each sampled key's larger count (over the two sides), for
// counts that reach `thr`.
template <typename K>
__global__ void k_heavy_hist(const K* __restrict__ tk, const unsigned int* __restrict__ tc, unsigned int thr,
                             unsigned int* __restrict__ hist) {
    __shared__ unsigned int sh[HV_CBINS];
    for (int i = threadIdx.x; i < HV_CBINS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int slots = 1 << HV_SAMPLE_LOG;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x) {
        if (tk[i] == key_sentinel<K>()) continue;
        const unsigned int c = max(tc[2 * i], tc[2 * i + 1]);
        if (c >= thr) atomicAdd(&sh[min(c, (unsigned int)HV_CBINS - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HV_CBINS; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One warp: the smallest count t >= thr that at most HV_MAX sampled keys
// reach, so the keys picked are the most frequent ones.
static __global__ void k_heavy_thr(const unsigned int* __restrict__ hist, unsigned int thr, unsigned int* __restrict__ t_out) {
    constexpr int PER = HV_CBINS / 32;
    const int lane = threadIdx.x;
    unsigned int part = 0;  // keys in this lane's bins
    for (int j = 0; j < PER; j++) part += hist[lane * PER + j];
    // keys in the bins of the lanes above this one
    unsigned int above = 0;
    for (int l = 31; l > 0; l--) {
        const unsigned int v = __shfl_sync(0xffffffffu, part, l);
        if (l > lane) above += v;
    }
    // the lane whose bins hold the crossing point finds it
    unsigned int t = 0;
    const bool cross = above <= (unsigned)HV_MAX && above + part > (unsigned)HV_MAX;
    if (cross) {
        unsigned int acc = above;
        t = (unsigned int)(lane * PER + PER);
        for (int j = PER - 1; j >= 0; j--) {
            acc += hist[lane * PER + j];
            if (acc > (unsigned)HV_MAX) break;
            t = (unsigned int)(lane * PER + j);
        }
        if (t == (unsigned int)HV_CBINS) t = HV_CBINS - 1;  // the top bin alone holds more than HV_MAX keys
    }
    const unsigned int any = __ballot_sync(0xffffffffu, cross);
    if (any) t = __shfl_sync(0xffffffffu, t, __ffs(any) - 1);
    if (lane == 0) *t_out = max(any ? t : 0u, thr);
}

// Picks keys whose sampled count (the larger side) reaches *thr, at most
// HV_MAX of them, into keys[0 .. *count).
template <typename K>
__global__ void k_heavy_collect(const K* __restrict__ tk, const unsigned int* __restrict__ tc,
                                const unsigned int* __restrict__ thr_p, K* __restrict__ keys, int* __restrict__ count) {
    const int slots = 1 << HV_SAMPLE_LOG;
    const unsigned int thr = *thr_p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x) {
        if (tk[i] == key_sentinel<K>()) continue;
        if (max(tc[2 * i], tc[2 * i + 1]) >= thr) {
            const int at = atomicAdd(count, 1);
            if (at < HV_MAX) keys[at] = tk[i];
        }
    }
}

// One block: caps the heavy count and builds the key -> index table.
template <typename K>
__global__ void k_heavy_table(const K* __restrict__ keys, K* __restrict__ tab_key, int* __restrict__ tab_idx,
                              int* __restrict__ count) {
    for (int i = threadIdx.x; i < HV_SLOTS; i += blockDim.x) tab_idx[i] = -1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int h = *count < HV_MAX ? *count : HV_MAX;
        for (int i = 0; i < h; i++) {
            uint32_t s = hv_slot(khash(keys[i]));
            while (tab_idx[s] >= 0) s = (s + 1) & (HV_SLOTS - 1);
            tab_key[s] = keys[i];
            tab_idx[s] = i;
        }
        *count = h;
    }
}

// Sets the presence bit of every heavy key (the presence kernel skips
// heavy rows; a bit set for a key a table lacks only weakens the filter).
template <typename K>
__global__ void k_heavy_bits(HeavySet<K> hs, uint32_t* __restrict__ a, uint32_t* __restrict__ b, uint32_t fmask) {
    const int h = *hs.count;
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const uint32_t x = fbits(hs.keys[i]) & fmask;
        if (a) atomicOr(&a[x >> 5], 1u << (x & 31));
        if (b) atomicOr(&b[x >> 5], 1u << (x & 31));
    }
}

// Digit of a row on the heavy grouping pass: the index of its key.
template <typename K>
struct HeavyIdxDigit {
    static constexpr int kFilterWords = 0;
    HeavySet<K> hs;
    __device__ __forceinline__ void bind(uint32_t*) {}
    __device__ __forceinline__ void set_seg(int) {}
    __device__ __forceinline__ uint32_t operator()(K k) const {
        const int i = hv_lookup(hs, k);
        return i < 0 ? 0u : (uint32_t)i;  // every row of the heavy region has a heavy key
    }
};

// Digit of pass 1 with heavy keys set aside: F1 for a heavy key, else the
// hash digit.  `f` is the block's shared-memory filter.
template <typename K>
struct HeavyHashDigit {
    static constexpr int kFilterWords = (1 << HV_FBITS) / 32;
    int shift;
    uint32_t mask;
    uint32_t heavy_digit;
    HeavySet<K> hs;
    const uint32_t* f;
    __device__ __forceinline__ bool is_special(uint32_t d) const { return d == heavy_digit; }
    __device__ __forceinline__ void set_seg(int) {}
    // Fills the block's filter; all threads call it (it synchronises).
    __device__ __forceinline__ void bind(uint32_t* smem_filter) {
        hv_filter_fill(smem_filter, hs);
        __syncthreads();
        f = smem_filter;
    }
    __device__ __forceinline__ uint32_t operator()(K k) const {
        return hv_find(f, hs, k) >= 0 ? heavy_digit : ((khash(k) >> shift) & mask);
    }
};

// ---------------------------------------------------------- cross product --
// Per heavy key h: pairs c_R(h) * c_S(h) (block x = 0 writes them) and, for
// the checksum, sum over R_h of f * sum over S_h of g, reduced over row
// chunks: block (x, h) sums f over its chunk of R_h into fsum[h] and g over
// its chunk of S_h into gsum[h].
template <typename R>
__global__ void k_heavy_pairs(const R* __restrict__ rr, const uint64_t* __restrict__ roff,
                              const R* __restrict__ sr, const uint64_t* __restrict__ soff,
                              const int* __restrict__ count, uint64_t* __restrict__ pairs,
                              uint64_t* __restrict__ chunks, unsigned long long* __restrict__ fsum,
                              unsigned long long* __restrict__ gsum, int with_chk, uint64_t chunk) {
    __shared__ unsigned long long tmp[33];
    const int h = blockIdx.y;
    const bool live = h < *count;
    const uint64_t nr = live ? roff[h + 1] - roff[h] : 0, ns = live ? soff[h + 1] - soff[h] : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pairs[h] = nr * ns;
        chunks[h] = (nr * ns + chunk - 1) / chunk;
    }
    if (!with_chk || nr == 0 || ns == 0) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long f = 0, g = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride)
        f += chk_f(rr[roff[h] + i].pay);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += stride)
        g += chk_g(sr[soff[h] + i].pay);
    f = block_sum(f, tmp);
    g = block_sum(g, tmp);
    if (threadIdx.x == 0) {
        if (f) atomicAdd(&fsum[h], f);
        if (g) atomicAdd(&gsum[h], g);
    }
}

// chk += sum over heavy keys of fsum[h] * gsum[h].
__global__ void k_heavy_chk(const unsigned long long* __restrict__ fsum, const unsigned long long* __restrict__ gsum,
                            unsigned long long* __restrict__ chk) {
    __shared__ unsigned long long tmp[33];
    unsigned long long v = 0;
    for (int h = threadIdx.x; h < HV_MAX; h += blockDim.x) v += fsum[h] * gsum[h];
    v = block_sum(v, tmp);
    if (threadIdx.x == 0 && v) atomicAdd(chk, v);
}

// Writes the cross product of every group: pair q of group h is
// (R[roff[h] + q % nr], S[soff[h] + q / nr]) at out[base + pair_off[h] + q].
// Work is dealt in chunks of `chunk` pairs, round-robin over the blocks.
template <typename R>
__global__ void __launch_bounds__(256)
k_cartesian(const R* __restrict__ rr, const uint64_t* __restrict__ roff, const R* __restrict__ sr,
            const uint64_t* __restrict__ soff, const uint64_t* __restrict__ pair_off,
            const uint64_t* __restrict__ chunk_prefix, int groups, uint64_t chunk, uint64_t base,
            jn_pair* __restrict__ out) {
    const uint64_t nchunks = chunk_prefix[groups];
    for (uint64_t it = blockIdx.x; it < nchunks; it += gridDim.x) {
        const int h = find_segment(chunk_prefix, groups, it);
        const uint64_t nr = roff[h + 1] - roff[h];
        const uint64_t total = nr * (soff[h + 1] - soff[h]);
        const uint64_t q0 = (it - chunk_prefix[h]) * chunk;
        const uint64_t q1 = min(total, q0 + chunk);
        const uint64_t ob = base + pair_off[h];
        // walk (s, r) incrementally: r = q % nr advances by blockDim.x per step
        uint64_t q = q0 + threadIdx.x;
        uint64_t si = q / nr, ri = q - si * nr;
        const uint64_t step_s = blockDim.x / nr, step_r = blockDim.x - step_s * nr;
        for (; q < q1; q += blockDim.x) {
            st_pair(out + ob + q, rr[roff[h] + ri].pay, sr[soff[h] + si].pay);
            ri += step_r;
            si += step_s;
            if (ri >= nr) {
                ri -= nr;
                si++;
            }
        }
    }
}

}  // namespace jnx
