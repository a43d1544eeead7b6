// Sort-merge equi join of one hash partition pair: the third category of
// join algorithms in Sec. 2.3 (sort both tables, then walk them in order),
// beside the nested-loop and hash joins the paper builds.
//
// It takes the same work items as the hash join kernel: a chunk of at most
// cap R rows of one partition against every S row of that partition.
// k_sort_chunks sorts every R chunk by key once (bitonic network in shared
// memory) into a copy of the partitioned rows; the count and emit passes then
// stage the sorted chunk and each S row finds its run of equal R keys by two
// binary searches, which is the merge step done per probe row instead of by
// a second sorted stream.
//   count: item_val[it] = sum over S rows of the run length;
//   agg:   as count, and chk += sum over matches of f(r) * g(s), from a
//          prefix sum of f over the sorted run order;
//   emit:  the item's pairs at out[item_off[it] ...], (R payload, S payload).
#pragma once

#include "jn_common.cuh"
#include "jn_partition.cuh"

namespace jnx {

constexpr int SJ_T = 512;  // threads per sort-merge block

// Order-preserving unsigned image of a signed key, and back.
__device__ __forceinline__ uint32_t sj_ord(int32_t k) { return (uint32_t)k ^ 0x80000000u; }
__device__ __forceinline__ uint64_t sj_ord(int64_t k) { return (uint64_t)k ^ 0x8000000000000000ull; }
template <typename K>
__device__ __forceinline__ K sj_key(typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type u) {
    return sizeof(K) == 4 ? (K)(int32_t)((uint32_t)u ^ 0x80000000u) : (K)(int64_t)((uint64_t)u ^ 0x8000000000000000ull);
}

template <typename K>
struct SortJoinSmem {
    using U = typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type;
    // sort pass, int32 keys: packed words (order key, padding flag, row
    // index) and payloads; int64 keys: keys, row indices and payloads
    static size_t sort_bytes(int cap) {
        return sizeof(K) == 4 ? (size_t)cap * (sizeof(uint64_t) + sizeof(int32_t)) + 16
                              : (size_t)cap * (sizeof(U) + sizeof(uint16_t) + sizeof(int32_t)) + 16;
    }
    // join passes: the sorted chunk's keys and payloads, and (aggregate
    // mode) the prefix sum of f over it
    static size_t bytes(int cap, int mode) {
        return (size_t)cap * (sizeof(U) + sizeof(int32_t)) +
               (mode == MODE_AGG ? (size_t)(cap + 1) * sizeof(unsigned long long) : 0) + 16;
    }
};

// Sorts R rows [rbeg, rbeg + rn) of every item by key into `sorted` (same
// positions).  Shared memory: SortJoinSmem<K>::sort_bytes(cap).
template <typename K>
__global__ void __launch_bounds__(SJ_T)
k_sort_chunks(const Row<K, false>* __restrict__ rrows, Row<K, false>* __restrict__ sorted,
              const Item* __restrict__ items, const uint64_t* __restrict__ nitems_p, int cap) {
    using U = typename SortJoinSmem<K>::U;
    extern __shared__ __align__(128) unsigned char smem[];
    U* s_k = reinterpret_cast<U*>(smem);
    int32_t* s_pay = reinterpret_cast<int32_t*>(s_k + cap);
    uint16_t* s_i = reinterpret_cast<uint16_t*>(s_pay + cap);
    constexpr uint16_t PAD = 0x8000u;
    const uint64_t nitems = *nitems_p;
    for (uint64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item d = items[it];  // every item owns one R chunk
        const int rn = d.rn;
        int n2 = 1;
        while (n2 < rn) n2 <<= 1;
        for (int i = threadIdx.x; i < n2; i += SJ_T) {
            if (i < rn) {
                const Row<K, false> x = rrows[d.rbeg + i];
                s_k[i] = sj_ord(x.key);
                s_pay[i] = x.pay;
                s_i[i] = (uint16_t)i;
            } else {
                s_k[i] = ~(U)0;
                s_i[i] = (uint16_t)(PAD | i);
            }
        }
        __syncthreads();
        for (int k = 2; k <= n2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < (n2 >> 1); t += SJ_T) {
                    const int a = 2 * j * (t / j) + (t % j), b = a + j;
                    const U ka = s_k[a], kb = s_k[b];
                    const uint16_t ia = s_i[a], ib = s_i[b];
                    const bool gt = ka > kb || (ka == kb && (ia & PAD) > (ib & PAD));
                    if (gt == ((a & k) == 0)) {
                        s_k[a] = kb;
                        s_k[b] = ka;
                        s_i[a] = ib;
                        s_i[b] = ia;
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < rn; i += SJ_T) {
            Row<K, false> x{};
            x.key = sj_key<K>(s_k[i]);
            x.pay = s_pay[s_i[i] & (PAD - 1)];
            sorted[d.rbeg + i] = x;
        }
        __syncthreads();
    }
}

// Compare-exchange of bitonic stage (k, j) on the 8 consecutive elements a
// thread holds (element index i = 8 * thread + e), for j < 256: partners
// 8 or more apart sit in another lane of the same warp (shuffle), closer
// ones in the same thread.
template <int J>
__device__ __forceinline__ void sj_stage_thread(uint64_t (&v)[8], int t, int k) {
#pragma unroll
    for (int e = 0; e < 8; e++) {
        if (e & J) continue;
        const int e2 = e | J, i = 8 * t + e;
        const bool asc = (i & k) == 0;
        const uint64_t x = v[e], y = v[e2];
        const bool sw = (x > y) == asc;
        v[e] = sw ? y : x;
        v[e2] = sw ? x : y;
    }
}

__device__ __forceinline__ void sj_stage_regs(uint64_t (&v)[8], int t, int k, int j) {
    if (j >= 8) {
        const int lm = j >> 3;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int i = 8 * t + e;
            const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], lm);
            const bool asc = (i & k) == 0, lower = (i & j) == 0;
            v[e] = (asc == lower) ? (v[e] < o ? v[e] : o) : (v[e] > o ? v[e] : o);
        }
    } else if (j == 4) {
        sj_stage_thread<4>(v, t, k);
    } else if (j == 2) {
        sj_stage_thread<2>(v, t, k);
    } else {
        sj_stage_thread<1>(v, t, k);
    }
}

// int32 keys: the sort runs on packed words (order key << 16 | padding flag
// << 15 | row index), 8 per thread in registers.  Stages with j < 256 stay
// in a warp (shuffles); only the 10 stages with j >= 256 of a 4096-row chunk
// go through shared memory, one barrier each.
template <>
__global__ void __launch_bounds__(SJ_T)
k_sort_chunks<int32_t>(const Row<int32_t, false>* __restrict__ rrows, Row<int32_t, false>* __restrict__ sorted,
                       const Item* __restrict__ items, const uint64_t* __restrict__ nitems_p, int cap) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* s_v = reinterpret_cast<uint64_t*>(smem);  // cap words
    int32_t* s_pay = reinterpret_cast<int32_t*>(s_v + cap);
    const int t = threadIdx.x;
    const uint64_t nitems = *nitems_p;
    for (uint64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item d = items[it];  // every item owns one R chunk
        const int rn = d.rn;
        int n2 = 256;  // one warp's 8 x 32 elements at least
        while (n2 < rn) n2 <<= 1;
        const bool act = 8 * t < n2;  // whole warps: n2 is a multiple of 256
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int i = 8 * t + e;
            if (i < rn) {
                const Row<int32_t, false> x = rrows[d.rbeg + i];
                s_pay[i] = x.pay;
                v[e] = ((uint64_t)sj_ord(x.key) << 16) | (uint64_t)i;
            } else {
                v[e] = (0xffffffffull << 16) | 0x8000ull | (uint64_t)(i & 0x7fff);
            }
        }
        if (act)
            for (int k = 2; k <= 256; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) sj_stage_regs(v, t, k, j);
        for (int k = 512; k <= n2; k <<= 1) {
            if (act) {
#pragma unroll
                for (int e = 0; e < 8; e++) s_v[8 * t + e] = v[e];
            }
            __syncthreads();
            for (int j = k >> 1; j >= 256; j >>= 1) {
                for (int q = t; q < (n2 >> 1); q += SJ_T) {
                    const int a = 2 * j * (q / j) + (q % j), b = a + j;
                    const uint64_t x = s_v[a], y = s_v[b];
                    if ((x > y) == ((a & k) == 0)) {
                        s_v[a] = y;
                        s_v[b] = x;
                    }
                }
                __syncthreads();
            }
            if (act) {
#pragma unroll
                for (int e = 0; e < 8; e++) v[e] = s_v[8 * t + e];
                for (int j = 128; j > 0; j >>= 1) sj_stage_regs(v, t, k, j);
            }
        }
        __syncthreads();  // every row's payload is in shared memory
        if (act) {
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int i = 8 * t + e;
                if (i < rn) {
                    Row<int32_t, false> x;
                    x.key = (int32_t)((uint32_t)(v[e] >> 16) ^ 0x80000000u);
                    x.pay = s_pay[(int)(v[e] & 0x7fffull)];
                    sorted[d.rbeg + i] = x;
                }
            }
        }
        __syncthreads();  // shared arrays are rewritten by the next chunk
    }
}

template <typename K, int MODE>
__global__ void __launch_bounds__(SJ_T)
k_sort_join(const Row<K, false>* __restrict__ rrows, const Row<K, false>* __restrict__ srows,
            const Item* __restrict__ items, const uint64_t* __restrict__ nitems_p, int cap,
            unsigned long long* __restrict__ item_val, unsigned long long* __restrict__ chk,
            const uint64_t* __restrict__ item_off, jn_pair* __restrict__ out, uint64_t item_lo,
            uint64_t item_hi) {
    using U = typename SortJoinSmem<K>::U;
    extern __shared__ __align__(128) unsigned char smem[];
    U* s_k = reinterpret_cast<U*>(smem);
    unsigned long long* s_f = reinterpret_cast<unsigned long long*>(s_k + cap);  // agg only
    int32_t* s_pay = reinterpret_cast<int32_t*>(MODE == MODE_AGG ? reinterpret_cast<unsigned char*>(s_f + cap + 1)
                                                                 : reinterpret_cast<unsigned char*>(s_k + cap));
    __shared__ unsigned long long tmp64[33];
    __shared__ uint32_t s_cursor;

    const int lane = threadIdx.x & 31;
    const uint64_t nitems = min(*nitems_p, item_hi);
    for (uint64_t it = item_lo + blockIdx.x; it < nitems; it += gridDim.x) {
        const Item d = items[it];
        const int rn = d.rn;
        for (int i = threadIdx.x; i < rn; i += SJ_T) {  // the chunk, sorted by key
            const Row<K, false> x = rrows[d.rbeg + i];
            s_k[i] = sj_ord(x.key);
            s_pay[i] = x.pay;
        }
        if (threadIdx.x == 0) s_cursor = 0;
        __syncthreads();
        if (MODE == MODE_AGG) {
            // s_f[e] = sum of f(payload) over sorted positions < e, e <= rn
            constexpr int PER = 8;  // SJ_T * PER >= every chunk size
            const int base = threadIdx.x * PER;
            unsigned long long v[PER], sum = 0;
#pragma unroll
            for (int q = 0; q < PER; q++) {
                const int e = base + q;
                v[q] = (e < rn) ? chk_f(s_pay[e]) : 0ull;
                sum += v[q];
            }
            unsigned long long tot;
            unsigned long long pre = block_excl_scan(sum, tmp64, &tot);
            if (threadIdx.x == 0) s_f[0] = 0;
#pragma unroll
            for (int q = 0; q < PER; q++) {
                const int e = base + q;
                pre += v[q];
                if (e < rn) s_f[e + 1] = pre;
            }
            __syncthreads();
        }
        unsigned long long acc = 0, csum = 0;
        const int rounds = (d.sn + SJ_T - 1) / SJ_T;
        for (int r = 0; r < rounds; r++) {
            const int j = r * SJ_T + threadIdx.x;
            uint32_t lo = 0, hi = 0;
            int32_t spay = 0;
            if (j < d.sn) {
                const Row<K, false> x = srows[d.sbeg + j];
                const U q = sj_ord(x.key);
                spay = x.pay;
                uint32_t a = 0, b = (uint32_t)rn;  // first entry >= q
                while (a < b) {
                    const uint32_t mid = (a + b) >> 1;
                    if (s_k[mid] < q) a = mid + 1; else b = mid;
                }
                lo = a;
                b = (uint32_t)rn;  // first entry > q
                while (a < b) {
                    const uint32_t mid = (a + b) >> 1;
                    if (s_k[mid] <= q) a = mid + 1; else b = mid;
                }
                hi = a;
            }
            const uint32_t m = hi - lo;
            if (MODE == MODE_EMIT) {
                const uint32_t incl = warp_incl_scan(m);
                const uint32_t wt = __shfl_sync(0xffffffffu, incl, 31);
                uint32_t wbase = 0;
                if (lane == 0 && wt) wbase = atomicAdd(&s_cursor, wt);
                wbase = __shfl_sync(0xffffffffu, wbase, 0);
                const uint64_t o = item_off[it] + wbase + (incl - m);
                // short runs by their lane, long runs by the whole warp
                const bool longr = m > 4;
                if (!longr)
                    for (uint32_t e = 0; e < m; e++) st_pair(out + o + e, s_pay[lo + e], spay);
                for (unsigned lanes = __ballot_sync(0xffffffffu, longr); lanes; lanes &= lanes - 1) {
                    const int src = __ffs(lanes) - 1;
                    const uint32_t bm = __shfl_sync(0xffffffffu, m, src);
                    const uint32_t bl = __shfl_sync(0xffffffffu, lo, src);
                    const int32_t bp = __shfl_sync(0xffffffffu, spay, src);
                    const uint64_t bo = __shfl_sync(0xffffffffu, o, src);
                    for (uint32_t e = lane; e < bm; e += 32)
                        st_pair(out + bo + e, s_pay[bl + e], bp);
                }
            } else {
                acc += m;
                if (MODE == MODE_AGG && m) csum += (s_f[hi] - s_f[lo]) * chk_g(spay);
            }
        }
        if (MODE != MODE_EMIT) {
            const unsigned long long t = block_sum(acc, tmp64);
            if (MODE == MODE_AGG) {
                const unsigned long long cs = block_sum(csum, tmp64);
                if (threadIdx.x == 0 && cs) atomicAdd(chk, cs);
            }
            if (threadIdx.x == 0) item_val[it] = t;
        }
        __syncthreads();  // the chunk's shared arrays are rewritten by the next item
    }
}

}  // namespace jnx
