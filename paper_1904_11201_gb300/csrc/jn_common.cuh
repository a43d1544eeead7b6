// Shared internals of libjn: context, launch helper, device primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <vector>

#include "jn.h"

namespace jnx {

// ------------------------------------------------------------ kernel ids --
enum KernelId {
    K_MEMSET = 0,
    K_PRESENCE,
    K_HIST,
    K_SCATTER,
    K_SEGMENTS,
    K_ITEMS,
    K_HASH_COUNT,
    K_HASH_EMIT,
    K_HEAVY_SAMPLE,
    K_HEAVY_SELECT,
    K_CROSS_EMIT,
    K_SCAN_REDUCE,
    K_SCAN_TOP,
    K_SCAN_DOWN,
    K_NLJ_COUNT,
    K_NLJ_EMIT,
    K_MINMAX,
    K_THETA_COUNT,
    K_THETA_EMIT,
    K_GATHER,
    K_BATCH,
    K_MISC,
    K_SORT_COUNT,
    K_SORT_EMIT,
    K_SORT_CHUNKS,
    K_CHUNK_HIST,
    K_REGION1,
    K_REGION2,
    K_THETA_GATHER,
    K_STAR,
    K_COUNT_IDS
};

const char* kernel_name(int kid);

struct PendingTiming {
    int kid;
    cudaEvent_t start, stop;
};

struct KernelStat {
    uint64_t launches = 0;
    double ms = 0.0;
};

}  // namespace jnx

struct jn_ctx {
    int device = 0;
    int num_sms = 0;     // SMs the grids are sized for (tuning `sms`, else all)
    int device_sms = 0;  // SMs of the device
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;  // the device's default pool (never destroyed)
    jn_tuning tune{};
    uint64_t* h_small = nullptr;  // pinned host words for count read-back
    unsigned int* d_err = nullptr;  // device error word (bounded waits that ran out)
    cudaStream_t capture_stream = nullptr;  // private stream for CUDA-graph capture
    bool profiling = false;
    std::vector<jnx::PendingTiming> pending;
    std::vector<cudaEvent_t> spare_events;
    jnx::KernelStat stats[jnx::K_COUNT_IDS];
    uint64_t launches_total = 0;
    uint64_t launches_at_call = 0;
    std::string err;
    jn_run_info info{};
    cudaStream_t copy_stream = nullptr;  // private stream for host-column copies
    cudaEvent_t copied_keys = nullptr;   // this run's host key columns have landed (or NULL)
    cudaEvent_t copied_r = nullptr;      // ... and every column of its first table (or NULL)
    cudaEvent_t copied_all = nullptr;    // every host column of this run has landed (or NULL)
    uint64_t scratch_bytes = 0;  // bytes held by live Scratch sets
    uint64_t mem_limit = 0;      // admission: output + scratch bound (0 = none)
    jn_admit_fn admit = nullptr;
    void* admit_user = nullptr;
};

namespace jnx {

// ----------------------------------------------------------- host errors --
jn_status fail(jn_ctx* c, jn_status s, const std::string& msg);
jn_status cuda_fail(jn_ctx* c, cudaError_t e, const char* what);

#define JN_CUDA(c, expr)                                             \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return ::jnx::cuda_fail((c), _e, #expr); \
    } while (0)

#define JN_TRY(expr)                     \
    do {                                 \
        jn_status _s = (expr);           \
        if (_s != JN_OK) return _s;      \
    } while (0)

// -------------------------------------------------------- device memory --
// Stream-ordered allocations from the context's pool.
jn_status dalloc(jn_ctx* c, void** p, size_t bytes);
void dfree(jn_ctx* c, void* p);

// A bundle of scratch buffers released together at scope exit.
struct Scratch {
    jn_ctx* c;
    std::vector<void*> ptrs;
    uint64_t held = 0;
    explicit Scratch(jn_ctx* ctx) : c(ctx) {}
    ~Scratch() {
        for (void* p : ptrs) dfree(c, p);
        c->scratch_bytes -= held;
    }
    template <typename T>
    jn_status get(T** p, size_t count) {
        void* q = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        jn_status s = dalloc(c, &q, bytes);
        if (s != JN_OK) return s;
        ptrs.push_back(q);
        held += bytes;
        c->scratch_bytes += bytes;
        if (c->scratch_bytes > c->info.scratch_peak) c->info.scratch_peak = c->scratch_bytes;
        *p = static_cast<T*>(q);
        return JN_OK;
    }
};

jn_status zero(jn_ctx* c, void* p, size_t bytes);

// --------------------------------------------------------------- launch --
cudaEvent_t take_event(jn_ctx* c);
void ensure_smem(const void* fn, size_t smem);

template <typename Kern, typename... Args>
jn_status launch(jn_ctx* c, int kid, Kern kern, dim3 grid, dim3 block, size_t smem,
                 Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return JN_OK;
    if (smem > 0) ensure_smem(reinterpret_cast<const void*>(kern), smem);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
        e0 = take_event(c);
        e1 = take_event(c);
        cudaEventRecord(e0, c->stream);
    }
    kern<<<grid, block, smem, c->stream>>>(args...);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, kernel_name(kid));
    c->stats[kid].launches++;
    c->launches_total++;
    if (c->profiling) {
        cudaEventRecord(e1, c->stream);
        c->pending.push_back({kid, e0, e1});
    }
    return JN_OK;
}

// Read `n` u64 words from device to host (synchronises the stream).
jn_status read_back(jn_ctx* c, const uint64_t* dsrc, uint64_t* hdst, int n);

// Exclusive scan: out[i] = sum(in[0..i-1]) for i in [0, n]; out has n + 1 words.
jn_status scan_u32(jn_ctx* c, const uint32_t* in, uint64_t* out, int64_t n);
jn_status scan_u64(jn_ctx* c, const uint64_t* in, uint64_t* out, int64_t n);

// Host-side column staging: returns a device pointer for a column that may
// be host memory (copied into scratch) or device memory (returned as is).
jn_status device_column(jn_ctx* c, Scratch& s, const void* p, size_t bytes, const void** dp);
// Device address of page-locked host memory the kernels may read and write
// in place (over the CPU-GPU link), or NULL for any other pointer.
const void* host_mapped(const void* p);
// Host columns are copied on the context's copy stream, key columns first;
// a run waits for the keys before its first key read and for the rest before
// it needs them (so the first passes overlap the remaining copies).
jn_status wait_copies(jn_ctx* c, bool all);
jn_status wait_copies_r(jn_ctx* c);  // the keys and the first table's other columns
bool is_device_pointer(const void* p);
int pointer_device(const void* p);  // device of device (or managed) memory, else -1

// ------------------------------------------------------------- helpers --
inline int ceil_log2(uint64_t x) {
    int b = 0;
    while ((uint64_t(1) << b) < x) b++;
    return b;
}
inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// ----------------------------------------------------- device primitives --
// Key hash.  Multiplicative hashing by an odd constant (Knuth); partition
// digits take the top bits, shared-memory bucket bits the bits below them.
__device__ __forceinline__ uint32_t khash(int32_t k) { return (uint32_t)k * 0x9E3779B1u; }
__device__ __forceinline__ uint32_t khash(int64_t k) {
    return (uint32_t)(((uint64_t)k * 0x9E3779B97F4A7C15ull) >> 32);
}

// Bit of the key-presence filter: the low bits of the key itself, so a key
// domain that fits the bitmap is filtered exactly.
__device__ __forceinline__ uint32_t fbits(int32_t k) { return (uint32_t)k; }
__device__ __forceinline__ uint32_t fbits(int64_t k) {
    return (uint32_t)k ^ (uint32_t)((uint64_t)k >> 32);
}

// Separable checksum mixers: f(x) = mix(C1 ^ x), g(x) = mix(C2 ^ x), mix =
// the SplitMix64 output mixer (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t chk_f(int32_t r) {
    return mix64(0x243F6A8885A308D3ull ^ (uint64_t)(uint32_t)r);
}
__device__ __forceinline__ uint64_t chk_g(int32_t s) {
    return mix64(0x13198A2E03707344ull ^ (uint64_t)(uint32_t)s);
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide exclusive scan of one value per thread.  `tmp` needs 33 words.
// Returns the exclusive prefix; *total receives the block total.  All threads
// of the block must call it.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < nwarps) ? tmp[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < nwarps) tmp[lane] = wi - w;
        if (lane == 31) tmp[32] = wi;
    }
    __syncthreads();
    T r = tmp[warp] + inc - v;
    *total = tmp[32];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* tmp) {
    T t;
    block_excl_scan(v, tmp, &t);
    return t;
}

// Adds the warp's total of v to *dst (one atomic per warp; every lane calls).
__device__ __forceinline__ void warp_add_to(unsigned long long* dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Stores one result pair as a single 8-byte word.  Every pair buffer a kernel
// writes is 8-byte aligned: library allocations and scratch are, and a caller
// buffer off that boundary is filled by a copy from aligned scratch.
__device__ __forceinline__ void st_pair(jn_pair* p, int32_t r, int32_t s) {
    *reinterpret_cast<int2*>(p) = make_int2(r, s);
}

// Membership of x in [lo, hi] for signed integers, by one unsigned compare:
// x in [lo, hi] <=> (x - lo) mod 2^w <= (hi - lo) mod 2^w, valid when lo <= hi.
__device__ __forceinline__ bool in_range(int32_t x, int32_t lo, uint32_t span) {
    return (uint32_t)x - (uint32_t)lo <= span;
}
__device__ __forceinline__ bool in_range(int64_t x, int64_t lo, uint64_t span) {
    return (uint64_t)x - (uint64_t)lo <= span;
}

// "R.x op s" as "R.x in [lo, hi] XOR inv" (an empty set is the inverted full
// range).  Exact for every op and every s, including the type's extremes.
template <typename K>
struct Interval {
    K lo;
    typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type span;
    bool inv;
};

template <typename K>
__device__ __forceinline__ Interval<K> op_interval(int op, K s) {
    using U = typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type;
    const K kmin = sizeof(K) == 4 ? (K)INT32_MIN : (K)INT64_MIN;
    const K kmax = sizeof(K) == 4 ? (K)INT32_MAX : (K)INT64_MAX;
    Interval<K> iv;
    K lo = kmin, hi = kmax;
    bool inv = false;
    switch (op) {
        case JN_EQ: lo = s; hi = s; break;
        case JN_NE: lo = s; hi = s; inv = true; break;
        case JN_LT:
            if (s == kmin) { inv = true; } else { hi = (K)(s - 1); }
            break;
        case JN_LE: hi = s; break;
        case JN_GT:
            if (s == kmax) { inv = true; } else { lo = (K)(s + 1); }
            break;
        case JN_GE: lo = s; break;
        default: break;  // JN_ANY: full range
    }
    iv.lo = lo;
    iv.span = (U)hi - (U)lo;
    iv.inv = inv;
    return iv;
}

// |R.k - s| <= band as an interval [s - band, s + band] clamped to the type.
template <typename K>
__device__ __forceinline__ Interval<K> band_interval(K s, int64_t band) {
    using U = typename std::conditional<sizeof(K) == 4, uint32_t, uint64_t>::type;
    Interval<K> iv;
    iv.inv = false;
    if (sizeof(K) == 4) {
        int64_t lo = (int64_t)s - band, hi = (int64_t)s + band;
        if (lo < INT32_MIN) lo = INT32_MIN;
        if (hi > INT32_MAX) hi = INT32_MAX;
        iv.lo = (K)lo;
        iv.span = (U)((K)hi) - (U)((K)lo);
    } else {
        // band >= 0, so INT64_MIN + band and INT64_MAX - band do not overflow
        int64_t lo = ((int64_t)s < INT64_MIN + band) ? INT64_MIN : (int64_t)s - band;
        int64_t hi = ((int64_t)s > INT64_MAX - band) ? INT64_MAX : (int64_t)s + band;
        iv.lo = (K)lo;
        iv.span = (U)hi - (U)lo;
    }
    return iv;
}

template <typename K>
__device__ __forceinline__ bool iv_test(const Interval<K>& iv, K x) {
    return in_range(x, iv.lo, iv.span) != iv.inv;
}

}  // namespace jnx
