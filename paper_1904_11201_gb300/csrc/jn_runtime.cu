// libjn runtime: contexts, errors, memory, scans, statistics.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <map>
#include <set>

#include "jn_async.cuh"
#include "jn_common.cuh"

namespace jnx {

static const char* kKernelNames[K_COUNT_IDS] = {
    "memset",       "presence",     "histogram",   "scatter",     "segments",
    "work_items",   "hash_count",   "hash_emit",   "heavy_sample", "heavy_select",
    "cross_emit",   "scan_reduce",  "scan_top",    "scan_down",   "nlj_count",
    "nlj_emit",     "minmax",       "theta_count", "theta_emit",  "gather",
    "batch",        "misc",         "sort_count",  "sort_emit",   "sort_chunks",
    "chunk_hist",   "region1",      "region2",     "theta_gather", "star"};

const char* kernel_name(int kid) {
    return (kid >= 0 && kid < K_COUNT_IDS) ? kKernelNames[kid] : "?";
}

jn_status fail(jn_ctx* c, jn_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

jn_status cuda_fail(jn_ctx* c, cudaError_t e, const char* what) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // not sticky: clear it
        return fail(c, JN_ERR_OOM, buf);
    }
    return fail(c, JN_ERR_CUDA, buf);
}

jn_status dalloc(jn_ctx* c, void** p, size_t bytes) {
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(c, e, "device allocation");
    }
    return JN_OK;
}

void dfree(jn_ctx* c, void* p) {
    if (p) cudaFreeAsync(p, c->stream);
}

jn_status zero(jn_ctx* c, void* p, size_t bytes) {
    if (bytes == 0) return JN_OK;
    JN_CUDA(c, cudaMemsetAsync(p, 0, bytes, c->stream));
    return JN_OK;
}

cudaEvent_t take_event(jn_ctx* c) {
    if (!c->spare_events.empty()) {
        cudaEvent_t e = c->spare_events.back();
        c->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Raises a kernel's dynamic shared-memory limit to at least `smem`; never
// lowers it (a lower limit would refuse later, larger launches of the kernel).
// Without the attribute, static and dynamic shared memory together may not
// pass 48 KB; the first call for a kernel records how much dynamic memory
// that default leaves it.
void ensure_smem(const void* fn, size_t smem) {
    static std::mutex mu;
    static std::map<const void*, size_t> limit;  // dynamic bytes a launch may use now
    std::lock_guard<std::mutex> g(mu);
    auto it = limit.find(fn);
    if (it == limit.end()) {
        cudaFuncAttributes fa;
        size_t dflt = 0;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.sharedSizeBytes < 48 * 1024)
            dflt = 48 * 1024 - fa.sharedSizeBytes;
        else
            cudaGetLastError();
        it = limit.emplace(fn, dflt).first;
    }
    if (it->second >= smem) return;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return;  // the launch reports the error
    }
    limit[fn] = smem;
}

jn_status read_back(jn_ctx* c, const uint64_t* dsrc, uint64_t* hdst, int n) {
    if (n > 0)
        JN_CUDA(c, cudaMemcpyAsync(c->h_small, dsrc, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost,
                                   c->stream));
    JN_CUDA(c, cudaMemcpyAsync(c->h_small + 63, c->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                               c->stream));
    JN_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n; i++) hdst[i] = c->h_small[i];
    const unsigned int e = (unsigned int)(c->h_small[63] & 0xffffffffu);
    if (e != 0) {
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream);
        return fail(c, (jn_status)e, "a bounded device-side wait ran out");
    }
    return JN_OK;
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pointer_device(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

const void* host_mapped(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

jn_status wait_copies(jn_ctx* c, bool all) {
    cudaEvent_t e = all ? c->copied_all : c->copied_keys;
    if (e) JN_CUDA(c, cudaStreamWaitEvent(c->stream, e, 0));
    return JN_OK;
}

jn_status wait_copies_r(jn_ctx* c) {
    if (c->copied_r) JN_CUDA(c, cudaStreamWaitEvent(c->stream, c->copied_r, 0));
    return JN_OK;
}

jn_status device_column(jn_ctx* c, Scratch& s, const void* p, size_t bytes, const void** dp) {
    if (p == nullptr || bytes == 0 || is_device_pointer(p)) {
        *dp = p;
        return JN_OK;
    }
    uint8_t* d = nullptr;
    JN_TRY(s.get(&d, bytes));
    JN_CUDA(c, cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, c->stream));
    *dp = d;
    return JN_OK;
}

// ------------------------------------------------------------------ scan --
// Three-phase exclusive scan: per-block sums, one block scanning the sums,
// then each block scanning its chunk from its carry.  4096 values per block.
constexpr int SCAN_T = 1024;
constexpr int SCAN_V = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_V;

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, uint64_t* __restrict__ sums) {
    __shared__ uint64_t tmp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < SCAN_V; j++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_V + j;
        if (i < n) v += (uint64_t)in[i];
    }
    uint64_t t = block_sum(v, tmp);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// One block scans in[0..n) with a running carry; out[n] = total.  With
// `carry_in` != nullptr, each block's carry comes from carry_in[blockIdx.x]
// (the down-sweep over chunks of SCAN_CHUNK).
template <typename T>
__global__ void k_scan_chunks(const T* __restrict__ in, int64_t n, uint64_t* __restrict__ out,
                              const uint64_t* __restrict__ carry_in) {
    __shared__ uint64_t tmp[33];
    uint64_t carry = carry_in ? carry_in[blockIdx.x] : 0;
    int64_t begin = carry_in ? (int64_t)blockIdx.x * SCAN_CHUNK : 0;
    int64_t end = carry_in ? min(n, begin + SCAN_CHUNK) : n;
    for (int64_t base = begin; base < end; base += SCAN_CHUNK) {
        uint64_t v[SCAN_V];
        uint64_t local = 0;
#pragma unroll
        for (int j = 0; j < SCAN_V; j++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_V + j;
            v[j] = (i < end) ? (uint64_t)in[i] : 0;
            local += v[j];
        }
        uint64_t total;
        uint64_t pre = block_excl_scan(local, tmp, &total) + carry;
#pragma unroll
        for (int j = 0; j < SCAN_V; j++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_V + j;
            if (i < end) out[i] = pre;
            pre += v[j];
        }
        carry += total;
    }
    if (threadIdx.x == 0 && end == n) out[n] = carry;
}

template <typename T>
static jn_status scan_impl(jn_ctx* c, const T* in, uint64_t* out, int64_t n) {
    if (n <= 8 * SCAN_CHUNK) {
        return launch(c, K_SCAN_TOP, k_scan_chunks<T>, dim3(1), dim3(SCAN_T), 0, in, n, out,
                      (const uint64_t*)nullptr);
    }
    int64_t nb = (int64_t)ceil_div(n, SCAN_CHUNK);
    Scratch s(c);
    uint64_t *sums = nullptr, *pre = nullptr;
    JN_TRY(s.get(&sums, nb));
    JN_TRY(s.get(&pre, nb + 1));
    JN_TRY(launch(c, K_SCAN_REDUCE, k_scan_reduce<T>, dim3((unsigned)nb), dim3(SCAN_T), 0, in, n,
                  sums));
    JN_TRY(scan_impl<uint64_t>(c, sums, pre, nb));
    JN_TRY(launch(c, K_SCAN_DOWN, k_scan_chunks<T>, dim3((unsigned)nb), dim3(SCAN_T), 0, in, n,
                  out, (const uint64_t*)pre));
    return JN_OK;
}

jn_status scan_u32(jn_ctx* c, const uint32_t* in, uint64_t* out, int64_t n) {
    return scan_impl<uint32_t>(c, in, out, n);
}
jn_status scan_u64(jn_ctx* c, const uint64_t* in, uint64_t* out, int64_t n) {
    return scan_impl<uint64_t>(c, in, out, n);
}

}  // namespace jnx
#include "jn_algos.h"
namespace jnx {

GraphPhase::~GraphPhase() {
    abort();
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
}

jn_status GraphPhase::begin() {
    if (!on) return JN_OK;
    if (!c->capture_stream) JN_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    user = c->stream;
    c->stream = c->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->stream = user;
        user = nullptr;
        return cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    return JN_OK;
}

jn_status GraphPhase::end_and_run() {
    if (!on) return JN_OK;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->stream = user;
    user = nullptr;
    JN_CUDA(c, e);
    JN_CUDA(c, cudaGraphInstantiate(&x, g, 0));
    JN_CUDA(c, cudaGraphLaunch(x, c->stream));
    return JN_OK;
}

void GraphPhase::abort() {
    if (!on || !user) return;
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(c->stream, &junk);
    if (junk) cudaGraphDestroy(junk);
    c->stream = user;
    user = nullptr;
    cudaGetLastError();
}

static void resolve_pending(jn_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) c->stats[p.kid].ms += ms;
        c->spare_events.push_back(p.start);
        c->spare_events.push_back(p.stop);
    }
    c->pending.clear();
    cudaGetLastError();
}

}  // namespace jnx

using namespace jnx;

// One block waits on the first phase of an mbarrier that expects one
// arrival; with `arrive` set, thread 0 arrives before the wait.  Writes the
// wait's device time to *ns.
__global__ void k_wait_selftest(unsigned int* err, uint32_t polls, int32_t arrive, uint64_t* ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && arrive) mbar_arrive(&bar);
    uint64_t t0 = 0, t1 = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    mbar_wait_polls(&bar, 0, err, polls);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    __syncthreads();
    if (threadIdx.x == 0) *ns = t1 - t0;
}

extern "C" {

const char* jn_version(void) { return "jn 0.1 (sm_103a)"; }

const char* jn_status_str(jn_status s) {
    switch (s) {
        case JN_OK: return "ok";
        case JN_ERR_INVALID: return "invalid argument";
        case JN_ERR_OOM: return "out of device memory";
        case JN_ERR_CAPACITY: return "output buffer too small";
        case JN_ERR_CUDA: return "CUDA error";
        case JN_ERR_TIMEOUT: return "device wait timed out";
        case JN_ERR_UNSUPPORTED: return "unsupported predicate or mode";
    }
    return "unknown status";
}

const char* jn_last_error(const jn_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

static void default_tuning(jn_tuning* t) {
    memset(t, 0, sizeof(*t));
    t->prefilter = -1;
    t->heavy = -1;
}

jn_status jn_create(jn_ctx** out, int device, void* stream) {
    if (!out) return JN_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return JN_ERR_INVALID;
    }
    jn_ctx* c = new jn_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    default_tuning(&c->tune);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) {
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, device);
        c->num_sms = c->device_sms = prop.multiProcessorCount;
        c->smem_optin = prop.sharedMemPerBlockOptin;
    }
    if (e == cudaSuccess) {
        // Outputs may outlive the context (jn_free accepts a NULL context), so
        // allocations come from the device's default pool, which lives as long
        // as the process; freed blocks are kept for reuse by later calls.
        e = cudaDeviceGetDefaultMemPool(&c->pool, device);
    }
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) {
        // A block freed on one stream is never handed to an allocation on
        // another by making that stream wait for the free: contexts on their
        // own streams (server workers) would otherwise queue behind each
        // other's joins.  Reuse on the same stream, or of a free already
        // complete, stays allowed.
        int no = 0;
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_small, 64 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->h_small) cudaFreeHost(c->h_small);
        if (c->d_err) cudaFree(c->d_err);
        delete c;
        return JN_ERR_CUDA;
    }
    *out = c;
    return JN_OK;
}

void jn_destroy(jn_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    resolve_pending(c);
    for (cudaEvent_t e : c->spare_events) cudaEventDestroy(e);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->d_err) cudaFree(c->d_err);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    cudaGetLastError();
    delete c;
}

jn_status jn_set_stream(jn_ctx* c, void* stream) {
    if (!c) return JN_ERR_INVALID;
    c->stream = (cudaStream_t)stream;
    return JN_OK;
}

jn_status jn_set_tuning(jn_ctx* c, const jn_tuning* t) {
    if (!c) return JN_ERR_INVALID;
    if (!t) {
        default_tuning(&c->tune);
        c->num_sms = c->device_sms;
        return JN_OK;
    }
    if (t->prefilter < -1 || t->prefilter > 3 || t->radix_bits < 0 || t->radix_bits > 20 || t->radix_bits1 < 0 || t->radix_bits1 > 10 ||
        t->filter_bits < 0 || t->filter_bits > 30 || t->theta_groups < 0 || t->theta_groups > 10 ||
        t->nlj_tile_r < 0 || (t->nlj_tile_r % 256) != 0 || t->nlj_tile_r > 4096 || t->part_rows < 0 ||
        t->host_io < 0 || t->host_io > 3 || t->hash_path < 0 || t->hash_path > 2 ||
        (t->table_rows != 0 && t->table_rows != 1024 && t->table_rows != 2048 && t->table_rows != 4096) ||
        t->sms < 0)
        return fail(c, JN_ERR_INVALID, "tuning value out of range");
    c->tune = *t;
    c->num_sms = t->sms > 0 && t->sms < c->device_sms ? t->sms : c->device_sms;
    return JN_OK;
}

jn_status jn_get_tuning(const jn_ctx* c, jn_tuning* t) {
    if (!c || !t) return JN_ERR_INVALID;
    *t = c->tune;
    return JN_OK;
}

void jn_free(jn_ctx* c, jn_pair* p) {
    if (p) cudaFreeAsync(p, c ? c->stream : (cudaStream_t)0);
}

jn_status jn_set_memory_limit(jn_ctx* c, uint64_t bytes) {
    if (!c) return JN_ERR_INVALID;
    c->mem_limit = bytes;
    return JN_OK;
}

jn_status jn_set_admission(jn_ctx* c, jn_admit_fn fn, void* user) {
    if (!c) return JN_ERR_INVALID;
    c->admit = fn;
    c->admit_user = user;
    return JN_OK;
}

jn_status jn_set_profiling(jn_ctx* c, int32_t on) {
    if (!c) return JN_ERR_INVALID;
    c->profiling = on != 0;
    return JN_OK;
}

jn_status jn_kernel_stats(jn_ctx* c, jn_kernel_stat* out, int32_t max, int32_t* n) {
    if (!c || !n || (max > 0 && !out)) return JN_ERR_INVALID;
    JN_CUDA(c, cudaStreamSynchronize(c->stream));
    resolve_pending(c);
    int k = 0;
    for (int i = 0; i < K_COUNT_IDS && k < max; i++) {
        if (c->stats[i].launches == 0) continue;
        memset(&out[k], 0, sizeof(out[k]));
        strncpy(out[k].name, kernel_name(i), sizeof(out[k].name) - 1);
        out[k].launches = c->stats[i].launches;
        out[k].ms = c->stats[i].ms;
        k++;
    }
    *n = k;
    return JN_OK;
}

jn_status jn_reset_stats(jn_ctx* c) {
    if (!c) return JN_ERR_INVALID;
    JN_CUDA(c, cudaStreamSynchronize(c->stream));
    resolve_pending(c);
    for (int i = 0; i < K_COUNT_IDS; i++) c->stats[i] = KernelStat();
    return JN_OK;
}

jn_status jn_last_run_info(const jn_ctx* c, jn_run_info* info) {
    if (!c || !info) return JN_ERR_INVALID;
    *info = c->info;
    return JN_OK;
}

uint64_t jn_launch_count(const jn_ctx* c) { return c ? c->launches_total : 0; }

int32_t jn_pointer_is_device(const void* p) { return p && is_device_pointer(p) ? 1 : 0; }

jn_status jn_selftest_wait(jn_ctx* c, uint32_t polls, int32_t arrive, uint64_t* elapsed_ns) {
    if (!c || polls < 1 || polls > (1u << 20) || (arrive != 0 && arrive != 1)) return JN_ERR_INVALID;
    c->err.clear();
    Scratch s(c);
    uint64_t* d_ns = nullptr;
    jn_status st = s.get(&d_ns, 1);
    if (st != JN_OK) return st;
    st = launch(c, K_MISC, k_wait_selftest, dim3(1), dim3(32), 0, c->d_err, polls, arrive, d_ns);
    if (st != JN_OK) return st;
    uint64_t ns = 0;
    st = read_back(c, d_ns, &ns, 1);
    if (elapsed_ns) *elapsed_ns = ns;
    return st;
}

}  // extern "C"
