// Asynchronous staging helpers for sm_103a: 1-D TMA bulk copies
// (cp.async.bulk global -> shared) completed on an mbarrier, with bounded
// waits.  A wait that runs out of iterations records JN_ERR_TIMEOUT in a
// device error word instead of spinning forever.
#pragma once

#include "jn_common.cuh"

namespace jnx {

// Iterations of mbarrier.try_wait before a wait is declared failed.  Each
// try_wait on an incomplete phase suspends for a hardware-chosen time,
// measured at about 3.8 us on GB300, so the limit is about 2 s: far above
// any bulk copy of a staging buffer, short enough that a lost copy frees
// the GPU quickly.
constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 19;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` for at most `polls` polls; false (and
// *err set to JN_ERR_TIMEOUT) when the phase has not completed by then.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, uint32_t parity, unsigned int* err, uint32_t polls) {
    for (uint32_t i = 0; i < polls; i++)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicExch(err, (unsigned int)JN_ERR_TIMEOUT);
    return false;
}

// The wait every pipeline uses: MBAR_SPIN_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned int* err) {
    return mbar_wait_polls(bar, parity, err, MBAR_SPIN_LIMIT);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses to the same buffer.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy of `bytes` (multiple of 16) from global `src` (16-byte
// aligned) to shared `dst` (16-byte aligned), completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Rows [beg, beg + cnt) of an array of E-byte elements, widened to 16-byte
// boundaries: the copy starts at row a0 = beg rounded down and spans `bytes`.
// `rows_ok` is how many rows of the array may be read (allocation size);
// returns false when the widened range would pass it or the base is not
// 16-byte aligned.
template <int E>
__device__ __forceinline__ bool aligned_span(const void* base, uint64_t beg, uint64_t cnt, uint64_t rows_ok,
                                             uint64_t* a0, uint32_t* bytes) {
    constexpr uint64_t per = 16 / E;
    const uint64_t lo = beg & ~(per - 1);
    const uint64_t hi = (beg + cnt + per - 1) & ~(per - 1);
    if ((((uintptr_t)base) & 15) != 0 || hi > rows_ok) return false;
    *a0 = lo;
    *bytes = (uint32_t)((hi - lo) * E);
    return true;
}

}  // namespace jnx
