// Device-side helpers shared by the library's kernels: status bits, mbarrier
// and bulk-copy (TMA) wrappers in inline PTX for sm_103a, bounded waits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cgh {

// Bits latched in the context's device status word.
enum : int {
    kStatusInput = 1,     // bad point data (z <= 0, NaN, non-integer or out-of-range x/y)
    kStatusTimeout = 2,   // a bounded device-side wait ran out
    kStatusBounds = 4,    // a bounds check of the debug build (CGH_DEBUG) failed; the access was skipped
};

// Debug build (-DCGH_DEBUG): an index that holds by construction is checked, and a failure latches
// kStatusBounds (the caller skips the access) instead of faulting.  Release builds compile it to true.
#ifdef CGH_DEBUG
#define CGH_DCHECK(cond, status) ((cond) ? true : (atomicOr((status), ::cgh::kStatusBounds), false))
#else
#define CGH_DCHECK(cond, status) true
#endif

// Layout of the prepared points (one entry per point, padded with zero-amplitude
// points to a multiple of the point tile).
//   geo[j] = {x_j, y_j, C_hi, C_lo}, C = round(frac(c_j) 2^64), c_j = p^2/(2 lambda z_j)
//   aux[j] = {Delta_j, bits of A_j}, Delta_j = top 32 bits of (2 C mod 2^64)
// x_j, y_j are integers with |x|, |y| <= 16384, so every squared distance the
// kernels form stays below 2^31 and the 64-bit products are exact modulo 2^64.
constexpr int kMaxCoord = 16384;
constexpr int kMaxSide = 16384;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// timeout_ns of global time.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns)
{
    const uint32_t a = smem_addr(bar);
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(a, parity)) return true;
        if (global_timer_ns() - t0 > timeout_ns) return false;
    }
}

// Acquire load of a counter another SM updates (never a stale L1 line).
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded spin of one thread until *count >= need; false when timeout_ns of global time ran out.
__device__ __forceinline__ bool wait_count(const int *count, int need, unsigned long long timeout_ns)
{
    if (ld_acquire(count) >= need) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        __nanosleep(200);
        if (ld_acquire(count) >= need) return true;
        if (global_timer_ns() - t0 > timeout_ns) return false;
    }
}

// 1-D bulk copy (TMA, non-tensor) global -> shared; completes tx bytes on bar.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace cgh
