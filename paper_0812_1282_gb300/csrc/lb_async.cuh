// Asynchronous bulk copies (TMA, cp.async.bulk) and mbarriers, sm_90+ PTX.
//
// Every wait is bounded in wall time: the waiter records the failure in a
// device error word and gives up, so a lost completion can never hang the
// GPU; the host turns the word into LB_ERR_TIMEOUT.
#pragma once

#include <cstdint>

namespace lbfe {

constexpr unsigned kErrTimeout = 1u;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) writes to it
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// plain arrival (release semantics) on a barrier
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
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

// Same test, but a thread that finds the phase incomplete sleeps until it
// completes or about `ns` nanoseconds pass (no busy polling).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity; bounded.  Gives up
// after kWaitNs of wall time, or when another waiter already recorded a
// failure, so a lost completion costs at most one timeout per waiter rather
// than a hang.  Returns false (and sets bit kErrTimeout of *err) when it
// gives up.
//
// The polls themselves suspend in hardware until the phase completes or a
// short time passes.  The clock and the error word (a global load, about a
// microsecond) are consulted only every kPollCheck polls: most waits here
// end within a few polls, and a load on that path would delay every
// pipeline meeting by its latency.
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;
constexpr unsigned kPollCheck = 32;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err)
{
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = 0;
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (n % kPollCheck == 0) {
            const unsigned long long now = global_ns();
            if (n == kPollCheck) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                if (err) atomicOr(err, kErrTimeout);
                return false;
            }
            if (err && *reinterpret_cast<volatile unsigned*>(err)) return false;
        }
    }
}

// Wait of a thread that is not on the critical path (the producer warp,
// several stages ahead of its consumers): the same bounded test, with a
// pause of about `ns` nanoseconds between polls so that the waiting warp
// leaves its issue slots to the compute warps.
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* bar, uint32_t parity, unsigned* err,
                                               unsigned ns = 128)
{
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = 0;
    for (unsigned n = 1;; ++n) {
        __nanosleep(ns);
        if (mbar_try_wait(bar, parity)) return true;
        if (n % kPollCheck == 0) {
            const unsigned long long now = global_ns();
            if (n == kPollCheck) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                if (err) atomicOr(err, kErrTimeout);
                return false;
            }
            if (err && *reinterpret_cast<volatile unsigned*>(err)) return false;
        }
    }
}

// Step flags of the persistent batched kernel (ints in global memory,
// shared by the CTAs of one launch): a release store publishes a count after
// the writer's earlier stores, an acquire load orders the reader's later
// accesses after it.
__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// order generic-proxy accesses of global memory with later bulk copies
// (async proxy) of the same memory
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Wait until *flag >= need; bounded like mbar_wait (gives up after kWaitNs,
// or at once when another waiter has recorded a failure).
__device__ __forceinline__ bool flag_wait(const int* flag, int need, unsigned* err)
{
    if (ld_acquire_gpu(flag) >= need) return true;
    unsigned long long t0 = 0;
    for (unsigned n = 1;; ++n) {
        __nanosleep(64);
        if (ld_acquire_gpu(flag) >= need) return true;
        if (n % kPollCheck == 0) {
            const unsigned long long now = global_ns();
            if (n == kPollCheck) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                if (err) atomicOr(err, kErrTimeout);
                return false;
            }
            if (err && *reinterpret_cast<volatile unsigned*>(err)) return false;
        }
    }
}

// Named CTA barrier `id` (1..15) over the `nthreads` threads (a multiple of
// 32, whole converged warps) that execute it; orders their shared-memory
// accesses like __syncthreads.  A hardware barrier, not a poll: it is used
// only where every participating warp runs the same sequence of barriers
// whatever any wait returns, so that it always completes.
__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The same barrier, returning whether `pred` holds on any participating
// thread (bar.red.or), so that the participants take one decision.
__device__ __forceinline__ bool named_sync_or(int id, int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

}  // namespace lbfe
