// rswr_device.cuh -- sm_103a device helpers for the RSWR kernels: 1-D TMA bulk
// copies (cp.async.bulk) with mbarrier completion, proxy fences, acquire/release
// flags, bounded waits and the device error record.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rswr {

// Device error codes (mirrored by rswr_status on the host side).
enum DevErrCode : int {
    kDevOk = 0,
    kDevTimeoutLoad = 1,   // an mbarrier (TMA load) wait ran out of time
    kDevTimeoutFlag = 2,   // a neighbour-flag wait ran out of time
    kDevBadTicket = 3,     // a ticket outside the table (internal consistency check)
};

struct DevError {
    int code;   // first error latched (0 = none)
    int tile;   // tile index that latched it
    int span;   // span index
    int where;  // 0 = span kernel, 1 = adjoint kernel
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier -------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
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

// Expect `bytes` more transaction bytes in the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Plain arrival (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Waits for the phase with the given parity to complete; gives up after
// limit_ns nanoseconds (returns false) or as soon as another CTA latched an
// error (err_code != 0).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_ns,
                                                  const volatile int* err_code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
        if (err_code && *err_code != 0) {
            // keep waiting a little: the copy was issued and normally lands
            if (global_ns() - t0 > (limit_ns >> 4)) return false;
        }
    }
}

// The same wait for a thread that has nothing else to do (a producer): it
// sleeps between polls (64 ns growing to 512 ns) so that it takes almost no
// issue slots from the warps that compute.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, long long limit_ns,
                                                  const volatile int* err_code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    unsigned ns = 64;
    for (;;) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        if (mbar_try_wait(bar, parity)) return true;
        const long long dt = global_ns() - t0;
        if (dt > limit_ns) return false;
        if (err_code && *err_code != 0 && dt > (limit_ns >> 4)) return false;
    }
}

// ---- 1-D bulk copies (TMA, non-tensor) -----------------------------------
// Global -> shared, completion signalled on an mbarrier (complete_tx).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Shared -> global, tracked by bulk async-groups.
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// All committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// All committed bulk stores are complete (writes performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Same for global memory (flag hand-off between bulk copies of different CTAs).
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ---- named barriers ---------------------------------------------------------
// Barrier 1 among the first NB threads of the CTA (NB a multiple of 32); the
// other threads of the CTA never touch it.  NB = 0 means the whole CTA
// (__syncthreads, barrier 0).
template <int NB>
__device__ __forceinline__ void block_sync()
{
    if constexpr (NB == 0) {
        __syncthreads();
    } else {
        static_assert(NB % 32 == 0, "named barriers count whole warps");
        asm volatile("barrier.cta.sync 1, %0;" ::"n"(NB) : "memory");
    }
}

// block_sync that also returns whether any participating thread passed p = true.
template <int NB>
__device__ __forceinline__ bool block_sync_or(bool p)
{
    if constexpr (NB == 0) {
        return __syncthreads_or(p) != 0;
    } else {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred a, b;\n\t"
            "setp.ne.u32 a, %1, 0;\n\t"
            "barrier.cta.red.or.pred b, 1, %2, a;\n\t"
            "selp.u32 %0, 1, 0, b;\n\t}"
            : "=r"(r)
            : "r"((uint32_t)p), "n"(NB)
            : "memory");
        return r != 0;
    }
}

// ---- acquire / release flags ---------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// With relaxed loads before it, the acquire side of a release/acquire pair:
// later memory operations observe what the releasing thread wrote before its
// release store (PTX memory model, fence-based acquire pattern).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void latch_error(DevError* e, int code, int tile, int span, int where)
{
    if (atomicCAS(&e->code, 0, code) == 0) {
        e->tile = tile;
        e->span = span;
        e->where = where;
        __threadfence();
    }
}

// ---- correctly rounded arithmetic with a fixed operation order ----------
// Explicit intrinsics so that no compiler contraction or reassociation can
// change the bits.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }

}  // namespace rswr
