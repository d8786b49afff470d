// tmem.cuh -- tensor memory (TMEM) as a per-thread scratch store on sm_103a.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM, separate from shared
// memory.  The tensor cores use it for accumulators; the stencil kernels use it
// only as storage: a warp reaches the 32 lanes of its quadrant (warp index
// within the CTA mod 4), and with the 32x32b shape thread t of the warp reads or
// writes lane 32 * quadrant + t, so a thread owns a row of the columns that its
// CTA allocated.
//
// Rules kept by the callers:
// * one warp allocates (all 32 lanes, a power of two >= 32 columns), writes
//   the base address to shared memory, gives up the allocation permit, and the
//   same warp frees the columns before the CTA exits, on every path;
// * the CTAs resident on one SM never ask for more than 512 columns together
//   (the launch sizes shared memory so that no more of them fit), so an
//   allocation never waits for another CTA;
// * tcgen05.ld results are read only after tcgen05.wait::ld (the wait below
//   names the destination registers, so the compiler cannot move their uses
//   above it), and a thread waits for its own stores (tcgen05.wait::st) before
//   it loads what they wrote.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rswr_device.cuh"

namespace rswr {

// Address of (lane, column) in the TMEM address space.
__device__ __forceinline__ uint32_t tmem_addr(uint32_t base, uint32_t lane, uint32_t col)
{
    return base + (lane << 16) + col;
}

// Whole warp: allocate ncols columns; the base address lands in *dst (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}

// Whole warp: this CTA makes no further allocation.
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp (the allocating one): free the columns.
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// Order tcgen05 operations around a thread barrier.
__device__ __forceinline__ void tmem_fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Whole warp: each thread stores 8 words into columns [col, col + 8) of its lane
// (addr: the warp's first lane, column col).
__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(addr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// Whole warp: issue the load of 8 words per thread; the registers are valid
// after tmem_wait_ld on the same array.
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(addr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace rswr
