// Tensor memory (TMEM, 128 lanes x 512 columns of 32 bits per SM on sm_100
// family GPUs) used as a per-thread register extension: a warp reaches the
// 32 lanes of its quarter, 32 * (warp % 4) .. + 31, lane = thread of the warp,
// through tcgen05.ld / tcgen05.st of the 32x32b shape (one 32-bit column per
// register).  Inline PTX, sm_103a.
//
// Allocation is per CTA and must be undone before the CTA exits: one full
// warp allocates (the address lands in shared memory) and the same warp
// frees it after every access has completed and the CTA has synchronised
// (tcgen05 fences on both sides of the barrier).  tcgen05.alloc waits while
// the SM lacks free columns, so a kernel that takes all 512 columns must not
// share its SM with another CTA holding any: the callers guarantee one CTA
// per SM through their shared-memory footprint.
#pragma once
#include <cstdint>

namespace lbo {
namespace tmem {

constexpr uint32_t kColumns = 512;

__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// order tcgen05 operations against a CTA barrier (before / after it)
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// address of (lane, column); the allocation base has lane 0
__device__ __forceinline__ uint32_t addr(uint32_t base, uint32_t lane, uint32_t col) {
  return base + (lane << 16) + col;
}

// r[c] <- column col + c of this thread's lane, c = 0..7 (warp-collective);
// the values are valid only after wait_ld(r).  Eight columns per call keep
// the fused kernels within their 96-register budget.
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// wait for this thread's tcgen05.ld; r is passed through so that no use of
// the loaded registers is scheduled before the wait
__device__ __forceinline__ void wait_ld(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// column col + c of this thread's lane <- r[c], c = 0..7 (warp-collective)
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// wait until this thread's tcgen05.st have completed
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace tmem
}  // namespace lbo
