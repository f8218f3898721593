// cp_async.cuh -- asynchronous global -> shared copies (cp.async, sm_80 and later) used to stage
// stencil windows: a thread issues all of its copies, then waits once, so a tile costs one memory
// latency instead of one per loop trip.
#pragma once

#include <cstdint>

namespace setk {

// 16 bytes, both addresses 16-byte aligned; cached in L2 only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
// 4 bytes, both addresses 4-byte aligned.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
// Waits for every cp.async this thread issued (the caller then synchronises the block).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace setk
