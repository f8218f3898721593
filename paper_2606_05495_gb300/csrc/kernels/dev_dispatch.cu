// dev_dispatch.cu -- the fetch kernel of a device-dispatch lane (layout in dev_dispatch.h).
//
// One warp.  Every wait is bounded: a lane polls its ring for at most idle_ns (and a fixed number
// of rounds), then ends its loop; the host relaunches the lane's graph when it has work again.
#include "dev_dispatch.h"

#include <type_traits>

#include "stages.h"

namespace setk {
namespace {

static_assert(std::is_same<cudaGraphConditionalHandle, unsigned long long>::value,
              "DdFetchArgs carries conditional handles as unsigned long long");

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kPollLimit = 1u << 24;  // rounds, a backstop beside the time limit

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_sys(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_sys32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(uint64_t* p, uint64_t v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(32) dd_fetch_kernel(const __grid_constant__ DdFetchArgs a) {
  DdLaneDev* L = a.lane;
  const uint32_t lane = threadIdx.x;

  // Retire the job the previous iteration ran: the SWITCH body that ran it has completed, so its
  // trailer is final.  The completion word is the trailer word, or 0 when the trailer does not
  // belong to the job (the host counts that as a canary error).
  if (lane == 0 && L->cur_seq != 0) {
    const uint64_t s = L->cur_seq;
    const volatile set_trailer* t = L->cur_trailer;
    uint32_t word = 0u;
    if (t && (reinterpret_cast<uintptr_t>(t) & 7u) == 0) {
      word = t->word;
      if (t->job_id != L->cur_job || (word >> 16) != SET_TRAILER_MAGIC) word = 0u;
    }
    st_relaxed_sys32(&a.cmpl[(s - 1) & (a.depth - 1)], word);
    st_release_sys(&a.ctl->done, s);
    L->cur_seq = 0;
  }

  // Wait for descriptor head + 1.  All 32 threads load the same word (one request); the decision
  // to give up is lane 0's, so the warp stays converged.
  const uint64_t head = L->head;
  const uint64_t want = head + 1;
  const DdEntry* e = a.ring + (head & (a.depth - 1));
  const uint64_t t0 = global_ns();
  bool found = false;
  for (uint32_t it = 0;; ++it) {
    const uint64_t s = ld_acquire_sys(&e->seq);
    if (__all_sync(kFull, s == want)) {
      found = true;
      break;
    }
    int quit = 0;
    if (lane == 0)
      quit = ld_relaxed_sys32(&a.ctl->stop) != 0u || global_ns() - t0 > a.idle_ns || it >= kPollLimit;
    if (__shfl_sync(kFull, quit, 0)) break;
    __nanosleep(it < 64 ? 32 : 256);
  }

  if (found) {
    // thread k copies word k of the entry; words 8..31 are the argument struct
    const uint64_t v = ld_relaxed_sys(reinterpret_cast<const uint64_t*>(e) + lane);
    const uint32_t kind = (uint32_t)__shfl_sync(kFull, v, 1);
    const uint64_t job = __shfl_sync(kFull, v, 2);
    const uint64_t tr = __shfl_sync(kFull, v, 3);
    if (kind < kDdKinds && lane >= 8) reinterpret_cast<uint64_t*>(L->args[kind])[lane - 8] = v;
    if (lane == 0) {
      L->head = want;
      L->cur_seq = want;
      L->cur_job = job;
      L->cur_trailer = reinterpret_cast<set_trailer*>(tr);
      cudaGraphSetConditional(a.kind, kind < kDdKinds ? kind : kDdKindNone);
    }
  } else if (lane == 0) {
    cudaGraphSetConditional(a.kind, kDdKindNone);
    cudaGraphSetConditional(a.loop, 0u);
    const uint32_t x = L->exits + 1u;
    L->exits = x;
    st_release_sys32(&a.ctl->exits, x);
  }
}

}  // namespace

const void* dd_fetch_func() { return reinterpret_cast<const void*>(&dd_fetch_kernel); }

}  // namespace setk
