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

// Copies the entry `e` (one 8-byte word per thread) into `args`; returns word `w` of the entry to
// every thread.
__device__ __forceinline__ uint64_t take_entry(const DdEntry* e, unsigned char* args, uint32_t lane, uint64_t* job,
                                               uint64_t* trailer) {
  const uint64_t v = ld_relaxed_sys(reinterpret_cast<const uint64_t*>(e) + lane);
  if (lane >= 8) reinterpret_cast<uint64_t*>(args)[lane - 8] = v;
  *job = __shfl_sync(kFull, v, 2);
  *trailer = __shfl_sync(kFull, v, 3);
  return __shfl_sync(kFull, v, 1);  // kind (low half), args_size (high half)
}

__global__ void __launch_bounds__(32) dd_fetch_kernel(const __grid_constant__ DdFetchArgs a) {
  DdLaneDev* L = a.lane;
  const uint32_t lane = threadIdx.x;
  const uint32_t mask = a.depth - 1;

  // Retire the jobs the previous iteration ran: the SWITCH body that ran them has completed, so
  // their trailers are final.  Thread i checks job i's trailer (its word, or 0 when the trailer
  // does not belong to the job: the host counts a canary error); thread 0 writes every completion
  // word and then the done counter with release order.
  const uint32_t cnt = L->cur_count;
  if (cnt != 0) {
    const uint64_t first = L->cur_first;
    uint32_t word = 0u;
    if (lane < cnt) {
      const volatile set_trailer* t = L->cur_trailer[lane];
      if (t && (reinterpret_cast<uintptr_t>(t) & 7u) == 0) {
        word = t->word;
        if (t->job_id != L->cur_job[lane] || (word >> 16) != SET_TRAILER_MAGIC) word = 0u;
      }
    }
    for (uint32_t i = 0; i < cnt; ++i) {
      const uint32_t w = __shfl_sync(kFull, word, i);
      if (lane == 0) st_relaxed_sys32(&a.cmpl[(first - 1 + i) & mask], w);
    }
    if (lane == 0) {
      st_release_sys(&a.ctl->done, first + cnt - 1);
      L->cur_count = 0;
    }
  }

  // Wait for descriptor head + 1.  All 32 threads load the same word (one request); the decision
  // to give up is thread 0's, so the warp stays converged.
  const uint64_t head = L->head;
  const uint64_t want = head + 1;
  const DdEntry* e = a.ring + (head & mask);
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

  if (!found) {
    if (lane == 0) {
      cudaGraphSetConditional(a.kind, kDdKindNone);
      cudaGraphSetConditional(a.loop, 0u);
      const uint32_t x = L->exits + 1u;
      L->exits = x;
      st_release_sys32(&a.ctl->exits, x);
    }
    return;
  }

  // Peek at the kind, then take the entry into the argument area of its node.  A blur or scan job
  // also takes the descriptors of the same kind that directly follow it and are already complete
  // (up to kDdBatch): they run in the same launch of the node.
  uint64_t job = 0, tr = 0;
  const uint32_t kind = (uint32_t)__shfl_sync(kFull, ld_relaxed_sys(reinterpret_cast<const uint64_t*>(e) + 1), 0);
  const bool batched = kind == kDdKindScan || kind == kDdKindBlur;
  uint32_t count = 1;
  if (batched) {
    take_entry(e, L->batch_args[0], lane, &job, &tr);
    if (lane == 0) {
      L->cur_job[0] = job;
      L->cur_trailer[0] = reinterpret_cast<set_trailer*>(tr);
    }
    for (; count < kDdBatch; ++count) {
      const DdEntry* f = a.ring + ((head + count) & mask);
      const uint64_t s = ld_acquire_sys(&f->seq);
      if (!__all_sync(kFull, s == want + count)) break;
      const uint64_t k = ld_relaxed_sys(reinterpret_cast<const uint64_t*>(f) + 1);
      if ((uint32_t)__shfl_sync(kFull, k, 0) != kind) break;
      take_entry(f, L->batch_args[count], lane, &job, &tr);
      if (lane == 0) {
        L->cur_job[count] = job;
        L->cur_trailer[count] = reinterpret_cast<set_trailer*>(tr);
      }
    }
  } else if (kind < kDdKinds) {
    take_entry(e, L->args[kind], lane, &job, &tr);
    if (lane == 0) {
      L->cur_job[0] = job;
      L->cur_trailer[0] = reinterpret_cast<set_trailer*>(tr);
    }
  } else if (lane == 0) {
    L->cur_job[0] = 0;  // not a kind of this lane: nothing runs, the job retires as a canary error
    L->cur_trailer[0] = nullptr;
  }
  if (lane == 0) {
    L->batch_count = batched ? count : 0u;
    L->head = head + count;
    L->cur_first = want;
    L->cur_count = count;
    cudaGraphSetConditional(a.kind, kind < kDdKinds ? kind : kDdKindNone);
  }
}

}  // namespace

const void* dd_fetch_func() { return reinterpret_cast<const void*>(&dd_fetch_kernel); }

}  // namespace setk
