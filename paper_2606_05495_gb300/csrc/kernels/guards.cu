// guards.cu -- guard bands of set_config.guards, the bounds check of the stage kernels on a pool
// without compute-sanitizer.  Around each job's in / out / scratch regions of its slot lie four
// 256-byte bands (layout.h, place_job_guarded).  guard_arm_kernel, the first node of the job's
// graph, fills them with a position-dependent pattern; guard_check_kernel, which runs after the
// last stage kernel and before the D2H copy, compares them and sets SET_DEVERR_GUARD in the
// job's trailer if any byte changed, so a stage kernel that writes past its regions fails its job.
#include "stages.h"

namespace setk {
namespace {

constexpr int kGuardThreads = 256;

struct GuardArgs {
  uint8_t* band[4];
  uint32_t* trailer_word;  // the trailer's word (device address, in the job's out region)
  uint32_t plant;          // test hook: arm one wrong byte in band 2
};

__device__ __forceinline__ uint8_t guard_pattern(int k) { return (uint8_t)(0xA5u ^ (uint32_t)(k * 29)); }

__global__ void __launch_bounds__(kGuardThreads) guard_arm_kernel(const GuardArgs a) {
  for (int i = threadIdx.x; i < 4 * (int)kGuardBytes; i += kGuardThreads) {
    const int b = i / (int)kGuardBytes, k = i - b * (int)kGuardBytes;
    const uint8_t wrong = (a.plant && b == 2 && k == 7) ? 0xFFu : 0u;
    a.band[b][k] = guard_pattern(k) ^ wrong;
  }
}

__global__ void __launch_bounds__(kGuardThreads) guard_check_kernel(const GuardArgs a) {
  bool bad = false;
  for (int i = threadIdx.x; i < 4 * (int)kGuardBytes; i += kGuardThreads) {
    const int b = i / (int)kGuardBytes, k = i - b * (int)kGuardBytes;
    bad |= a.band[b][k] != guard_pattern(k);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.trailer_word, SET_DEVERR_GUARD);
}

}  // namespace

void plan_guards(uint8_t* slot_base, const JobLayout& L, bool plant, KernelLaunch* arm, KernelLaunch* check) {
  size_t off[4];
  guard_offsets(L, off);
  GuardArgs a{};
  for (int b = 0; b < 4; ++b) a.band[b] = slot_base + off[b];
  a.trailer_word = reinterpret_cast<uint32_t*>(slot_base + L.out_off + L.out_bytes - sizeof(set_trailer) +
                                               offsetof(set_trailer, word));
  a.plant = plant ? 1u : 0u;
  for (KernelLaunch* k : {arm, check}) {
    k->func = k == arm ? reinterpret_cast<const void*>(&guard_arm_kernel)
                       : reinterpret_cast<const void*>(&guard_check_kernel);
    k->grid = dim3(1);
    k->block = dim3(kGuardThreads);
    k->smem = 0;
    k->deps = 0;
    set_args(*k, a);
  }
}

}  // namespace setk
