// copy.cu -- copy kernel of set_config.sm_copies: a job graph's H2D and D2H steps done by SM
// loads and stores over NVLink-C2C instead of memcpy nodes on the copy engines.
//
// At the job sizes of this executor (64 KiB to a few MiB) a copy-engine transfer pays a fixed
// setup per copy and one engine per direction; many CTAs each moving 16-byte words keep far
// more requests in flight on the coherent host link.  Every thread issues its loads before its
// stores; the last bytes % 16 are copied one byte per thread by the first block.
#include <algorithm>

#include "stages.h"

namespace setk {
namespace {

constexpr int kCopyThreads = 256;
constexpr int kCopyPer = 2;           // 16-byte words a thread keeps in flight per round
constexpr uint32_t kCopyMaxCtas = 128;

struct CopyArgs {
  uint4* dst;
  const uint4* src;
  size_t n16;  // whole 16-byte words
  uint32_t tail;
  uint32_t pad;
};

__global__ void __launch_bounds__(kCopyThreads) copy_kernel(const __grid_constant__ CopyArgs a) {
  const size_t stride = (size_t)gridDim.x * kCopyThreads;
  size_t i = (size_t)blockIdx.x * kCopyThreads + threadIdx.x;
  for (; i + (kCopyPer - 1) * stride < a.n16; i += kCopyPer * stride) {
    uint4 v[kCopyPer];
#pragma unroll
    for (int u = 0; u < kCopyPer; ++u) v[u] = a.src[i + u * stride];
#pragma unroll
    for (int u = 0; u < kCopyPer; ++u) a.dst[i + u * stride] = v[u];
  }
  for (; i < a.n16; i += stride) a.dst[i] = a.src[i];
  if (blockIdx.x == 0 && threadIdx.x < a.tail)
    reinterpret_cast<uint8_t*>(a.dst + a.n16)[threadIdx.x] = reinterpret_cast<const uint8_t*>(a.src + a.n16)[threadIdx.x];
}

}  // namespace

void plan_copy(void* dst, const void* src, size_t bytes, KernelLaunch* k) {
  CopyArgs a{};
  a.dst = static_cast<uint4*>(dst);
  a.src = static_cast<const uint4*>(src);
  a.n16 = bytes / 16;
  a.tail = (uint32_t)(bytes % 16);
  const size_t per_cta = (size_t)kCopyThreads * kCopyPer;
  k->func = reinterpret_cast<const void*>(&copy_kernel);
  k->grid = dim3((unsigned)std::clamp<size_t>((a.n16 + per_cta - 1) / per_cta, 1, kCopyMaxCtas));
  k->block = dim3(kCopyThreads);
  k->smem = 0;
  k->deps = 0;
  set_args(*k, a);
}

}  // namespace setk
