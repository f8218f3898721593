// stages.h -- internal interface between the executor runtime and the stage kernels.
//
// Each job type is planned as a short list of kernel launches over one slot (the job's DAG
// of Sec. 4.1 minus its two copy nodes).  The runtime turns a plan into graph kernel nodes
// once per slot and, per job, into cudaGraphExecKernelNodeSetParams updates; the same plan
// also drives direct stream launches.  Every kernel takes one argument struct by value.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../runtime/layout.h"
#include "params.h"
#include "set.h"

namespace setk {

constexpr int kMaxKernels = 6;
constexpr size_t kMaxArgBytes = 512;  // room for two 128-byte TMA descriptors

struct KernelLaunch {
  const void* func = nullptr;
  dim3 grid, block;
  unsigned smem = 0;
  alignas(64) unsigned char args[kMaxArgBytes];
  size_t args_size = 0;
  uint32_t deps = 0;  // bit k: waits for kernel k of the plan; 0 = waits for the H2D copy only
  void* params[1];    // kernel parameter array for launch APIs (points at args)
};

struct JobPlanIn {
  uint32_t type = 0;
  uint32_t dims[4] = {0, 0, 0, 0};
  float scalar = 0.f;
  const void* shared[2] = {nullptr, nullptr};
  const void* d_in = nullptr;
  void* d_out = nullptr;
  void* d_scratch = nullptr;  // transient work buffers (JobLayout::scratch_bytes)
  void* d_persist = nullptr;  // persistent control state (JobLayout::persist_bytes), zeroed once
  uint64_t job_id = 0;
  uint32_t slot_gen = 0;
  int img_fused = 1;
};

// Fills kl[0 .. *nk) with the job's kernel launches in dependency order.
bool plan_job(const JobPlanIn& in, KernelLaunch* kl, int* nk);

// Per-type planners (one per kernel source file).
bool plan_blur_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_saxpy_scan_max(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_img_sobel_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_mlp_ln(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);

// Batched form planners: fill the host table (L.table_bytes) and the kernel launches of one
// launch over nb jobs whose block starts at d_block.
bool plan_img_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, int ctas_per_sm, int tile_variant, KernelLaunch* kl, int* nk);
bool plan_mlp_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, const void* w1, const void* w2, KernelLaunch* kl, int* nk);

// One-time function attributes (dynamic shared memory limits, cluster sizes).
cudaError_t kernels_init();
cudaError_t blur_hist_init();
cudaError_t mlp_init();

template <class A>
inline void set_args(KernelLaunch& k, const A& a) {
  static_assert(sizeof(A) <= kMaxArgBytes, "kernel argument struct too large");
  __builtin_memcpy(k.args, &a, sizeof(A));
  k.args_size = sizeof(A);
  k.params[0] = k.args;
}

// Trailer word written by each job's last kernel.
__host__ __device__ inline uint32_t trailer_word(uint32_t err) { return (SET_TRAILER_MAGIC << 16) | (err & 0xFFFFu); }

}  // namespace setk
