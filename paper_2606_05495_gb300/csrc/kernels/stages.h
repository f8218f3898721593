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

// Stage-order stamps (a test invariant, off unless the context enables it): the first CTA of a
// kernel to arrive writes an entry ticket and the last CTA to leave writes an exit ticket, both
// drawn from one device counter, into the slot's mapped host array.  Every kernel's argument
// struct starts with a Stamp so that the planner can fill it generically.
struct Stamp {
  unsigned long long* clock = nullptr;  // device ticket counter (null: stamps off)
  uint32_t* ctr = nullptr;              // device {arrive, depart} counters of this kernel
  uint64_t* out = nullptr;              // mapped host {entry, exit} of this kernel
  uint64_t pad = 0;
};
static_assert(sizeof(Stamp) == 32, "stamp header of every argument struct");

#ifdef __CUDACC__
__device__ __forceinline__ void stamp_entry(const Stamp& s) {
  if (s.clock && threadIdx.x == 0 && atomicAdd(&s.ctr[0], 1u) == 0u)
    *reinterpret_cast<volatile uint64_t*>(&s.out[0]) = atomicAdd(s.clock, 1ull) + 1ull;  // tickets start at 1
}
__device__ __forceinline__ void stamp_exit(const Stamp& s) {
  if (s.clock && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&s.ctr[1], 1u) == gridDim.x * gridDim.y * gridDim.z - 1u) {
      *reinterpret_cast<volatile uint64_t*>(&s.out[1]) = atomicAdd(s.clock, 1ull) + 1ull;
      s.ctr[0] = 0u;  // every CTA has arrived and left: ready for the next launch
      s.ctr[1] = 0u;
    }
  }
}
#endif

constexpr int kMaxKernels = 8;
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
  uint32_t flags = 0;  // set_job_desc.flags
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
  Stamp stamps;  // base of this slot's stamps (ctr / out point at kernel 0), clock null = off
};

// Fills the Stamp header of kernel k's arguments from a slot's stamp base.
inline void attach_stamp(KernelLaunch& k, const Stamp& base, int idx) {
  Stamp st = base;
  if (st.clock) {
    st.ctr = base.ctr + 2 * idx;
    st.out = base.out + 2 * idx;
  }
  __builtin_memcpy(k.args, &st, sizeof st);
}

// Fills kl[0 .. *nk) with the job's kernel launches in dependency order.
bool plan_job(const JobPlanIn& in, KernelLaunch* kl, int* nk);

// Per-type planners (one per kernel source file).
bool plan_blur_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_saxpy_scan_max(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_img_sobel_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_mlp_ln(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);
bool plan_hotspot(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk);

// Batched form planners: fill the host table (L.table_bytes) and the kernel launches of one
// launch over nb jobs whose block starts at d_block.
bool plan_img_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, int ctas_per_sm, int tile_variant, KernelLaunch* kl, int* nk);
bool plan_mlp_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, const void* w1, const void* w2, KernelLaunch* kl, int* nk);

// set_config.guards: the arming and checking kernels of a job placed with place_job_guarded in
// the slot at slot_base (plant: the SET_F_TEST_GUARD hook).
void plan_guards(uint8_t* slot_base, const JobLayout& L, bool plant, KernelLaunch* arm, KernelLaunch* check);

// Device-dispatch lane kernels and their fixed launch shapes.  The blur kernel takes (argument
// areas of kDdArgBytes each, pointer to the number of jobs) and runs on kDdBatch clusters of 8
// CTAs, its dynamic shared memory covering the lane's widest image (blur_lane_smem).  The scan
// kernel takes (argument areas, pointer to the number of jobs, tmax, scratch stride) and runs on
// a grid of kDdBatch * tmax blocks, tmax = scan_lane_tiles(the lane's largest n).  The image
// kernel takes one argument, a pointer to the job's argument struct in device memory.
const void* scan_lane_func();
uint32_t scan_lane_tiles(uint32_t max_n);
const void* blur_lane_func();
unsigned blur_lane_smem(uint32_t max_w);
const void* img_lane_func();
uint32_t img_lane_grid();
// The image lane kernel's argument struct (ticket mode over the lane's image state in d_persist).
bool plan_img_lane(const JobPlanIn& in, unsigned char* args, uint32_t* args_size);
const void* dd_fetch_func();

// set_config.sm_copies: one copy kernel launch moving `bytes` from src to dst (both 16-byte
// aligned and addressable by the GPU, e.g. page-locked host memory mapped at the same address).
void plan_copy(void* dst, const void* src, size_t bytes, KernelLaunch* k);

// One-time function attributes (dynamic shared memory limits, cluster sizes).
cudaError_t kernels_init();
cudaError_t blur_hist_init();
cudaError_t mlp_init();
cudaError_t hotspot_init();

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
