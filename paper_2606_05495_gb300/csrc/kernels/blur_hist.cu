// blur_hist.cu -- blur job: 3x3 box blur (integer sum / 9, floored, edge-clamped) fused with
// the 256-bin histogram of the blurred image.
//
// One thread-block cluster of 8 CTAs per job.  Each CTA owns a band of rows, stages it (plus a
// one-row halo, rows clamped) in shared memory with 16-byte cp.async, writes 16 output pixels per
// work item with one 16-byte store, and counts them in per-warp privatised shared histograms.
// The 8 CTA histograms are summed through distributed shared memory (each CTA reduces 32 bins
// across the cluster), so the job needs no global atomics, no zeroing pass and no scratch.
#include <cooperative_groups.h>

#include "cp_async.cuh"
#include "dev_dispatch.h"
#include "stages.h"

namespace cg = cooperative_groups;

namespace setk {
namespace {

constexpr int kCluster = 8;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkRows = 32;
constexpr int kMaxW = kBlurMaxW;

struct BlurHistArgs {
  Stamp stamp;  // first member: filled by the planner
  const uint8_t* in;
  uint8_t* out;
  uint8_t* pad;  // zero bytes between image and histogram
  uint32_t* hist;
  set_trailer* trailer;
  uint64_t job_id;
  uint32_t W, H;
  uint32_t slot_gen, npad;
};

// The whole kernel body: shared by the kernel that takes its arguments by value and the
// device-dispatch lane kernel that reads them from device memory.
__device__ __forceinline__ void blur_hist_body(const BlurHistArgs& a) {
  extern __shared__ __align__(16) uint8_t tile[];  // (kChunkRows + 2) rows x pitch
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t chist[256];
  stamp_entry(a.stamp);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kWarps * 256; i += kThreads) (&whist[0][0])[i] = 0u;

  const int W = (int)a.W, H = (int)a.H;
  const int pitch = (W + 15) & ~15;
  const int rows_per = (H + kCluster - 1) / kCluster;
  const int y0 = rank * rows_per, y1 = min(H, y0 + rows_per);
  const bool vec = (W & 15) == 0 && ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.out)) & 15) == 0;
  const int gpr = (W + 15) >> 4;  // 16-pixel groups per row
  __syncthreads();

  for (int cy = y0; cy < y1; cy += kChunkRows) {
    const int ny = min(kChunkRows, y1 - cy);
    if (vec) {  // every 16-byte copy of the band in flight at once
      const int vpr = W >> 4;
      for (int i = tid; i < (ny + 2) * vpr; i += kThreads) {
        const int r = i / vpr, c = i - r * vpr;
        const int sy = min(max(cy - 1 + r, 0), H - 1);
        cp_async16(tile + r * pitch + 16 * c, a.in + (size_t)sy * W + 16 * c);
      }
      cp_async_wait_all();
    } else {
      for (int i = tid; i < (ny + 2) * W; i += kThreads) {
        const int r = i / W, c = i - r * W;
        const int sy = min(max(cy - 1 + r, 0), H - 1);
        tile[r * pitch + c] = a.in[(size_t)sy * W + c];
      }
    }
    __syncthreads();
    for (int i = tid; i < ny * gpr; i += kThreads) {
      const int r = i / gpr, x0 = (i - r * gpr) << 4;
      const uint8_t* t0 = tile + r * pitch;
      const uint8_t* t1 = t0 + pitch;
      const uint8_t* t2 = t1 + pitch;
      unsigned v[18];  // vertical 3-sums of columns x0-1 .. x0+16 (clamped)
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        const int x = min(max(x0 - 1 + k, 0), W - 1);
        v[k] = (unsigned)t0[x] + (unsigned)t1[x] + (unsigned)t2[x];
      }
      uint32_t o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t w = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int k = 4 * q + b;
          w |= ((v[k] + v[k + 1] + v[k + 2]) / 9u) << (8 * b);
        }
        o[q] = w;
      }
      uint8_t* dst = a.out + (size_t)(cy + r) * W + x0;
      const int nvalid = min(16, W - x0);
      if (vec) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
      } else {
        for (int k = 0; k < nvalid; ++k) dst[k] = (uint8_t)(o[k >> 2] >> (8 * (k & 3)));
      }
      for (int k = 0; k < nvalid; ++k) atomicAdd(&whist[warp][(o[k >> 2] >> (8 * (k & 3))) & 0xFFu], 1u);
    }
    __syncthreads();
  }

  for (int b = tid; b < 256; b += kThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += whist[w][b];
    chist[b] = s;
  }
  cluster.sync();
  constexpr int kBinsPerRank = 256 / kCluster;
  if (tid < kBinsPerRank) {
    const int b = rank * kBinsPerRank + tid;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kCluster; ++q) s += cluster.map_shared_rank(chist, q)[b];
    a.hist[b] = s;
  }
  if (rank == 0 && tid < (int)a.npad) a.pad[tid] = 0;
  if (rank == 0 && tid == 0) {
    a.trailer->job_id = a.job_id;
    a.trailer->slot_gen = a.slot_gen;
    a.trailer->word = trailer_word(0);
  }
  cluster.sync();  // every CTA's chist stays alive until the remote reads are done
  stamp_exit(a.stamp);
}

__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(kThreads)
    blur_hist_kernel(const __grid_constant__ BlurHistArgs a) {
  blur_hist_body(a);
}

// Device-dispatch lane kernel: the node's grid is kDdBatch clusters; the lane's fetch kernel
// writes the arguments of the `*count` blur jobs of this iteration into consecutive kDdArgBytes
// areas of device memory, cluster j runs job j and clusters past `*count` leave at once (all CTAs
// of a cluster take the same decision, so no cluster barrier is left waiting).  The node's
// dynamic shared memory covers the lane's widest image.
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(kThreads)
    blur_hist_lane_kernel(const unsigned char* __restrict__ args, const uint32_t* __restrict__ count) {
  const uint32_t j = blockIdx.x / kCluster;
  if (j >= *count || j >= kDdBatch) return;
  const BlurHistArgs* pa = reinterpret_cast<const BlurHistArgs*>(args + (size_t)j * kDdArgBytes);
  // arguments that do not describe a job this node can run (an empty or too wide image for the
  // node's shared memory, null or unaligned buffers) run nothing: every CTA of the cluster takes
  // the same decision, the trailer stays unwritten and the fetch kernel reports it
  uint32_t dsmem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
  const uint32_t W = pa->W, H = pa->H;
  const uintptr_t al = reinterpret_cast<uintptr_t>(pa->hist) | reinterpret_cast<uintptr_t>(pa->trailer);
  if (W == 0 || H == 0 || W > (uint32_t)kMaxW || (uint64_t)(kChunkRows + 2) * ((W + 15) & ~15u) > dsmem || !pa->in ||
      !pa->out || !pa->pad || (al & 7u) != 0)
    return;
  blur_hist_body(*pa);
}

static_assert(sizeof(BlurHistArgs) <= kDdArgBytes, "a blur job's arguments fit one lane argument area");

inline unsigned blur_smem(uint32_t W) { return (unsigned)((kChunkRows + 2) * ((W + 15) & ~15u)); }

inline size_t blur_img_bytes(const uint32_t d[4]) { return (size_t)d[0] * d[1]; }

}  // namespace

bool plan_blur_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk) {
  BlurHistArgs a{};
  const size_t img = blur_img_bytes(in.dims);
  const size_t hist_off = (img + 15) & ~size_t(15);
  a.in = static_cast<const uint8_t*>(in.d_in);
  a.out = static_cast<uint8_t*>(in.d_out);
  a.pad = a.out + img;
  a.npad = (uint32_t)(hist_off - img);
  a.hist = reinterpret_cast<uint32_t*>(a.out + hist_off);
  a.trailer = reinterpret_cast<set_trailer*>(a.out + L.out_bytes - sizeof(set_trailer));
  a.job_id = in.job_id;
  a.slot_gen = in.slot_gen;
  a.W = in.dims[0];
  a.H = in.dims[1];
  KernelLaunch& k = kl[0];
  k.func = reinterpret_cast<const void*>(&blur_hist_kernel);
  k.grid = dim3(kCluster);
  k.block = dim3(kThreads);
  k.smem = blur_smem(in.dims[0]);
  k.deps = 0;
  set_args(k, a);
  *nk = 1;
  return true;
}

cudaError_t blur_hist_init() {
  for (const void* f : {reinterpret_cast<const void*>(&blur_hist_kernel), reinterpret_cast<const void*>(&blur_hist_lane_kernel)}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (kChunkRows + 2) * kMaxW);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

const void* blur_lane_func() { return reinterpret_cast<const void*>(&blur_hist_lane_kernel); }
unsigned blur_lane_smem(uint32_t max_w) { return blur_smem(max_w); }

}  // namespace setk
