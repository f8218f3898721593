// saxpy_scan_max.cu -- scan job: z = fmaf(a, x, y), S = exclusive prefix sum of z, m = max|S_i|,
// in one single-pass kernel.
//
// Tiles of 4096 elements (256 threads x 16 contiguous elements, 16-byte loads and stores), one
// per block in block-index order, resolve their prefix with decoupled look-back (Merrill &
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016): each tile
// publishes its aggregate, then one warp reads the status words of 32 predecessors per round trip
// and sums back to the nearest inclusive prefix.  Inside a tile the scan is thread-serial, then
// warp-shuffle, then across the 8 warps.
//
// Latency is the cost of a 1 MiB job, so the kernel keeps its chain of dependent global round
// trips short: z stays in registers until the prefix is known (nothing has to drain before a
// status word is published), status words are self-contained (relaxed stores and loads, no
// fences), and instead of a done counter every tile publishes an epoch-tagged max|S| word that
// the last tile gathers with one warp to write m and the trailer.
//
// Scratch: a 64-byte header {unused, unused, epoch, err}, then per tile one 64-bit status word
// {epoch, flag, value} and one 64-bit max word {epoch, max|S| bits}.  Words carry the header's
// epoch, so stale words of an earlier launch never match; the last tile bumps the epoch and
// clears err once every tile has published, which leaves the scratch ready for the next launch
// without a zeroing pass.  Every wait is bounded: a tile that gives up sets SET_DEVERR_WAIT in the
// header, which the trailer reports.
#include <mutex>

#include "../runtime/thread_error.h"
#include "dev_dispatch.h"
#include "stages.h"

namespace setk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPer = 16;
constexpr int kTile = kThreads * kPer;
static_assert(kTile == (int)kScanTile, "tile size shared with the layout code");
constexpr int kSpinLimit = 1 << 22;  // ~0.1-0.4 s with the back-off below

constexpr uint32_t kFlagAgg = 1, kFlagInc = 2;

struct ScanHdr {
  uint32_t unused0, unused1, epoch, err;
  uint32_t pad[12];
};
static_assert(sizeof(ScanHdr) == kScanHdrBytes, "scan header size shared with the layout code");
static_assert(kScanBytesPerTile == 16, "status word + max word per tile");

struct ScanArgs {
  Stamp stamp;  // first member: filled by the planner
  const float* x;
  const float* y;
  float* z;
  float* S;
  float* m_out;  // followed by 12 zero bytes
  set_trailer* trailer;
  uint8_t* scratch;
  uint64_t job_id;
  uint32_t n, T;
  float a;
  uint32_t slot_gen;
  uint32_t skip_tile;  // test hook (SET_F_TEST_STALL): this tile never publishes; else ~0u
};

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t status_word(uint32_t epoch, uint32_t flag, float v) {
  return ((uint64_t)(epoch & 0x3FFFFFFFu) << 34) | ((uint64_t)flag << 32) | (uint64_t)__float_as_uint(v);
}
__device__ __forceinline__ uint64_t max_word(uint32_t epoch, float m) {
  return ((uint64_t)(epoch | 0x80000000u) << 32) | (uint64_t)__float_as_uint(m);
}

// One tile of the job (the whole kernel body): shared by the kernel that takes its arguments by
// value and the device-dispatch lane kernel that reads them from device memory.
__device__ __forceinline__ void scan_tile(const ScanArgs& p, uint8_t* const scratch, const uint32_t tile) {
  __shared__ float s_wsum[kWarps], s_wexcl[kWarps], s_wmax[kWarps];
  __shared__ float s_prefix;
  ScanHdr* hdr = reinterpret_cast<ScanHdr*>(scratch);
  uint64_t* status = reinterpret_cast<uint64_t*>(scratch + sizeof(ScanHdr));
  uint64_t* maxw = status + p.T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // tile = blockIdx.x: blocks are dispatched in index order, so every tile a look-back waits for
  // has started.  The epoch load is issued first and only consumed by the look-back, so its
  // latency overlaps the data loads.
  stamp_entry(p.stamp);
  if (tile == p.skip_tile) {  // test hook: the look-back of the next tile and the max gather time out
    stamp_exit(p.stamp);
    return;
  }
  const uint32_t epoch = *reinterpret_cast<volatile uint32_t*>(&hdr->epoch) & 0x3FFFFFFFu;
  const uint32_t n = p.n;
  const size_t base = (size_t)tile * kTile + (size_t)tid * kPer;
  const bool vec = (n & 3u) == 0 && base + kPer <= n;

  // saxpy: z = fmaf(a, x, y), kept in registers until the prefix is known
  float z[kPer];
  if (vec) {
#pragma unroll
    for (int q = 0; q < kPer / 4; ++q) {
      const float4 xv = __ldg(reinterpret_cast<const float4*>(p.x + base) + q);
      const float4 yv = __ldg(reinterpret_cast<const float4*>(p.y + base) + q);
      z[4 * q + 0] = fmaf(p.a, xv.x, yv.x);
      z[4 * q + 1] = fmaf(p.a, xv.y, yv.y);
      z[4 * q + 2] = fmaf(p.a, xv.z, yv.z);
      z[4 * q + 3] = fmaf(p.a, xv.w, yv.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const size_t i = base + k;
      z[k] = i < n ? fmaf(p.a, p.x[i], p.y[i]) : 0.f;
    }
  }

  // thread-serial exclusive scan of the thread's 16 elements
  float e[kPer];
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    e[k] = acc;
    acc += z[k];
  }
  // warp: inclusive shuffle scan of thread totals, exclusive by one more shuffle
  float inc = acc;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float t = __shfl_up_sync(0xFFFFFFFFu, inc, off);
    if (lane >= off) inc += t;
  }
  float lane_excl = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
  if (lane == 0) lane_excl = 0.f;
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const float w = lane < kWarps ? s_wsum[lane] : 0.f;
    float wi = w;
#pragma unroll
    for (int off = 1; off < kWarps; off <<= 1) {
      const float t = __shfl_up_sync(0xFFFFFFFFu, wi, off);
      if (lane >= off) wi += t;
    }
    float we = __shfl_up_sync(0xFFFFFFFFu, wi, 1);
    if (lane == 0) we = 0.f;
    if (lane < kWarps) s_wexcl[lane] = we;
    // the tile aggregate is the last lane's inclusive value: warp 0 continues straight into the
    // look-back without another block barrier
    const float agg = __shfl_sync(0xFFFFFFFFu, wi, kWarps - 1);

    // decoupled look-back: each round reads the status words of the 32 nearest unresolved
    // predecessors at once, waits until all are published, then sums back to the nearest
    // inclusive prefix (positions before tile 0 count as an inclusive prefix of 0)
    if (tile == 0) {
      if (lane == 0) {
        st_relaxed(&status[0], status_word(epoch, kFlagInc, agg));
        s_prefix = 0.f;
      }
    } else {
      if (lane == 0) st_relaxed(&status[tile], status_word(epoch, kFlagAgg, agg));
      float prefix = 0.f;
      int lb = (int)tile - 1;
      for (;;) {
        const int j = lb - lane;
        uint32_t flag = kFlagInc;
        float v = 0.f;
        if (j >= 0) {
          int it = 0;
          uint64_t w;
          for (;;) {
            w = ld_relaxed(&status[j]);
            if ((uint32_t)(w >> 34) == epoch && ((w >> 32) & 3u) != 0) break;
            if (++it > kSpinLimit) {
              atomicOr(&hdr->err, SET_DEVERR_WAIT);
              w = status_word(epoch, kFlagInc, 0.f);
              break;
            }
            if (it > 16) __nanosleep(20);
          }
          flag = (uint32_t)(w >> 32) & 3u;
          v = __uint_as_float((uint32_t)w);
        }
        const unsigned incm = __ballot_sync(0xFFFFFFFFu, flag == kFlagInc);
        const int stop = incm ? __ffs(incm) - 1 : 31;  // nearest inclusive prefix in this window
        float t = lane <= stop ? v : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        prefix += t;
        if (incm) break;
        lb -= 32;
      }
      if (lane == 0) {
        st_relaxed(&status[tile], status_word(epoch, kFlagInc, prefix + agg));
        s_prefix = prefix;
      }
    }
  }
  __syncthreads();

  // S = tile prefix + warp offset + lane offset + thread-serial offset; z and S stored together
  const float off = s_prefix + s_wexcl[warp] + lane_excl;
  float mx = 0.f;
  if (vec) {
#pragma unroll
    for (int q = 0; q < kPer / 4; ++q) {
      const float4 sv = make_float4(off + e[4 * q], off + e[4 * q + 1], off + e[4 * q + 2], off + e[4 * q + 3]);
      reinterpret_cast<float4*>(p.z + base)[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
      reinterpret_cast<float4*>(p.S + base)[q] = sv;
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(sv.x), fabsf(sv.y)), fmaxf(fabsf(sv.z), fabsf(sv.w))));
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const size_t i = base + k;
      if (i < n) {
        const float sv = off + e[k];
        p.z[i] = z[k];
        p.S[i] = sv;
        mx = fmaxf(mx, fabsf(sv));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if (lane == 0) s_wmax[warp] = mx;
  __syncthreads();
  if (warp != 0) return;
  float tm = lane < kWarps ? s_wmax[lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = fmaxf(tm, __shfl_xor_sync(0xFFFFFFFFu, tm, o));
  if (lane == 0) st_relaxed(&maxw[tile], max_word(epoch, tm));
  if (tile != p.T - 1) {
    stamp_exit(p.stamp);
    return;
  }

  // last tile: gather every tile's max word (32 per round), write m and the trailer, then
  // recycle the scratch (new epoch, clear err): every tile has finished its look-back by now
  const uint64_t tag = (uint64_t)(epoch | 0x80000000u);
  float m = 0.f;
  for (uint32_t t0 = 0; t0 < p.T; t0 += 32) {
    const uint32_t t = t0 + lane;
    if (t < p.T) {
      int it = 0;
      uint64_t w;
      for (;;) {
        w = ld_relaxed(&maxw[t]);
        if ((w >> 32) == tag) break;
        if (++it > kSpinLimit) {
          atomicOr(&hdr->err, SET_DEVERR_WAIT);
          w = 0;
          break;
        }
        if (it > 16) __nanosleep(20);
      }
      m = fmaxf(m, __uint_as_float((uint32_t)w));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if (lane == 0) {
    p.m_out[0] = m;
    p.m_out[1] = 0.f;
    p.m_out[2] = 0.f;
    p.m_out[3] = 0.f;
    const uint32_t err = atomicExch(&hdr->err, 0u);
    p.trailer->job_id = p.job_id;
    p.trailer->slot_gen = p.slot_gen;
    p.trailer->word = trailer_word(err);
    hdr->epoch = (epoch + 1u) & 0x3FFFFFFFu;
  }
  stamp_exit(p.stamp);
}

__global__ void __launch_bounds__(kThreads) saxpy_scan_max_kernel(const __grid_constant__ ScanArgs p) {
  scan_tile(p, p.scratch, blockIdx.x);
}

// Device-dispatch lane kernel: the graph node's grid is fixed, kDdBatch groups of tmax blocks
// (tmax = the tiles of the lane's largest job).  The lane's fetch kernel writes the arguments of
// the `*count` scan jobs of this iteration into consecutive kDdArgBytes areas of device memory;
// group j runs job j (block j * tmax + t is its tile t) on scratch area j (the planned scratch +
// j * scratch_stride), and blocks past a job's tile count, or of groups past `*count`, leave at once.
__global__ void __launch_bounds__(kThreads, 6)
    saxpy_scan_max_lane_kernel(const unsigned char* __restrict__ args, const uint32_t* __restrict__ count,
                               uint32_t tmax, uint64_t scratch_stride) {
  const uint32_t j = blockIdx.x / tmax, tile = blockIdx.x - j * tmax;
  if (j >= *count || j >= kDdBatch) return;
  const ScanArgs& p = *reinterpret_cast<const ScanArgs*>(args + (size_t)j * kDdArgBytes);
  uint8_t* const scratch = p.scratch + (size_t)j * scratch_stride;
  const uint32_t T = p.T, n = p.n;
  if (tile >= T) return;
  // arguments that do not describe a job this node can run (a tile count beyond the group, n out
  // of the tiles' range, unaligned buffers) run nothing: the job's trailer stays unwritten and
  // the fetch kernel reports it
  // (x, z and the scratch start 16-byte aligned; y, S and m follow n floats later, and the
  // kernel's 16-byte accesses to them are taken only when n is a multiple of 4; the trailer
  // follows 8n + 16 bytes of output, so it is 8-byte aligned)
  const uintptr_t al16 = reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.z) |
                         reinterpret_cast<uintptr_t>(scratch);
  const uintptr_t al4 = reinterpret_cast<uintptr_t>(p.y) | reinterpret_cast<uintptr_t>(p.S) |
                        reinterpret_cast<uintptr_t>(p.m_out);
  if (T > tmax || n == 0 || n > T * kTile || n <= (T - 1) * kTile || (al16 & 15u) != 0 || (al4 & 3u) != 0 ||
      (reinterpret_cast<uintptr_t>(p.trailer) & 7u) != 0)
    return;
  scan_tile(p, scratch, tile);
}

static_assert(sizeof(ScanArgs) <= kDdArgBytes, "a scan job's arguments fit one lane argument area");

inline uint32_t num_tiles(uint32_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

const void* scan_lane_func() { return reinterpret_cast<const void*>(&saxpy_scan_max_lane_kernel); }
uint32_t scan_lane_tiles(uint32_t max_n) { return num_tiles(max_n); }

bool plan_saxpy_scan_max(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk) {
  const uint32_t n = in.dims[0];
  ScanArgs a{};
  a.x = static_cast<const float*>(in.d_in);
  a.y = a.x + n;
  a.z = static_cast<float*>(in.d_out);
  a.S = a.z + n;
  a.m_out = a.S + n;
  a.trailer = reinterpret_cast<set_trailer*>(static_cast<uint8_t*>(in.d_out) + L.out_bytes - sizeof(set_trailer));
  a.scratch = static_cast<uint8_t*>(in.d_persist);
  a.job_id = in.job_id;
  a.n = n;
  a.T = num_tiles(n);
  a.a = in.scalar;
  a.slot_gen = in.slot_gen;
  a.skip_tile = (in.flags & SET_F_TEST_STALL) && a.T >= 3 ? 1u : ~0u;
  KernelLaunch& k = kl[0];
  k.func = reinterpret_cast<const void*>(&saxpy_scan_max_kernel);
  k.grid = dim3(a.T);
  k.block = dim3(kThreads);
  k.smem = 0;
  k.deps = 0;
  set_args(k, a);
  *nk = 1;
  return true;
}

// ---- scan launch whose scratch needs no allocation by anyone ----
//
// Some callers cannot call cudaMalloc or hold a scratch buffer of their own: a plugin loaded into
// a host process whose device memory belongs to another allocator (a serving framework, a
// caching allocator that must not be bypassed), or a latency-critical path where an allocation
// would synchronise the device.  For them the scan's scratch (header + per-tile status words and
// maxima) lives in this file-scope device array, sized for n <= kStaticScanMaxN.  Every GPU that
// loads the library holds it (65,792 bytes) until the process exits.
namespace {
constexpr uint32_t kStaticScanMaxN = 1u << 24;
constexpr size_t kStaticScanBytes = kScanHdrBytes + (size_t)kScanBytesPerTile * (kStaticScanMaxN / kScanTile);
constexpr int kStaticMaxDevices = 64;
__device__ __align__(256) uint8_t g_static_scan_scratch[(kStaticScanBytes + 255) & ~size_t(255)];
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};
}  // namespace

}  // namespace setk

// Host code may not use g_static_scan_scratch as an address: its device address is looked up once
// per device with cudaGetSymbolAddress (on the first call made while that device is current).
extern "C" set_status set_launch_scan_static(const set_job_desc* job, const void* d_in, void* d_out, uint64_t job_id,
                                             uint32_t slot_gen, void* stream) {
  using namespace setk;
  if (!job || !d_in || !d_out || job->type != SET_JOB_SAXPY_SCAN_MAX) {
    setrt::set_thread_error("set_launch_scan_static: needs a SET_JOB_SAXPY_SCAN_MAX descriptor and device in/out");
    return SET_EINVAL;
  }
  const uint32_t n = job->dims[0];
  if (n < 1 || n > kStaticScanMaxN) {
    setrt::set_thread_error("set_launch_scan_static: n must be in 1..16777216 (size of the static scratch array)");
    return SET_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
    cudaGetLastError();
    setrt::set_thread_error("set_launch_scan_static: no current CUDA device (or ordinal >= 64)");
    return SET_ECUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scan_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        setrt::set_thread_error("set_launch_scan_static: cudaGetSymbolAddress of the static scratch failed");
        return SET_ECUDA;
      }
      g_static_ptr[dev] = p;
    }
    scratch = g_static_ptr[dev];
  }
  JobLayout L;
  if (!job_sizes(job->type, job->dims, &L)) return SET_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear the header and status words this call uses
  if (cudaMemsetAsync(scratch, 0, L.persist_bytes, st) != cudaSuccess) {
    cudaGetLastError();
    setrt::set_thread_error("set_launch_scan_static: clearing the static scratch failed");
    return SET_ECUDA;
  }
  JobPlanIn in;
  in.type = job->type;
  in.dims[0] = n;
  in.scalar = job->scalar;
  in.d_in = d_in;
  in.d_out = d_out;
  in.d_persist = scratch;
  in.job_id = job_id;
  in.slot_gen = slot_gen;
  KernelLaunch kl[kMaxKernels];
  int nk = 0;
  if (!plan_saxpy_scan_max(in, L, kl, &nk)) return SET_EINVAL;
  if (cudaLaunchKernel(kl[0].func, kl[0].grid, kl[0].block, kl[0].params, kl[0].smem, st) != cudaSuccess) {
    cudaGetLastError();
    setrt::set_thread_error("set_launch_scan_static: kernel launch failed");
    return SET_ECUDA;
  }
  return SET_OK;
}
