// mlp_ln.cu -- MLP job: a fork/join DAG after the input copy
//   branch B  layernorm_kernel : B = (x - mu) / sqrt(var + 1e-5) per row (fp32, no affine)
//   branch A  gemm<GELU>       : h = GELU(x W1^T), BF16 inputs, FP32 accumulation, h stored BF16
//   join      gemm<JOIN>       : out = h W2^T + B  (fp32), then the trailer
// Graph edges: H2D -> {LN, GEMM1}; {LN, GEMM1} -> GEMM2 -> D2H.
//
// The GEMMs run on the 5th-generation tensor cores: TMA loads 128 x 64 (A) and BN x 64 (B) BF16
// tiles in the 128-byte swizzle layout into a multi-stage shared-memory ring (mbarrier
// full/empty pairs), one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into
// a TMEM accumulator and frees each stage with tcgen05.commit, and all four warps read the
// accumulator back with tcgen05.ld (one TMEM lane = one output row per thread) for the fused
// epilogue (exact-erf GELU -> BF16, or + LayerNorm -> FP32).  cta_group::1, no clusters, no
// multicast.  Rows past m are zero-filled by TMA and never stored.
//
// Every mbarrier wait is bounded; a wait that gives up sets an error bit in the job's control
// block, the MMA thread still commits the accumulator barrier (so nobody waits on MMAs that were
// never issued), the producer waits for its own copies before the CTA leaves, and TMEM is always
// freed.  The last GEMM2 CTA (done counter) writes the trailer with the error bits and resets the
// control block.
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include <string>

#include "../runtime/thread_error.h"
#include "stages.h"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace setk {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // one 128-byte swizzle row of BF16
constexpr int kGemmThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 22;  // polls of ~100 ns: about 0.4 s

enum : int { kEpiGelu = 0, kEpiJoin = 1 };

struct MlpCtl {  // job state in the slot control block
  uint32_t err;
  uint32_t done;
  uint32_t pad[14];
};

struct TrailerRec {  // batched form: one per job of the launch
  set_trailer* dst;
  uint64_t job_id;
  uint32_t slot_gen;
  uint32_t pad[3];
};
static_assert(sizeof(TrailerRec) == kMlpTrailerRecBytes, "trailer record size shared with the layout code");

struct GemmArgs {
  Stamp stamp;  // first member: filled by the planner
  CUtensorMap ta;  // A: rows x K, K-major, box {64, 128}
  CUtensorMap tb;  // B: N x K, K-major, box {64, BN}
  void* out;       // GELU: bf16 [M][N]; JOIN: f32 [M][N]
  const float* addend;   // JOIN: f32 [M][N] (LayerNorm of x)
  set_trailer* trailer;  // JOIN: written by the last CTA (single job)
  const TrailerRec* recs;  // JOIN, batched form: the last CTA writes every job's trailer
  uint32_t nrecs;
  MlpCtl* ctl;
  uint64_t job_id;
  uint32_t M, N, K;
  uint32_t slot_gen;
};

struct LnArgs {
  Stamp stamp;  // first member: filled by the planner
  const uint16_t* x;  // bf16 [M][1024]
  float* y;           // f32 [M][1024]
  uint32_t M;
};

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ float gelu_erf(float v) { return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f)); }

// Epilogue of NV consecutive outputs of one row: GELU -> BF16 (GEMM1) or + LayerNorm -> FP32 (join).
template <int EPI, int NV>
__device__ __forceinline__ void store_row(const GemmArgs& p, int row, int col, const float (&v)[NV]) {
  static_assert(NV % 8 == 0, "whole 16-byte stores");
  if constexpr (EPI == kEpiGelu) {
    uint16_t* dst = static_cast<uint16_t*>(p.out) + (size_t)row * p.N + col;
#pragma unroll
    for (int q = 0; q < NV / 8; ++q) {
      uint4 w;
      w.x = pack_bf16x2(gelu_erf(v[8 * q + 0]), gelu_erf(v[8 * q + 1]));
      w.y = pack_bf16x2(gelu_erf(v[8 * q + 2]), gelu_erf(v[8 * q + 3]));
      w.z = pack_bf16x2(gelu_erf(v[8 * q + 4]), gelu_erf(v[8 * q + 5]));
      w.w = pack_bf16x2(gelu_erf(v[8 * q + 6]), gelu_erf(v[8 * q + 7]));
      reinterpret_cast<uint4*>(dst)[q] = w;
    }
  } else {
    float* dst = static_cast<float*>(p.out) + (size_t)row * p.N + col;
    const float* add = p.addend + (size_t)row * p.N + col;
#pragma unroll
    for (int q = 0; q < NV / 4; ++q) {
      const float4 a = reinterpret_cast<const float4*>(add)[q];
      reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q] + a.x, v[4 * q + 1] + a.y, v[4 * q + 2] + a.z,
                                                      v[4 * q + 3] + a.w);
    }
  }
}

template <int BN, int STAGES>
struct GemmSmem {
  static constexpr size_t kA = (size_t)kBM * kBK * 2;  // 16 KiB per stage
  static constexpr size_t kB = (size_t)BN * kBK * 2;
  static constexpr size_t kTiles = STAGES * (kA + kB);
  static constexpr size_t kBytes = kTiles + 1024 /*alignment*/ + 256 /*barriers*/;
};

// SPLIT > 1: split-K over a cluster of SPLIT CTAs along z (each takes K / SPLIT); the FP32
// partial tiles are parked in each CTA's shared memory and rank r reduces rows
// [r * 128 / SPLIT, (r + 1) * 128 / SPLIT) over distributed shared memory before the epilogue.
template <int BN, int STAGES, int EPI, int SPLIT>
__global__ void __cluster_dims__(1, 1, SPLIT) __launch_bounds__(kGemmThreads, 2)
    mlp_gemm_kernel(const __grid_constant__ GemmArgs p) {
  using SM = GemmSmem<BN, STAGES>;
  static_assert(SPLIT == 1 || (size_t)kBM * BN * 4 <= SM::kTiles, "the partial tile fits the stage buffers");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * SM::kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SM::kTiles);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(accum + 1);
  uint32_t* s_err = s_tmem + 1;
  uint32_t* s_last = s_tmem + 2;

  stamp_entry(p.stamp);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
  const int nk = (int)(p.K / kBK) / SPLIT;
  const int kb0 = (int)blockIdx.z * nk;  // this CTA's share of K (in 64-wide blocks)

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(accum, 1);
    *s_err = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&p.ta);
    tc::prefetch_tmap(&p.tb);
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, BN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;

  if (warp == 0 && lane == 0) {
    // TMA producer: stage s is refilled once the MMAs that read it have completed
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !tc::mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, kWaitLimit)) {
        atomicOr(s_err, 1u);
        break;
      }
      tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(SM::kA + SM::kB));
      tc::tma_load_2d(sA + s * SM::kA, &p.ta, &full[s], (kb0 + kb) * kBK, m0);
      tc::tma_load_2d(sB + s * SM::kB, &p.tb, &full[s], (kb0 + kb) * kBK, n0);
      issued = kb + 1;
    }
    // before the CTA can leave, every copy it started must have landed
    for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
      if (!tc::mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, kWaitLimit)) atomicOr(s_err, 1u);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 x (128 x BN x 16) per 64-wide K block
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!tc::mbar_wait(&full[s], (kb / STAGES) & 1, kWaitLimit)) {
        atomicOr(s_err, 1u);
        break;
      }
      tc::fence_after_sync();
      const uint64_t da = tc::desc_sw128(sA + s * SM::kA), db = tc::desc_sw128(sB + s * SM::kB);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)  // +32 bytes per K step inside the swizzle row
        tc::mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(accum);  // always: the epilogue waits on this
  }
  __syncwarp();

  // epilogue: warp w owns accumulator rows 32w .. 32w + 31 (TMEM lanes), one row per thread
  const bool acc_ok = tc::mbar_wait(accum, 0, kWaitLimit);
  tc::fence_after_sync();
  if (!acc_ok) atomicOr(s_err, 1u);
  if constexpr (SPLIT == 1) {
    const int row = m0 + warp * 32 + lane;
    const bool row_ok = row < (int)p.M;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
      tc::tmem_ld_wait();
      if (!acc_ok || !row_ok) continue;
      float v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
      store_row<EPI, 32>(p, row, n0 + c * 32, v);
    }
  } else {
    // park the partial tile (row-major [128][BN] FP32) in this CTA's stage buffers: every MMA
    // has completed (accum barrier) and every TMA copy has landed (the producer drained them)
    __syncthreads();
    float* part = reinterpret_cast<float*>(smem);
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
      tc::tmem_ld_wait();
      float* dst = part + (size_t)(warp * 32 + lane) * BN + c * 32;
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        *reinterpret_cast<float4*>(dst + q) = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                                                          __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
    }
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    // rank r sums rows [r * 128 / SPLIT, ...) over the SPLIT partials; 4 threads per row
    constexpr int kRows = kBM / SPLIT, kTpr = kGemmThreads / kRows, kCols = BN / kTpr;
    static_assert(kGemmThreads % kRows == 0 && BN % kTpr == 0 && kCols % 8 == 0, "reduction mapping");
    const int rr = (int)cluster.block_rank() * kRows + threadIdx.x / kTpr;
    const int c0 = (threadIdx.x % kTpr) * kCols;
    const int row = m0 + rr;
    float v[kCols];
#pragma unroll
    for (int q = 0; q < kCols; ++q) v[q] = 0.f;
#pragma unroll 1
    for (int src = 0; src < SPLIT; ++src) {  // fixed order: the sum is the same in every run
      const float* rp = cluster.map_shared_rank(part, src) + (size_t)rr * BN + c0;
#pragma unroll
      for (int q = 0; q < kCols; q += 4) {
        const float4 t = *reinterpret_cast<const float4*>(rp + q);
        v[q] += t.x;
        v[q + 1] += t.y;
        v[q + 2] += t.z;
        v[q + 3] += t.w;
      }
    }
    if (acc_ok && row < (int)p.M) store_row<EPI, kCols>(p, row, n0 + c0, v);
    cluster.sync();  // keep every partial alive until all ranks have read it
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
  if (threadIdx.x == 0 && *s_err) atomicOr(&p.ctl->err, SET_DEVERR_WAIT);
  if constexpr (EPI == kEpiJoin) {
    if (threadIdx.x == 0) {
      __threadfence();
      *s_last = atomicAdd(&p.ctl->done, 1u) == gridDim.x * gridDim.y * gridDim.z - 1;
    }
    __syncthreads();
    if (*s_last) {
      __threadfence();
      __shared__ uint32_t s_errw;
      if (threadIdx.x == 0) {
        s_errw = atomicExch(&p.ctl->err, 0u);
        p.ctl->done = 0u;
      }
      __syncthreads();
      if (p.nrecs == 0) {
        if (threadIdx.x == 0) {
          p.trailer->job_id = p.job_id;
          p.trailer->slot_gen = p.slot_gen;
          p.trailer->word = trailer_word(s_errw);
        }
      } else {
        for (uint32_t r = threadIdx.x; r < p.nrecs; r += kGemmThreads) {
          const TrailerRec t = p.recs[r];
          t.dst->job_id = t.job_id;
          t.dst->slot_gen = t.slot_gen;
          t.dst->word = trailer_word(s_errw);
        }
      }
    }
  }
  stamp_exit(p.stamp);
}

// One warp per row of 1024: two-pass mean / variance in registers.
__global__ void __launch_bounds__(256) layernorm_kernel(const LnArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t row = blockIdx.x * 8 + warp;
  stamp_entry(a.stamp);  // thread 0 is warp 0, whose row always exists
  if (row >= a.M) return;
  const uint4* src = reinterpret_cast<const uint4*>(a.x + (size_t)row * kMlpD);
  float v[32];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint4 w = __ldg(src + lane + 32 * i);
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[8 * i + 2 * k] = bf16_to_f32((uint16_t)(u[k] & 0xFFFFu));
      v[8 * i + 2 * k + 1] = bf16_to_f32((uint16_t)(u[k] >> 16));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 32; ++k) s += v[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  const float mean = s * (1.0f / kMlpD);
  float q = 0.f;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float d = v[k] - mean;
    q += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
  const float inv = 1.0f / sqrtf(q * (1.0f / kMlpD) + 1e-5f);
  float4* dst = reinterpret_cast<float4*>(a.y + (size_t)row * kMlpD);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    dst[2 * (lane + 32 * i)] = make_float4((v[8 * i] - mean) * inv, (v[8 * i + 1] - mean) * inv,
                                           (v[8 * i + 2] - mean) * inv, (v[8 * i + 3] - mean) * inv);
    dst[2 * (lane + 32 * i) + 1] = make_float4((v[8 * i + 4] - mean) * inv, (v[8 * i + 5] - mean) * inv,
                                               (v[8 * i + 6] - mean) * inv, (v[8 * i + 7] - mean) * inv);
  }
  stamp_exit(a.stamp);
}

// ---- host side ----
// Stage rings of 96 KiB let two CTAs share an SM (one's epilogue overlaps the other's main loop).
constexpr int kBN1 = 128, kStages1 = 3;  // GEMM1: 1024 -> 4096
constexpr int kBN2 = 64, kStages2 = 4;   // GEMM2: 4096 -> 1024 (narrower tiles: more CTAs)
constexpr int kSplit2 = 4;               // GEMM2 split-K for one job (m <= 256: 16 N-tiles only)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D BF16 K-major operand: `rows` rows of `k` elements (row pitch k * 2 bytes), box {64, box_rows}.
bool make_map(CUtensorMap* m, const void* base, uint64_t k, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (k * 2) % 16) {
    setrt::set_thread_error(!fn ? "cuTensorMapEncodeTiled unavailable" : "tensor map base null or misaligned");
    return false;
  }
  const cuuint64_t dims[2] = {k, rows};
  const cuuint64_t strides[1] = {k * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    const std::string msg = "cuTensorMapEncodeTiled failed: CUresult " + std::to_string((int)r) + " base " +
                            std::to_string(reinterpret_cast<uintptr_t>(base)) + " k " + std::to_string(k) +
                            " rows " + std::to_string(rows) + " map@" + std::to_string(reinterpret_cast<uintptr_t>(m));
    setrt::set_thread_error(msg.c_str());
    return false;
  }
  return true;
}

// Weight maps are the same for every job that shares the weights: keep the last one per operand.
// (A process-wide cache under a mutex: thread-local storage of a dlopen'd library need not honour
// the 64-byte alignment that cuTensorMapEncodeTiled requires of its output.)
bool weight_map(CUtensorMap* m, const void* w, uint64_t k, uint64_t rows, uint32_t box_rows, int which) {
  static std::mutex mu;
  static const void* key[2] = {nullptr, nullptr};
  alignas(64) static CUtensorMap maps[2];
  std::lock_guard<std::mutex> g(mu);
  if (key[which] != w) {
    alignas(64) CUtensorMap tmp;
    if (!make_map(&tmp, w, k, rows, box_rows)) return false;
    maps[which] = tmp;
    key[which] = w;
  }
  *m = maps[which];
  return true;
}

template <int BN, int STAGES, int EPI, int SPLIT = 1>
void fill_gemm(KernelLaunch& k, const GemmArgs& a, uint32_t deps) {
  k.func = reinterpret_cast<const void*>(&mlp_gemm_kernel<BN, STAGES, EPI, SPLIT>);
  k.grid = dim3(a.N / BN, (a.M + kBM - 1) / kBM, SPLIT);
  k.block = dim3(kGemmThreads);
  k.smem = (unsigned)GemmSmem<BN, STAGES>::kBytes;
  k.deps = deps;
  set_args(k, a);
}

}  // namespace

bool plan_mlp_ln(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk) {
  const uint32_t m = in.dims[0];
  const uint16_t* x = static_cast<const uint16_t*>(in.d_in);
  const uint16_t* w1 = static_cast<const uint16_t*>(in.shared[0]);
  const uint16_t* w2 = static_cast<const uint16_t*>(in.shared[1]);
  const size_t mp = (m + kBM - 1) / kBM * kBM;
  uint16_t* h = static_cast<uint16_t*>(in.d_scratch);
  float* ln = reinterpret_cast<float*>(static_cast<uint8_t*>(in.d_scratch) + align256(mp * kMlpF * 2));
  MlpCtl* ctl = static_cast<MlpCtl*>(in.d_persist);

  LnArgs la{Stamp{}, x, ln, m};
  KernelLaunch& k0 = kl[0];
  k0.func = reinterpret_cast<const void*>(&layernorm_kernel);
  k0.grid = dim3((m + 7) / 8);
  k0.block = dim3(256);
  k0.smem = 0;
  k0.deps = 0;
  set_args(k0, la);

  GemmArgs g1{};
  GemmArgs g2{};
  if (!make_map(&g1.ta, x, kMlpD, m, kBM) || !weight_map(&g1.tb, w1, kMlpD, kMlpF, kBN1, 0) ||
      !make_map(&g2.ta, h, kMlpF, m, kBM) || !weight_map(&g2.tb, w2, kMlpF, kMlpD, kBN2, 1))
    return false;
  g1.out = h;
  g1.ctl = ctl;
  g1.M = m;
  g1.N = kMlpF;
  g1.K = kMlpD;
  g2.out = in.d_out;
  g2.addend = ln;
  g2.trailer = reinterpret_cast<set_trailer*>(static_cast<uint8_t*>(in.d_out) + L.out_bytes - sizeof(set_trailer));
  g2.ctl = ctl;
  g2.job_id = in.job_id;
  g2.slot_gen = in.slot_gen;
  g2.M = m;
  g2.N = kMlpD;
  g2.K = kMlpF;
  fill_gemm<kBN1, kStages1, kEpiGelu>(kl[1], g1, 0);
  fill_gemm<kBN2, kStages2, kEpiJoin, kSplit2>(kl[2], g2, (1u << 0) | (1u << 1));
  *nk = 3;
  return true;
}

cudaError_t mlp_init() {
  const struct {
    const void* f;
    size_t smem;
  } fs[] = {
      {reinterpret_cast<const void*>(&mlp_gemm_kernel<kBN1, kStages1, kEpiGelu, 1>), GemmSmem<kBN1, kStages1>::kBytes},
      {reinterpret_cast<const void*>(&mlp_gemm_kernel<kBN2, kStages2, kEpiJoin, 1>), GemmSmem<kBN2, kStages2>::kBytes},
      {reinterpret_cast<const void*>(&mlp_gemm_kernel<kBN2, kStages2, kEpiJoin, kSplit2>),
       GemmSmem<kBN2, kStages2>::kBytes},
  };
  for (const auto& f : fs) {
    const cudaError_t e = cudaFuncSetAttribute(f.f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Batched form: the rows of nb jobs packed into one M = sum(m_j + 1); the same three kernels run
// over the packed rows.  Job j owns rows [R_j, R_j + m_j); its spare row R_j + m_j is computed
// like any other row (rows are independent) and its first 16 bytes are then overwritten with the
// job's trailer by the last GEMM2 CTA, so one D2H copy returns rows and trailer.
bool plan_mlp_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, const void* w1v, const void* w2v, KernelLaunch* kl, int* nk) {
  std::memset(h_table, 0, L.table_bytes);
  MlpCtl* ctl = reinterpret_cast<MlpCtl*>(d_block);
  const TrailerRec* recs = reinterpret_cast<const TrailerRec*>(d_block + kMlpCtlBytes);
  for (int j = 0; j < nb; ++j) {
    TrailerRec t{};
    t.dst = reinterpret_cast<set_trailer*>(d_block + L.out_off[j] + (size_t)items[j].dims[0] * kMlpD * 4);
    t.job_id = items[j].job_id;
    t.slot_gen = slot_gen;
    std::memcpy(h_table + kMlpCtlBytes + (size_t)j * sizeof(TrailerRec), &t, sizeof t);
  }
  const uint32_t M = (uint32_t)L.rows;
  const size_t x_off = L.table_bytes;
  const size_t h_off = x_off + align256((size_t)M * kMlpD * 2);
  const size_t ln_off = h_off + align256((size_t)M * kMlpF * 2);
  const size_t o_off = ln_off + align256((size_t)M * kMlpD * 4);
  const uint16_t* x = reinterpret_cast<const uint16_t*>(d_block + x_off);
  uint16_t* h = reinterpret_cast<uint16_t*>(d_block + h_off);
  float* ln = reinterpret_cast<float*>(d_block + ln_off);
  LnArgs la{Stamp{}, x, ln, M};
  KernelLaunch& k0 = kl[0];
  k0.func = reinterpret_cast<const void*>(&layernorm_kernel);
  k0.grid = dim3((M + 7) / 8);
  k0.block = dim3(256);
  k0.smem = 0;
  k0.deps = 0;
  set_args(k0, la);
  GemmArgs g1{};
  GemmArgs g2{};
  if (!make_map(&g1.ta, x, kMlpD, M, kBM) || !weight_map(&g1.tb, w1v, kMlpD, kMlpF, kBN1, 0) ||
      !make_map(&g2.ta, h, kMlpF, M, kBM) || !weight_map(&g2.tb, w2v, kMlpF, kMlpD, kBN2, 1))
    return false;
  g1.out = h;
  g1.ctl = ctl;
  g1.M = M;
  g1.N = kMlpF;
  g1.K = kMlpD;
  g2.out = d_block + o_off;
  g2.addend = ln;
  g2.recs = recs;
  g2.nrecs = (uint32_t)nb;
  g2.ctl = ctl;
  g2.M = M;
  g2.N = kMlpD;
  g2.K = kMlpF;
  fill_gemm<kBN1, kStages1, kEpiGelu>(kl[1], g1, 0);
  fill_gemm<kBN2, kStages2, kEpiJoin>(kl[2], g2, (1u << 0) | (1u << 1));
  *nk = 3;
  return true;
}

}  // namespace setk
