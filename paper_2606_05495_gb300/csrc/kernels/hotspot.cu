// hotspot.cu -- hotspot job: K explicit Euler steps of the compact thermal RC grid of the HotSpot
// model (Huang et al. 2006), the iterative thermal simulation Sec. 5.1.2 lists among its
// workloads.  For an R x C grid of cells over a silicon die, with dx = width / C, dy = height / R:
//   Gx = k t dy / dx, Gy = k t dx / dy (lateral conductances), Gz = k dx dy / t (to the ambient),
//   Cap = c_v t dx dy, dt = 0.2 Cap / (2 Gx + 2 Gy + Gz),
//   T' = T + dt/Cap P + dt/Cap Gy (T_N + T_S - 2T) + dt/Cap Gx (T_W + T_E - 2T) + dt/Cap Gz (T_amb - T),
// a neighbour outside the die being the cell itself (adiabatic edges).  Die 16 x 16 x 0.5 mm,
// k = 100 W/(m K), c_v = 1.75e6 J/(m^3 K), T_amb = 80.  FP32 arithmetic.
//
// Temporal blocking: one launch advances the grid up to kHotStepsPerLaunch steps.  Each CTA
// stages the (64 + 2h) x (64 + 2h) window of T and P around its 64 x 64 output tile (h = 8,
// 16-byte cp.async copies when rows allow), turns P into q = dt/Cap P + dt Gz/Cap T_amb, runs the
// steps in shared memory over a region that shrinks by one cell per step (a cell's new value needs
// its neighbours' old values) and writes its tile.  Thread t owns a group of four columns of one
// of sixteen 5-row strips and walks down it with the group's north / centre / south rows in
// float4 registers (two 128-bit and two 32-bit shared loads per four cells).  CTAs whose window
// lies inside the die skip the edge selects.  Neighbour reads clamp to the die, so staged cells outside it are never read.  A job
// is kHotLaunches launches that alternate between the slot's scratch buffer and the output; the
// last CTA of the last launch writes the zero pad and the trailer.
#include "cp_async.cuh"
#include "stages.h"

namespace setk {
namespace {

constexpr int kTile = 64;
constexpr int kHalo = kHotStepsPerLaunch;
constexpr int kS = kTile + 2 * kHalo;  // staged window side
constexpr int kGroups = kS / 4;        // four-column groups across the window
constexpr int kStrips = 16;            // row strips of the window; a thread per (group, strip)
constexpr int kStripRows = kS / kStrips;
constexpr int kThreads = kGroups * kStrips;
static_assert(kS % kStrips == 0 && kS % 4 == 0, "strips and groups tile the window");
constexpr unsigned kSmemBytes = 3u * kS * kS * sizeof(float);  // two T buffers and q
static_assert(kS % 4 == 0 && kHalo % 4 == 0, "16-byte staging needs 4-cell aligned windows");

struct HotArgs {
  Stamp stamp;  // first member: filled by the planner
  const float* tin;
  const float* p;
  float* tout;
  uint32_t C, R, steps;
  float cx, cy, cz, cp, tamb;  // dt Gx / Cap, dt Gy / Cap, dt Gz / Cap, dt / Cap, T_amb
  uint32_t* done;              // last launch: CTAs-done counter in the slot's control block; else null
  uint8_t* pad;                // last launch: zero bytes between T and the trailer
  uint32_t npad;
  set_trailer* trailer;
  uint64_t job_id;
  uint32_t slot_gen;
};


// dst[r][c] = src[gy0 + r][gx0 + c] for the window cells inside the die; the others are left.
__device__ void stage(float* dst, const float* __restrict__ src, int C, int R, int gx0, int gy0, bool vec) {
  if (vec) {  // C % 4 == 0, src 16-byte aligned, gx0 % 4 == 0: a 4-cell group is in or out whole
    constexpr int Q = kS / 4;
    for (int i = threadIdx.x; i < kS * Q; i += kThreads) {
      const int r = i / Q, q = i - r * Q;
      const int gy = gy0 + r, gx = gx0 + 4 * q;
      if (gy < 0 || gy >= R || gx < 0 || gx >= C) continue;
      cp_async16(dst + r * kS + 4 * q, src + (size_t)gy * C + gx);
    }
  } else {
    for (int i = threadIdx.x; i < kS * kS; i += kThreads) {
      const int r = i / kS, c = i - r * kS;
      const int gy = gy0 + r, gx = gx0 + c;
      if (gy < 0 || gy >= R || gx < 0 || gx >= C) continue;
      cp_async4(dst + i, src + (size_t)gy * C + gx);
    }
  }
}

// One explicit step over this thread's rows of the region [s, kS - s)^2.  Groups that reach into
// the region compute all four columns: the cells outside it are never read again.  EDGE: the
// window touches the die's border, so neighbours clamp to the die (adiabatic edges).
template <bool EDGE>
__device__ __forceinline__ void step(const float* __restrict__ cur, float* __restrict__ nxt, const float* __restrict__ qs,
                                     int s, int grp, int g, int gx0, int gy0, int C, int R, float cx, float cy,
                                     float cz) {
  const int c0 = 4 * grp;
  const int r0 = max(g * kStripRows, s), r1 = min((g + 1) * kStripRows, kS - s);
  if (c0 + 3 < s || c0 >= kS - s || r0 >= r1) return;
  bool west[4], east[4];  // the neighbour exists on the die
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    west[k] = !EDGE || gx0 + c0 + k > 0;
    east[k] = !EDGE || gx0 + c0 + k < C - 1;
  }
  const float4* cur4 = reinterpret_cast<const float4*>(cur);
  float4 up = cur4[((r0 - 1) * kS + c0) / 4], mid = cur4[(r0 * kS + c0) / 4];
#pragma unroll 5
  for (int r = r0; r < r1; ++r) {
    const int i = r * kS + c0;  // in-bounds: 1 <= r <= kS - 2, and i + 4 <= (r + 1) * kS
    const float4 dn = cur4[(i + kS) / 4];
    const float4 q = reinterpret_cast<const float4*>(qs)[i / 4];
    const float w = cur[i - 1], e = cur[i + 4];  // c0 = kS - 4: the next row's first cell, never in a region
    const bool north = !EDGE || gy0 + r > 0, south = !EDGE || gy0 + r < R - 1;
    const float m[4] = {mid.x, mid.y, mid.z, mid.w}, u[4] = {up.x, up.y, up.z, up.w}, d[4] = {dn.x, dn.y, dn.z, dn.w};
    const float qq[4] = {q.x, q.y, q.z, q.w};
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float t = m[k];
      const float tn = north ? u[k] : t, ts = south ? d[k] : t;
      const float tw = west[k] ? (k == 0 ? w : m[k - 1]) : t, te = east[k] ? (k == 3 ? e : m[k + 1]) : t;
      float acc = fmaf(cy, (tn + ts) - 2.f * t, qq[k]);
      acc = fmaf(cx, (tw + te) - 2.f * t, acc);
      acc = fmaf(-cz, t, acc);
      o[k] = t + acc;
    }
    reinterpret_cast<float4*>(nxt)[i / 4] = make_float4(o[0], o[1], o[2], o[3]);
    up = mid;
    mid = dn;
  }
}

__global__ void __launch_bounds__(kThreads, 2) hotspot_kernel(const HotArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* cur = sm;
  float* nxt = sm + kS * kS;
  float* qs = sm + 2 * kS * kS;
  stamp_entry(a.stamp);
  const int C = (int)a.C, R = (int)a.R;
  const int tx = blockIdx.x * kTile, ty = blockIdx.y * kTile;
  const int gx0 = tx - kHalo, gy0 = ty - kHalo;
  const bool vec = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.tin) | reinterpret_cast<uintptr_t>(a.p) |
                                     reinterpret_cast<uintptr_t>(a.tout)) & 15) == 0;
  stage(cur, a.tin, C, R, gx0, gy0, vec);
  stage(qs, a.p, C, R, gx0, gy0, vec);
  cp_async_wait_all();
  __syncthreads();
  {
    const float cp = a.cp, czt = a.cz * a.tamb;
    float4* q4 = reinterpret_cast<float4*>(qs);
    for (int i = threadIdx.x; i < kS * kS / 4; i += kThreads) {  // cells off the die: unused
      const float4 p = q4[i];
      q4[i] = make_float4(fmaf(cp, p.x, czt), fmaf(cp, p.y, czt), fmaf(cp, p.z, czt), fmaf(cp, p.w, czt));
    }
  }
  __syncthreads();
  const int grp = threadIdx.x % kGroups, g = threadIdx.x / kGroups;
  const bool edge = gx0 < 0 || gy0 < 0 || gx0 + kS > C || gy0 + kS > R;
  for (int s = 1; s <= (int)a.steps; ++s) {
    if (edge)
      step<true>(cur, nxt, qs, s, grp, g, gx0, gy0, C, R, a.cx, a.cy, a.cz);
    else
      step<false>(cur, nxt, qs, s, grp, g, gx0, gy0, C, R, a.cx, a.cy, a.cz);
    __syncthreads();
    float* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  if (vec) {
    constexpr int Q = kTile / 4;
    for (int i = threadIdx.x; i < kTile * Q; i += kThreads) {
      const int r = i / Q, c = 4 * (i - r * Q);
      const int gy = ty + r, gx = tx + c;
      if (gy >= R || gx >= C) continue;
      *reinterpret_cast<float4*>(a.tout + (size_t)gy * C + gx) =
          *reinterpret_cast<const float4*>(cur + (r + kHalo) * kS + c + kHalo);
    }
  } else {
    for (int i = threadIdx.x; i < kTile * kTile; i += kThreads) {
      const int r = i / kTile, c = i - r * kTile;
      const int gy = ty + r, gx = tx + c;
      if (gy >= R || gx >= C) continue;
      a.tout[(size_t)gy * C + gx] = cur[(r + kHalo) * kS + c + kHalo];
    }
  }
  if (a.done) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(a.done, 1u) == gridDim.x * gridDim.y - 1u) {
      __threadfence();
      for (uint32_t b = 0; b < a.npad; ++b) a.pad[b] = 0;
      a.trailer->job_id = a.job_id;
      a.trailer->slot_gen = a.slot_gen;
      a.trailer->word = trailer_word(0);
      *a.done = 0u;  // ready for the slot's next hotspot job
    }
  }
  stamp_exit(a.stamp);
}

// Model constants (SI units; temperatures in degrees).
constexpr double kDieW = 0.016, kDieH = 0.016, kThick = 0.0005, kKSi = 100.0, kCvSi = 1.75e6, kTAmb = 80.0;
constexpr double kDtFrac = 0.2;

}  // namespace

cudaError_t hotspot_init() {
  return cudaFuncSetAttribute(hotspot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

bool plan_hotspot(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk) {
  const uint32_t C = in.dims[0], R = in.dims[1], K = in.dims[2];
  if (C < 1 || R < 1 || K < 1 || K > (uint32_t)kHotMaxSteps) return false;
  const double dx = kDieW / C, dy = kDieH / R;
  const double gx = kKSi * kThick * dy / dx, gy = kKSi * kThick * dx / dy, gz = kKSi * dx * dy / kThick;
  const double cap = kCvSi * kThick * dx * dy;
  const double dt = kDtFrac * cap / (2.0 * gx + 2.0 * gy + gz);
  const size_t cells = (size_t)C * R;
  const float* t0 = static_cast<const float*>(in.d_in);
  float* out = static_cast<float*>(in.d_out);
  float* scratch = static_cast<float*>(in.d_scratch);
  const float* src = t0;
  for (int k = 0; k < kHotLaunches; ++k) {
    HotArgs a{};
    a.tin = src;
    a.p = t0 + cells;
    a.tout = ((kHotLaunches - 1 - k) % 2 == 0) ? out : scratch;  // the last launch writes the output
    a.C = C;
    a.R = R;
    a.steps = (uint32_t)(((uint64_t)K * (k + 1)) / kHotLaunches - ((uint64_t)K * k) / kHotLaunches);
    a.cx = (float)(dt * gx / cap);
    a.cy = (float)(dt * gy / cap);
    a.cz = (float)(dt * gz / cap);
    a.cp = (float)(dt / cap);
    a.tamb = (float)kTAmb;
    if (k == kHotLaunches - 1) {
      a.done = reinterpret_cast<uint32_t*>(in.d_persist);
      a.pad = reinterpret_cast<uint8_t*>(out + cells);
      a.npad = (uint32_t)(L.out_bytes - sizeof(set_trailer) - 4 * cells);
      a.trailer = reinterpret_cast<set_trailer*>(static_cast<uint8_t*>(in.d_out) + L.out_bytes - sizeof(set_trailer));
      a.job_id = in.job_id;
      a.slot_gen = in.slot_gen;
    }
    KernelLaunch& kn = kl[k];
    kn.func = reinterpret_cast<const void*>(&hotspot_kernel);
    kn.grid = dim3((C + kTile - 1) / kTile, (R + kTile - 1) / kTile);
    kn.block = dim3(kThreads);
    kn.smem = kSmemBytes;
    kn.deps = k == 0 ? 0u : 1u << (k - 1);
    set_args(kn, a);
    src = a.tout;
  }
  *nk = kHotLaunches;
  return true;
}

}  // namespace setk
