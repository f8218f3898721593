// img_sobel_hist.cu -- image job: gray = (77R + 150G + 29B) >> 8, 5x5 Gaussian [1,4,6,4,1] (x)
// [1,4,6,4,1] >> 8, Sobel min(|gx| + |gy|, 255), 256-bin histogram of the Sobel image.  Every
// stage clamps its own input at the border (replicate edge).
//
// Two forms over the same device functions:
//   - per stage: gray_kernel, gauss_kernel, sobel_hist_kernel (three graph nodes in a chain);
//   - fused: img_fused_kernel computes RGB -> Sobel + histogram per tile with a 3-pixel halo, and
//     takes a table of jobs, so one persistent launch can carry many uneven images (the batched
//     form).  CTAs pull work items (a band of up to 32 rows x 512 columns of one job) from an
//     atomic ticket, stage tiles of 32 x 128 output pixels in shared memory and never write the
//     gray or Gaussian images to global memory.
//
// Clamping in the fused halo: the Sobel stencil needs the Gaussian *of the border pixel* at
// out-of-image positions (q[cl(y)][cl(x)]), not a Gaussian evaluated at an outside coordinate.
// The Gaussian tile is therefore evaluated at the clamped centre of every halo position; the gray
// tile holds g[cl(Y)][cl(X)] for every staged coordinate, so clamp(centre) + offset reproduces the
// per-stage definition exactly.
//
// Histogram: per-warp privatised shared histograms; at the end of a work item the CTA adds its
// non-zero bins into the job's accumulator (persistent per-job state, zero at kernel start); the
// CTA that completes the job's last item (items-done counter) copies the accumulator into the
// job's output, zeroes it and resets the counter, then writes the pad and the trailer.  The last
// CTA to leave resets the ticket.  No zeroing pass, no memset node.
#include <algorithm>
#include <cstring>

#include "cp_async.cuh"
#include "stages.h"

namespace setk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRB = 32;   // output rows of a tile (= band rows)
constexpr int kTW = 128;  // output columns of a tile
static_assert(kRB == kImgBandRows, "band rows shared with the layout code");
static_assert(kImgChunkCols % kTW == 0, "a work item is a whole number of tiles wide");

struct ImgJobDev {
  const uint8_t* rgb;
  uint8_t* out;         // Sobel image, W*H bytes
  uint8_t* pad;         // zero bytes up to the histogram
  uint32_t* hist;       // 256 u32
  set_trailer* trailer;
  uint32_t* acc;        // persistent [256] accumulator, acc[256] = items done
  uint64_t job_id;
  uint32_t W, H;
  uint32_t item0, nitems;  // first global work item of this job, number of items
  uint32_t chunks;         // column chunks per band
  uint32_t slot_gen, npad;
  uint32_t chunk_cols;     // columns of one work item (a multiple of the tile width)
};

static_assert(sizeof(ImgJobDev) <= kImgJobDescBytes, "job descriptor fits its table stride");

struct ImgHdr {
  uint32_t ticket;
  uint32_t pad[15];
};
static_assert(sizeof(ImgHdr) == kImgHdrBytes, "image header size shared with the layout code");

struct ImgFusedArgs {
  Stamp stamp;  // first member: filled by the planner
  const ImgJobDev* table;  // device table of njobs entries, or nullptr: use `one`
  ImgHdr* hdr;
  uint32_t njobs, total_items;
  uint32_t direct;  // 1: CTA b runs work item b once (grid = total_items), no ticket
  ImgJobDev one;
};

struct SobelHistArgs {
  Stamp stamp;  // first member: filled by the planner
  ImgFusedArgs a;
  const uint8_t* q;  // Gaussian image
};

struct GrayArgs {
  Stamp stamp;  // first member: filled by the planner
  const uint8_t* rgb;
  uint8_t* gray;
  size_t px;
};

struct GaussArgs {
  Stamp stamp;  // first member: filled by the planner
  const uint8_t* g;
  uint8_t* q;
  uint32_t W, H;
};

__device__ __forceinline__ int clampi(int v, int n) { return min(max(v, 0), n - 1); }

__device__ __forceinline__ uint32_t gray_of(uint32_t r, uint32_t g, uint32_t b) { return (77u * r + 150u * g + 29u * b) >> 8; }

// g_s[r][c] = gray(rgb[cl(y0 + r)][cl(x0 + c)]) for r < GR, c < GC.
template <int GR, int GC, int P>
__device__ void stage_gray(uint8_t (*g_s)[P], const uint8_t* __restrict__ rgb, int W, int H, int y0, int x0) {
  for (int i = threadIdx.x; i < GR * GC; i += kThreads) {
    const int r = i / GC, c = i - r * GC;
    const uint8_t* p = rgb + 3 * ((size_t)clampi(y0 + r, H) * W + clampi(x0 + c, W));
    g_s[r][c] = (uint8_t)gray_of(__ldg(p), __ldg(p + 1), __ldg(p + 2));
  }
}


// Words of 16 bytes that one staged RGB row run occupies in shared memory: up to 15 bytes of lead
// (the run starts anywhere inside its first 16-byte word) plus 3 * GC bytes, rounded up.
template <int GC>
__host__ __device__ constexpr int raw_words() { return (15 + 3 * GC + 15) / 16; }

// stage_gray for an RGB buffer that starts on a 16-byte boundary.  Staged row r holds the image
// row cl(y0 + r) over the columns [xs, xe) = [x0, x0 + GC) clipped to the image; its bytes are
// copied with 16-byte cp.async (all of a thread's copies in flight at once, one memory latency per
// tile) from the 16-byte word that contains the run's first byte.  A copy whose word would pass
// the end of the image is done bytewise, keeping only the run's own bytes.  The conversion then
// reads the clamped column cl(x0 + c), which always lies in [xs, xe).
template <int GR, int GC, int P, int RW>
__device__ void stage_gray_async(uint8_t (*g_s)[P], uint4 (*raw_s)[RW], const uint8_t* __restrict__ rgb, int W,
                                 int H, int y0, int x0) {
  static_assert(RW >= raw_words<GC>(), "raw row holds the run and its lead");
  const int xs = max(x0, 0), xe = min(x0 + GC, W);
  const int nbytes = 3 * (xe - xs);
  const uint8_t* end = rgb + 3 * (size_t)W * H;
  for (int i = threadIdx.x; i < GR * RW; i += kThreads) {
    const int r = i / RW, w = i - r * RW;
    const uint8_t* run = rgb + 3 * ((size_t)clampi(y0 + r, H) * W + xs);
    const uint8_t* a0 = run - (reinterpret_cast<uintptr_t>(run) & 15);
    const int lead = (int)(run - a0);
    if (16 * w >= lead + nbytes) continue;
    const uint8_t* src = a0 + 16 * w;
    if (src + 16 <= end) {
      cp_async16(&raw_s[r][w], src);
    } else {
      uint8_t* dst = reinterpret_cast<uint8_t*>(&raw_s[r][w]);
      for (int b = 0; b < 16; ++b) {
        const int off = 16 * w + b - lead;
        if (off >= 0 && off < nbytes) dst[b] = __ldg(src + b);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < GR * GC; i += kThreads) {
    const int r = i / GC, c = i - r * GC;
    const uint8_t* run = rgb + 3 * ((size_t)clampi(y0 + r, H) * W + xs);
    const int lead = (int)(reinterpret_cast<uintptr_t>(run) & 15);
    const uint8_t* b = reinterpret_cast<const uint8_t*>(raw_s[r]) + lead + 3 * (clampi(x0 + c, W) - xs);
    g_s[r][c] = (uint8_t)gray_of(b[0], b[1], b[2]);
  }
}

// s_s[r][c] = img[cl(y0 + r)][cl(x0 + c)] for r < R, c < C.
template <int R, int C, int P>
__device__ void stage_u8(uint8_t (*s_s)[P], const uint8_t* __restrict__ img, int W, int H, int y0, int x0) {
  for (int i = threadIdx.x; i < R * C; i += kThreads) {
    const int r = i / C, c = i - r * C;
    s_s[r][c] = __ldg(img + (size_t)clampi(y0 + r, H) * W + clampi(x0 + c, W));
  }
}

// Gaussian of the QR x QC positions starting at (qy0, qx0), each evaluated at its clamped centre:
// q_s[r][c] = (sum_ij w_i w_j g[cl(cl(qy0+r)+i)][cl(cl(qx0+c)+j)]) >> 8, where g_s[r][c] holds
// g[cl(gy0 + r)][cl(gx0 + c)].  Separable in exact integer arithmetic (vertical then horizontal).
template <int QR, int QC, int GC, int GP, int VP, int QP>
__device__ void gauss_tile(uint8_t (*q_s)[QP], const uint8_t (*g_s)[GP], uint16_t (*v_s)[VP], int W, int H, int qy0,
                           int qx0, int gy0, int gx0) {
  for (int i = threadIdx.x; i < QR * GC; i += kThreads) {
    const int r = i / GC, c = i - r * GC;
    const int cy = clampi(qy0 + r, H) - gy0;
    const uint32_t v = (uint32_t)g_s[cy - 2][c] + 4u * g_s[cy - 1][c] + 6u * g_s[cy][c] + 4u * g_s[cy + 1][c] +
                       (uint32_t)g_s[cy + 2][c];
    v_s[r][c] = (uint16_t)v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < QR * QC; i += kThreads) {
    const int r = i / QC, c = i - r * QC;
    const int cx = clampi(qx0 + c, W) - gx0;
    const uint32_t s = (uint32_t)v_s[r][cx - 2] + 4u * v_s[r][cx - 1] + 6u * v_s[r][cx] + 4u * v_s[r][cx + 1] +
                       (uint32_t)v_s[r][cx + 2];
    q_s[r][c] = (uint8_t)(s >> 8);
  }
}

// Sobel of the tile's output pixels: thread t computes 16 pixels of row t / (TW / 16).  q_s[r][c]
// holds q[cl(y0 - 1 + r)][cl(x0 - 1 + c)].  Writes the pixels inside the image and counts them.
template <int QP, int TW = kTW>
__device__ void sobel_tile(const uint8_t (*q_s)[QP], uint8_t* __restrict__ out, uint32_t (*whist)[256], int W, int H,
                           int y0, int x0, bool vec) {
  constexpr int kSegs = TW / 16;
  const int r = threadIdx.x / kSegs, s = (threadIdx.x % kSegs) << 4;
  const int y = y0 + r;
  if (y >= H || x0 + s >= W) return;
  const uint8_t* a = q_s[r] + s;  // row y-1, columns x-1 ..
  const uint8_t* b = q_s[r + 1] + s;
  const uint8_t* c = q_s[r + 2] + s;
  uint32_t o[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int gx = ((int)a[k + 2] + 2 * b[k + 2] + c[k + 2]) - ((int)a[k] + 2 * b[k] + c[k]);
    const int gy = ((int)c[k] + 2 * c[k + 1] + c[k + 2]) - ((int)a[k] + 2 * a[k + 1] + a[k + 2]);
    const uint32_t m = (uint32_t)min(abs(gx) + abs(gy), 255);
    o[k >> 2] |= m << (8 * (k & 3));
  }
  uint8_t* dst = out + (size_t)y * W + x0 + s;
  const int nvalid = min(16, W - (x0 + s));
  uint32_t(*h)[256] = whist;
  const int w = threadIdx.x >> 5;
  if (vec && nvalid == 16) {
    *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
  } else {
    for (int k = 0; k < nvalid; ++k) dst[k] = (uint8_t)(o[k >> 2] >> (8 * (k & 3)));
  }
  for (int k = 0; k < nvalid; ++k) atomicAdd(&h[w][(o[k >> 2] >> (8 * (k & 3))) & 0xFFu], 1u);
}

// Next work item of this CTA.  Direct launches: CTA b takes item b on its first pass.  Otherwise
// items come from the atomic ticket; the last CTA to leave resets it.  False: the CTA is done.
__device__ __forceinline__ bool next_item(const ImgFusedArgs& a, uint32_t pass, uint32_t* s_item, uint32_t* item) {
  if (a.direct) {
    *item = blockIdx.x;
    return pass == 0 && blockIdx.x < a.total_items;
  }
  __syncthreads();
  if (threadIdx.x == 0) *s_item = atomicAdd(&a.hdr->ticket, 1u);
  __syncthreads();
  *item = *s_item;
  if (*item < a.total_items) return true;
  if (threadIdx.x == 0 && *item == a.total_items + gridDim.x - 1) a.hdr->ticket = 0u;
  return false;
}

__device__ __forceinline__ const ImgJobDev& find_job(const ImgFusedArgs& a, uint32_t item) {
  if (!a.table) return a.one;
  uint32_t lo = 0, hi = a.njobs - 1;  // last job with item0 <= item
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (a.table[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return a.table[lo];
}

// Adds the CTA's histogram into the job accumulator; the CTA finishing the job's last item
// publishes the histogram, pad and trailer and leaves the accumulator zeroed.
__device__ void finish_item(const ImgJobDev& j, uint32_t (*whist)[256], uint32_t* s_flag) {
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += kThreads) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      t += whist[w][b];
      whist[w][b] = 0;
    }
    if (t) atomicAdd(&j.acc[b], t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = atomicAdd(&j.acc[256], 1u) == j.nitems - 1;
  __syncthreads();
  if (*s_flag) {
    __threadfence();
    for (int b = threadIdx.x; b < 256; b += kThreads) {
      j.hist[b] = atomicExch(&j.acc[b], 0u);
    }
    if (threadIdx.x < (int)j.npad) j.pad[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      j.acc[256] = 0u;
      j.trailer->job_id = j.job_id;
      j.trailer->slot_gen = j.slot_gen;
      j.trailer->word = trailer_word(0);
    }
  }
}

// Tile shapes of the fused kernel (rows x columns, 4096 outputs for 256 threads x 16 pixels); the
// work item is a band of RB rows x up to kImgChunkCols columns.  The autotuner picks one.
template <int RB, int TW>
__device__ __forceinline__ void img_fused_body(const ImgFusedArgs& a) {
  static_assert(RB * TW == kThreads * 16, "one 16-pixel segment per thread");
  constexpr int GR = RB + 6, GC = TW + 6, QR = RB + 2, QC = TW + 2, P = TW + 8;
  constexpr int RW = raw_words<GC>();
  __shared__ __align__(16) uint8_t g_s[GR][P];
  __shared__ __align__(16) uint4 raw_s[GR][RW];
  __shared__ __align__(16) uint16_t v_s[QR][P];
  __shared__ __align__(16) uint8_t q_s[QR][P];
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t s_item, s_flag;
  stamp_entry(a.stamp);
  for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&whist[0][0])[i] = 0u;
  __syncthreads();
  for (uint32_t pass = 0;; ++pass) {
    uint32_t item;
    if (!next_item(a, pass, &s_item, &item)) {
      stamp_exit(a.stamp);
      return;
    }
    const ImgJobDev& j = find_job(a, item);
    const int W = (int)j.W, H = (int)j.H;
    const uint32_t local = item - j.item0;
    const int band = (int)(local / j.chunks), chunk = (int)(local - (uint32_t)band * j.chunks);
    const int y0 = band * RB;
    const int xa = chunk * (int)j.chunk_cols, xb = min(W, xa + (int)j.chunk_cols);
    const bool vec = (W & 15) == 0 && (reinterpret_cast<uintptr_t>(j.out) & 15) == 0;
    for (int x0 = xa; x0 < xb; x0 += TW) {
      if ((reinterpret_cast<uintptr_t>(j.rgb) & 15) == 0)
        stage_gray_async<GR, GC, P, RW>(g_s, raw_s, j.rgb, W, H, y0 - 3, x0 - 3);
      else
        stage_gray<GR, GC, P>(g_s, j.rgb, W, H, y0 - 3, x0 - 3);
      __syncthreads();
      gauss_tile<QR, QC, GC, P, P, P>(q_s, g_s, v_s, W, H, y0 - 1, x0 - 1, y0 - 3, x0 - 3);
      __syncthreads();
      sobel_tile<P, TW>(q_s, j.out, whist, W, H, y0, x0, vec);
      __syncthreads();
    }
    finish_item(j, whist, &s_flag);
  }
}

template <int RB, int TW>
__global__ void __launch_bounds__(kThreads) img_fused_kernel(const __grid_constant__ ImgFusedArgs a) {
  img_fused_body<RB, TW>(a);
}

// Device-dispatch lane kernel: a fixed grid pulls the job's work items from the lane's ticket
// (every CTA count works for every image size); arguments of the job in flight in device memory.
__global__ void __launch_bounds__(kThreads) img_fused_lane_kernel(const ImgFusedArgs* __restrict__ pa) {
  img_fused_body<kRB, kTW>(*pa);
}

__global__ void __launch_bounds__(kThreads) gray_kernel(const GrayArgs a) {
  stamp_entry(a.stamp);
  const size_t groups = (a.px + 15) / 16;
  const bool vec = ((reinterpret_cast<uintptr_t>(a.rgb) | reinterpret_cast<uintptr_t>(a.gray)) & 15) == 0;
  for (size_t g = (size_t)blockIdx.x * kThreads + threadIdx.x; g < groups; g += (size_t)gridDim.x * kThreads) {
    const size_t p0 = g * 16;
    if (vec && p0 + 16 <= a.px) {
      uint4 w[3];
      const uint4* src = reinterpret_cast<const uint4*>(a.rgb + 3 * p0);
      w[0] = __ldg(src);
      w[1] = __ldg(src + 1);
      w[2] = __ldg(src + 2);
      const uint8_t* b = reinterpret_cast<const uint8_t*>(w);
      uint32_t o[4] = {0, 0, 0, 0};
#pragma unroll
      for (int k = 0; k < 16; ++k) o[k >> 2] |= gray_of(b[3 * k], b[3 * k + 1], b[3 * k + 2]) << (8 * (k & 3));
      *reinterpret_cast<uint4*>(a.gray + p0) = make_uint4(o[0], o[1], o[2], o[3]);
    } else {
      for (size_t p = p0; p < min(p0 + 16, a.px); ++p)
        a.gray[p] = (uint8_t)gray_of(a.rgb[3 * p], a.rgb[3 * p + 1], a.rgb[3 * p + 2]);
    }
  }
  stamp_exit(a.stamp);
}

// One CTA per 32 x 128 output tile of the Gaussian image.
__global__ void __launch_bounds__(kThreads) gauss_kernel(const GaussArgs a) {
  constexpr int GR = kRB + 4, GC = kTW + 4, P = kTW + 8;
  __shared__ __align__(16) uint8_t g_s[GR][P];
  __shared__ __align__(16) uint16_t v_s[kRB][P];
  __shared__ __align__(16) uint8_t q_s[kRB][P];
  const int W = (int)a.W, H = (int)a.H;
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kRB;
  stamp_entry(a.stamp);
  stage_u8<GR, GC, P>(g_s, a.g, W, H, y0 - 2, x0 - 2);
  __syncthreads();
  gauss_tile<kRB, kTW, GC, P, P, P>(q_s, g_s, v_s, W, H, y0, x0, y0 - 2, x0 - 2);
  __syncthreads();
  for (int i = threadIdx.x; i < kRB * kTW; i += kThreads) {
    const int r = i / kTW, c = i - r * kTW;
    if (y0 + r < H && x0 + c < W) a.q[(size_t)(y0 + r) * W + x0 + c] = q_s[r][c];
  }
  stamp_exit(a.stamp);
}

// Sobel + histogram over the Gaussian image: same work items, tiles and histogram protocol as
// the fused kernel (single job).
__global__ void __launch_bounds__(kThreads) sobel_hist_kernel(const SobelHistArgs sa) {
  const ImgFusedArgs& a = sa.a;
  const uint8_t* __restrict__ q = sa.q;
  stamp_entry(sa.stamp);
  constexpr int QR = kRB + 2, QC = kTW + 2, P = kTW + 8;
  __shared__ __align__(16) uint8_t q_s[QR][P];
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t s_item, s_flag;
  for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&whist[0][0])[i] = 0u;
  const ImgJobDev& j = a.one;
  const int W = (int)j.W, H = (int)j.H;
  const bool vec = (W & 15) == 0 && (reinterpret_cast<uintptr_t>(j.out) & 15) == 0;
  __syncthreads();
  for (uint32_t pass = 0;; ++pass) {
    uint32_t item;
    if (!next_item(a, pass, &s_item, &item)) {
      stamp_exit(sa.stamp);
      return;
    }
    const int band = (int)(item / j.chunks), chunk = (int)(item - (uint32_t)band * j.chunks);
    const int y0 = band * kRB;
    const int xa = chunk * (int)j.chunk_cols, xb = min(W, xa + (int)j.chunk_cols);
    for (int x0 = xa; x0 < xb; x0 += kTW) {
      stage_u8<QR, QC, P>(q_s, q, W, H, y0 - 1, x0 - 1);
      __syncthreads();
      sobel_tile<P>(q_s, j.out, whist, W, H, y0, x0, vec);
      __syncthreads();
    }
    finish_item(j, whist, &s_flag);
  }
}

constexpr int kTileRows[3] = {32, 16, 64};  // tile variants: 32x128, 16x256, 64x64

uint32_t items_of(uint32_t W, uint32_t H, uint32_t* chunks, int rows = kRB, uint32_t cols = kImgChunkCols) {
  *chunks = (W + cols - 1) / cols;
  return ((H + rows - 1) / rows) * *chunks;
}

const void* fused_func(int variant) {
  switch (variant) {
    case 1:
      return reinterpret_cast<const void*>(&img_fused_kernel<16, 256>);
    case 2:
      return reinterpret_cast<const void*>(&img_fused_kernel<64, 64>);
    default:
      return reinterpret_cast<const void*>(&img_fused_kernel<32, 128>);
  }
}

ImgJobDev job_dev(const JobPlanIn& in, const JobLayout& L) {
  ImgJobDev j{};
  const uint32_t W = in.dims[0], H = in.dims[1];
  const size_t px = (size_t)W * H, hist_off = (px + 15) & ~size_t(15);
  uint8_t* out = static_cast<uint8_t*>(in.d_out);
  j.rgb = static_cast<const uint8_t*>(in.d_in);
  j.out = out;
  j.pad = out + px;
  j.npad = (uint32_t)(hist_off - px);
  j.hist = reinterpret_cast<uint32_t*>(out + hist_off);
  j.trailer = reinterpret_cast<set_trailer*>(out + L.out_bytes - sizeof(set_trailer));
  j.acc = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(in.d_persist) + kImgHdrBytes);
  j.job_id = in.job_id;
  j.W = W;
  j.H = H;
  j.item0 = 0;
  j.chunk_cols = kTW;  // one launch per image: one tile per work item spreads the image over more SMs
  j.nitems = items_of(W, H, &j.chunks, kRB, j.chunk_cols);
  j.slot_gen = in.slot_gen;
  return j;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

}  // namespace

const void* img_lane_func() { return reinterpret_cast<const void*>(&img_fused_lane_kernel); }
uint32_t img_lane_grid() { return (uint32_t)sm_count() * 2; }

bool plan_img_lane(const JobPlanIn& in, unsigned char* args, uint32_t* args_size) {
  JobLayout L;
  if (!job_sizes(SET_JOB_IMG_SOBEL_HIST, in.dims, &L)) return false;
  ImgFusedArgs fa{};
  fa.table = nullptr;
  fa.hdr = static_cast<ImgHdr*>(in.d_persist);
  fa.one = job_dev(in, L);
  fa.njobs = 1;
  fa.total_items = fa.one.nitems;
  fa.direct = 0;  // items from the ticket: the lane's grid is fixed
  static_assert(sizeof(ImgFusedArgs) <= 192, "image arguments fit a lane descriptor");
  __builtin_memcpy(args, &fa, sizeof fa);
  *args_size = (uint32_t)sizeof fa;
  return true;
}

bool plan_img_sobel_hist(const JobPlanIn& in, const JobLayout& L, KernelLaunch* kl, int* nk) {
  const ImgJobDev j = job_dev(in, L);
  ImgFusedArgs fa{};
  fa.table = nullptr;
  fa.hdr = static_cast<ImgHdr*>(in.d_persist);
  fa.njobs = 1;
  fa.total_items = j.nitems;
  fa.direct = 1;  // one CTA per tile: the hardware schedules the waves, no ticket round trips
  fa.one = j;
  const uint32_t grid = j.nitems;
  if (in.img_fused) {
    KernelLaunch& k = kl[0];
    k.func = fused_func(0);
    k.grid = dim3(grid);
    k.block = dim3(kThreads);
    k.deps = 0;
    set_args(k, fa);
    *nk = 1;
    return true;
  }
  const uint32_t W = in.dims[0], H = in.dims[1];
  const size_t px = (size_t)W * H;
  uint8_t* gray = static_cast<uint8_t*>(in.d_scratch);
  uint8_t* gauss = gray + align256(px);
  GrayArgs ga{Stamp{}, j.rgb, gray, px};
  KernelLaunch& k0 = kl[0];
  k0.func = reinterpret_cast<const void*>(&gray_kernel);
  k0.grid = dim3((unsigned)std::min<size_t>((px + 16 * kThreads - 1) / (16 * kThreads), (size_t)sm_count() * 8));
  k0.block = dim3(kThreads);
  k0.deps = 0;
  set_args(k0, ga);
  GaussArgs qa{Stamp{}, gray, gauss, W, H};
  KernelLaunch& k1 = kl[1];
  k1.func = reinterpret_cast<const void*>(&gauss_kernel);
  k1.grid = dim3((W + kTW - 1) / kTW, (H + kRB - 1) / kRB);
  k1.block = dim3(kThreads);
  k1.deps = 1u << 0;
  set_args(k1, qa);
  SobelHistArgs sa{Stamp{}, fa, gauss};
  KernelLaunch& k2 = kl[2];
  k2.func = reinterpret_cast<const void*>(&sobel_hist_kernel);
  k2.grid = dim3(grid);
  k2.block = dim3(kThreads);
  k2.deps = 1u << 1;
  set_args(k2, sa);
  *nk = 3;
  return true;
}

// Batched form: one persistent fused launch over nb image jobs.  The table region of the batch
// block holds {header (ticket 0), nb job descriptors, nb zeroed histogram accumulators}; it is
// written here into the host staging buffer and copied in by the batch graph's first node.
bool plan_img_batch(const BatchItem* items, int nb, const BatchLayout& L, uint8_t* d_block, uint8_t* h_table,
                    uint32_t slot_gen, int ctas_per_sm, int variant, KernelLaunch* kl, int* nk) {
  if (variant < 0 || variant > 2) variant = 0;
  std::memset(h_table, 0, L.table_bytes);
  const size_t desc_off = kImgHdrBytes, acc_off = kImgHdrBytes + (size_t)nb * kImgJobDescBytes;
  uint32_t item = 0;
  for (int j = 0; j < nb; ++j) {
    const uint32_t W = items[j].dims[0], H = items[j].dims[1];
    const size_t px = (size_t)W * H, hist_off = (px + 15) & ~size_t(15);
    uint8_t* out = d_block + L.out_off[j];
    ImgJobDev jd{};
    jd.rgb = d_block + L.in_off[j];
    jd.out = out;
    jd.pad = out + px;
    jd.npad = (uint32_t)(hist_off - px);
    jd.hist = reinterpret_cast<uint32_t*>(out + hist_off);
    jd.trailer = reinterpret_cast<set_trailer*>(out + L.out_bytes[j] - sizeof(set_trailer));
    jd.acc = reinterpret_cast<uint32_t*>(d_block + acc_off + (size_t)j * kImgJobStateBytes);
    jd.job_id = items[j].job_id;
    jd.W = W;
    jd.H = H;
    jd.item0 = item;
    jd.chunk_cols = kImgChunkCols;  // many jobs per launch: wider items, fewer histogram flushes
    jd.nitems = items_of(W, H, &jd.chunks, kTileRows[variant], jd.chunk_cols);
    jd.slot_gen = slot_gen;
    item += jd.nitems;
    std::memcpy(h_table + desc_off + (size_t)j * sizeof(ImgJobDev), &jd, sizeof jd);
  }
  ImgFusedArgs fa{};
  fa.table = reinterpret_cast<const ImgJobDev*>(d_block + desc_off);
  fa.hdr = reinterpret_cast<ImgHdr*>(d_block);
  fa.njobs = (uint32_t)nb;
  fa.total_items = item;
  KernelLaunch& k = kl[0];
  k.func = fused_func(variant);
  k.grid = dim3(std::min<uint32_t>(item, (uint32_t)(sm_count() * std::max(1, ctas_per_sm))));
  k.block = dim3(kThreads);
  k.smem = 0;
  k.deps = 0;
  set_args(k, fa);
  *nk = 1;
  return true;
}

}  // namespace setk
