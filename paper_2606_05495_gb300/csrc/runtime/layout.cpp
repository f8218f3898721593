// layout.cpp -- job payload sizes (the layouts documented in set.h) and slot placement.
#include "layout.h"

#include "../kernels/params.h"
#include "set.h"

namespace setk {

namespace {
size_t scan_tiles(size_t n) { return (n + kScanTile - 1) / kScanTile; }
}  // namespace

bool job_sizes(uint32_t type, const uint32_t d[4], JobLayout* L) {
  *L = JobLayout{};
  switch (type) {
    case SET_JOB_BLUR_HIST: {
      if (d[0] < 1 || d[0] > (uint32_t)kBlurMaxW || d[1] < 1 || d[1] > (uint32_t)kBlurMaxH) return false;
      const size_t img = (size_t)d[0] * d[1];
      L->in_bytes = img;
      L->out_bytes = ((img + 15) & ~size_t(15)) + 256 * sizeof(uint32_t) + sizeof(set_trailer);
      return true;
    }
    case SET_JOB_SAXPY_SCAN_MAX: {
      const size_t n = d[0];
      if (n < 1 || n > kScanMaxN) return false;
      L->in_bytes = 8 * n;
      L->out_bytes = 8 * n + 16 + sizeof(set_trailer);
      L->persist_bytes = kScanHdrBytes + kScanBytesPerTile * scan_tiles(n);
      return true;
    }
    case SET_JOB_IMG_SOBEL_HIST: {
      if (d[0] < 1 || d[0] > (uint32_t)kImgMaxSide || d[1] < 1 || d[1] > (uint32_t)kImgMaxSide) return false;
      const size_t px = (size_t)d[0] * d[1];
      L->in_bytes = 3 * px;
      L->out_bytes = ((px + 15) & ~size_t(15)) + 256 * sizeof(uint32_t) + sizeof(set_trailer);
      L->scratch_bytes = 2 * align256(px);  // gray and Gaussian images of the per-stage chain
      L->persist_bytes = kImgHdrBytes + kImgJobStateBytes;
      return true;
    }
    case SET_JOB_MLP_LN: {
      const size_t m = d[0];
      if (m < 1 || m > (size_t)kMlpMaxM) return false;
      L->in_bytes = m * kMlpD * 2;
      L->out_bytes = m * kMlpD * 4 + sizeof(set_trailer);
      // h (bf16, m x F) and LayerNorm(x) (f32, m x D), rows padded to the 128-row GEMM tile
      const size_t mp = (m + 127) & ~size_t(127);
      L->scratch_bytes = align256(mp * kMlpF * 2) + align256(mp * kMlpD * 4);
      return true;
    }
    default:
      return false;
  }
}

size_t slot_control_bytes(size_t slot_bytes) {
  // a scan job of n elements needs 8n payload bytes, so n <= slot_bytes / 8
  return kCtlImgBytes + align256(kScanHdrBytes + kScanBytesPerTile * scan_tiles(slot_bytes / 8 + 1));
}

size_t control_offset(uint32_t type) { return type == SET_JOB_SAXPY_SCAN_MAX ? kCtlScanOff : kCtlImgOff; }

void place_job(JobLayout* L, size_t ctl) {
  L->in_off = ctl;
  L->out_off = L->in_off + align256(L->in_bytes);
  L->scratch_off = L->out_off + align256(L->out_bytes);
  L->end = L->scratch_off + align256(L->scratch_bytes);
}

}  // namespace setk
