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
      L->persist_bytes = kMlpCtlBytes;
      return true;
    }
    case SET_JOB_HOTSPOT: {
      if (d[0] < 1 || d[0] > (uint32_t)kHotMaxSide || d[1] < 1 || d[1] > (uint32_t)kHotMaxSide || d[2] < 1 ||
          d[2] > (uint32_t)kHotMaxSteps)
        return false;
      const size_t cells = (size_t)d[0] * d[1];
      L->in_bytes = 8 * cells;
      L->out_bytes = ((4 * cells + 15) & ~size_t(15)) + sizeof(set_trailer);
      L->scratch_bytes = 4 * cells;  // the other buffer of the launches' ping-pong
      L->persist_bytes = kHotCtlBytes;
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

size_t control_offset(uint32_t type) {
  switch (type) {
    case SET_JOB_SAXPY_SCAN_MAX:
      return kCtlScanOff;
    case SET_JOB_MLP_LN:
      return kCtlMlpOff;
    case SET_JOB_HOTSPOT:
      return kCtlHotOff;
    default:
      return kCtlImgOff;
  }
}

void place_job_guarded(JobLayout* L, size_t ctl) {
  L->in_off = align256(ctl) + kGuardBytes;
  L->out_off = align256(L->in_off + L->in_bytes + kGuardBytes);
  L->scratch_off = align256(L->out_off + L->out_bytes + kGuardBytes);
  L->end = align256(L->scratch_off + L->scratch_bytes + kGuardBytes);
}

void guard_offsets(const JobLayout& L, size_t off[4]) {
  off[0] = L.in_off - kGuardBytes;
  off[1] = L.in_off + L.in_bytes;
  off[2] = L.out_off + L.out_bytes;
  off[3] = L.scratch_off + L.scratch_bytes;
}

void place_job(JobLayout* L, size_t ctl) {
  L->in_off = ctl;
  L->out_off = L->in_off + align256(L->in_bytes);
  L->scratch_off = L->out_off + align256(L->out_bytes);
  L->end = L->scratch_off + align256(L->scratch_bytes);
}

bool batchable(uint32_t type) { return type == SET_JOB_IMG_SOBEL_HIST || type == SET_JOB_MLP_LN; }

// Image batch: table = {header, job descriptors, per-job histogram accumulators}, then each job's
// input and output region.  MLP batch: table = {control word, per-job trailer records}, then the
// packed buffers x, h, LayerNorm, out over sum(m_j + 1) rows: job j owns rows [R_j, R_j + m_j)
// and the spare row R_j + m_j whose first 16 bytes receive its trailer, so that one D2H copy of
// m_j * 4096 + 16 bytes returns the job's rows and trailer.
bool batch_layout(uint32_t type, const BatchItem* items, int nb, BatchLayout* L) {
  if (nb < 1 || nb > kMaxBatch || !batchable(type)) return false;
  L->nb = nb;
  size_t off = 0;
  if (type == SET_JOB_IMG_SOBEL_HIST) {
    L->table_bytes = align256(kImgHdrBytes + (size_t)nb * (kImgJobDescBytes + kImgJobStateBytes));
    off = L->table_bytes;
    for (int j = 0; j < nb; ++j) {
      JobLayout J;
      if (!job_sizes(type, items[j].dims, &J)) return false;
      L->in_off[j] = off;
      L->in_bytes[j] = J.in_bytes;
      off += align256(J.in_bytes);
      L->out_off[j] = off;
      L->out_bytes[j] = J.out_bytes;
      off += align256(J.out_bytes);
    }
    L->block_bytes = off;
    return true;
  }
  L->table_bytes = align256(kMlpCtlBytes + (size_t)nb * kMlpTrailerRecBytes);
  size_t rows = 0;
  size_t R[kMaxBatch];
  for (int j = 0; j < nb; ++j) {
    const uint32_t m = items[j].dims[0];
    if (m < 1 || m > (uint32_t)kMlpMaxM) return false;
    R[j] = rows;
    rows += m + 1;
  }
  L->rows = rows;
  const size_t x_off = L->table_bytes;
  const size_t h_off = x_off + align256(rows * kMlpD * 2);
  const size_t ln_off = h_off + align256(rows * kMlpF * 2);
  const size_t o_off = ln_off + align256(rows * kMlpD * 4);
  L->block_bytes = o_off + align256(rows * kMlpD * 4);
  for (int j = 0; j < nb; ++j) {
    const uint32_t m = items[j].dims[0];
    L->in_off[j] = x_off + R[j] * kMlpD * 2;
    L->in_bytes[j] = (size_t)m * kMlpD * 2;
    L->out_off[j] = o_off + R[j] * kMlpD * 4;
    L->out_bytes[j] = (size_t)m * kMlpD * 4 + sizeof(set_trailer);
  }
  return true;
}

}  // namespace setk
