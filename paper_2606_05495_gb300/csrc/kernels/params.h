// params.h -- size limits and tile constants shared by the host layout code and the kernels.
#pragma once

#include <cstdint>

namespace setk {

constexpr int kBlurMaxW = 2048;
constexpr int kBlurMaxH = 65535;

constexpr uint32_t kScanTile = 4096;       // elements per scan tile (256 threads x 16)
constexpr uint32_t kScanMaxN = 1u << 26;
constexpr uint32_t kScanHdrBytes = 64;     // {ticket, done, epoch, err} + padding
constexpr uint32_t kScanBytesPerTile = 16; // 64-bit status word + 64-bit tile max word

constexpr int kImgMaxSide = 4096;
constexpr uint32_t kImgHdrBytes = 64;        // {ticket} + padding
constexpr uint32_t kImgJobStateBytes = 1152; // hist accumulator [256] u32 + items-done counter, padded
constexpr uint32_t kImgJobDescBytes = 128;   // device job descriptor of the fused kernel
constexpr int kImgBandRows = 32;             // output rows of one work item
constexpr int kImgChunkCols = 512;           // output columns of one work item
constexpr int kImgMaxBatch = 4096;           // jobs of one batched launch

// Slot control block: [image state (fixed) | scan state (grows with the slot)].
constexpr uint32_t kCtlImgOff = 0;
constexpr uint32_t kCtlMlpOff = 1536;        // MLP job state {err, done} inside the fixed region
constexpr uint32_t kCtlStampOff = 1664;      // stamps mode: {arrive, depart} per kernel of the job
constexpr uint32_t kCtlImgBytes = 2048;
constexpr uint32_t kCtlScanOff = kCtlImgBytes;

constexpr uint32_t kCtlHotOff = 1600;        // hotspot job state {CTAs done} inside the fixed region
constexpr uint32_t kHotCtlBytes = 64;
static_assert(kCtlHotOff >= kCtlMlpOff + 64 && kCtlHotOff + kHotCtlBytes <= kCtlStampOff, "control regions overlap");
constexpr int kHotMaxSide = 8192;
constexpr int kHotLaunches = 8;              // kernel nodes of every hotspot job
constexpr int kHotStepsPerLaunch = 8;        // time steps one launch advances (its staged halo)
constexpr int kHotMaxSteps = kHotLaunches * kHotStepsPerLaunch;

constexpr int kMlpD = 1024;
constexpr int kMlpF = 4096;
constexpr int kMlpMaxM = 256;
constexpr uint32_t kMlpCtlBytes = 64;
constexpr uint32_t kMlpTrailerRecBytes = 32; // batch: {trailer pointer, job id, slot generation}

}  // namespace setk
