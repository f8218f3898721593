// params.h -- size limits and tile constants shared by the host layout code and the kernels.
#pragma once

#include <cstdint>

namespace setk {

constexpr int kBlurMaxW = 2048;
constexpr int kBlurMaxH = 65535;

constexpr uint32_t kScanTile = 4096;       // elements per scan tile (256 threads x 16)
constexpr uint32_t kScanMaxN = 1u << 26;
constexpr uint32_t kScanHdrBytes = 64;     // {ticket, done, epoch, err} + padding
constexpr uint32_t kScanBytesPerTile = 12; // 64-bit status word + float tile max

constexpr int kImgMaxSide = 4096;
constexpr uint32_t kImgHdrBytes = 64;        // {ticket} + padding
constexpr uint32_t kImgJobStateBytes = 1152; // hist accumulator [256] u32 + items-done counter, padded
constexpr int kImgBandRows = 32;             // output rows of one work item
constexpr int kImgChunkCols = 512;           // output columns of one work item
constexpr int kImgMaxBatch = 4096;           // jobs of one batched launch

// Slot control block: [image state (fixed) | scan state (grows with the slot)].
constexpr uint32_t kCtlImgOff = 0;
constexpr uint32_t kCtlImgBytes = 2048;
constexpr uint32_t kCtlScanOff = kCtlImgBytes;

constexpr int kMlpD = 1024;
constexpr int kMlpF = 4096;
constexpr int kMlpMaxM = 256;

}  // namespace setk
