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

constexpr int kMlpD = 1024;
constexpr int kMlpF = 4096;
constexpr int kMlpMaxM = 256;

}  // namespace setk
