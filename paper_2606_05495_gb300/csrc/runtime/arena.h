// arena.h -- buddy allocator over one device memory range (host-side bookkeeping only).
//
// Serving admits jobs by free device memory: each job's [in | out | scratch] is carved from the
// arena at dispatch and returned by its completion callback.  Blocks are powers of two between
// min_block and the largest power of two that fits; a freed block merges with its free buddy.
// Thread-safe (one mutex); O(log(size / min_block)) per call.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <set>
#include <vector>

namespace setrt {

class BuddyArena {
 public:
  BuddyArena() = default;
  void init(uint8_t* base, size_t bytes, size_t min_block) {
    base_ = base;
    min_ = min_block;
    orders_ = 0;
    while ((min_ << (orders_ + 1)) <= bytes) ++orders_;
    free_.assign(orders_ + 1, {});
    size_ = min_ << orders_;
    free_[orders_].insert(0);
    used_ = peak_ = 0;
  }
  size_t capacity() const { return size_; }
  size_t max_block() const { return size_; }

  // Returns the device pointer of a block of at least `bytes`, or nullptr if none is free.
  uint8_t* alloc(size_t bytes, size_t* block_bytes) {
    const int o = order_of(bytes);
    if (o < 0) return nullptr;
    std::lock_guard<std::mutex> g(mu_);
    int k = o;
    while (k <= orders_ && free_[k].empty()) ++k;
    if (k > orders_) return nullptr;
    size_t off = *free_[k].begin();
    free_[k].erase(free_[k].begin());
    while (k > o) {  // split, keep the lower half
      --k;
      free_[k].insert(off + (min_ << k));
    }
    *block_bytes = min_ << o;
    used_ += *block_bytes;
    if (used_ > peak_) peak_ = used_;
    return base_ + off;
  }

  void free(uint8_t* p, size_t block_bytes) {
    int o = order_of(block_bytes);
    size_t off = (size_t)(p - base_);
    std::lock_guard<std::mutex> g(mu_);
    used_ -= block_bytes;
    while (o < orders_) {
      const size_t buddy = off ^ (min_ << o);
      auto it = free_[o].find(buddy);
      if (it == free_[o].end()) break;
      free_[o].erase(it);
      off = off < buddy ? off : buddy;
      ++o;
    }
    free_[o].insert(off);
  }

  size_t used() {
    std::lock_guard<std::mutex> g(mu_);
    return used_;
  }
  size_t peak() {
    std::lock_guard<std::mutex> g(mu_);
    return peak_;
  }

 private:
  int order_of(size_t bytes) const {
    int o = 0;
    while ((min_ << o) < bytes) {
      if (++o > orders_) return -1;
    }
    return o;
  }
  uint8_t* base_ = nullptr;
  size_t min_ = 0, size_ = 0, used_ = 0, peak_ = 0;
  int orders_ = 0;
  std::vector<std::set<size_t>> free_;
  std::mutex mu_;
};

}  // namespace setrt
