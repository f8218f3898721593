// dd_backend.h -- what the device-dispatch lanes (set_dd_*) need from the device side.
//
// DevDispatch (dev_dispatch.cpp) runs the host protocol: lane choice, ring entries and their
// reuse, completion handling, relaunch of lanes whose loop has ended, shutdown.  A backend owns
// the memory the protocol shares with the device and the lanes' loops: the CUDA backend
// (dd_cuda.cpp) builds one graph per lane (WHILE { fetch -> SWITCH { blur | scan | image } }); the
// test library's simulated backend runs each launched loop on a host thread.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../kernels/dev_dispatch.h"
#include "set.h"

namespace setrt {

// One lane's structures shared with the device (host views).
struct DdLaneMem {
  setk::DdEntry* ring = nullptr;  // `depth` descriptors, written by the host
  setk::DdCtl* ctl = nullptr;     // done counter and loop exits (device), stop flag (host)
  uint32_t* cmpl = nullptr;       // completion word per ring entry (device)
  void* scan_scratch = nullptr;   // the scan kernel's look-back areas, one per job of a batch (device
                                  // memory); jobs are planned on the first, the kernel adds j * stride
  void* img_state = nullptr;      // the image kernel's ticket and histogram accumulator (device memory)
};

// Device allocations a backend has already accepted during one submit call ([lo, hi) ranges), so
// that jobs carved out of the same allocations are not checked with the driver again.  Lives no
// longer than the call: memory freed and mapped again later is checked afresh.
struct DdRangeCache {
  static constexpr int kN = 4;
  uintptr_t lo[kN] = {}, hi[kN] = {};
  int n = 0, next = 0;
  bool has(uintptr_t p, size_t bytes) const {
    for (int i = 0; i < n; ++i)
      if (p >= lo[i] && p <= hi[i] && bytes <= hi[i] - p) return true;
    return false;
  }
  void add(uintptr_t a, uintptr_t b) {
    lo[next] = a;
    hi[next] = b;
    next = (next + 1) % kN;
    if (n < kN) ++n;
  }
};

class DdBackend {
 public:
  virtual ~DdBackend() = default;
  // Allocates and zeroes every lane's structures, builds the lanes' loops (not launched).
  virtual set_status init(const set_dd_config& cfg, uint32_t depth, std::vector<DdLaneMem>* lanes,
                          std::string* err) = 0;
  // The job's kernel argument struct (<= kDdArgBytes) over the lane's kernel state.
  virtual bool plan(const set_job_desc& d, uint64_t job_id, uint32_t lane, unsigned char* args,
                    uint32_t* args_size) = 0;
  // True if the lanes' kernels may use [p, p + bytes) as a job buffer in place.  cache (may be
  // null): allocations accepted earlier in the same submit call.
  virtual bool buffer_ok(const void* p, size_t bytes, DdRangeCache* cache) const = 0;
  // Launches the lane's loop, ordered after its previous launch.
  virtual set_status launch(uint32_t lane, std::string* err) = 0;
  // 1: every launch of the lane has completed; 0: one is still running; -1: the lane failed (err).
  virtual int ended(uint32_t lane, std::string* err) = 0;
  // Makes the backend's device current for the calling thread.
  virtual void bind_thread() = 0;
  // Frees everything (leak: keep memory a running loop may still use).
  virtual void release(bool leak) = 0;
};

std::unique_ptr<DdBackend> make_dd_backend();

}  // namespace setrt
