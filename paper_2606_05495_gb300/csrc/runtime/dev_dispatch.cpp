// dev_dispatch.cpp -- device-dispatch lanes (set_dd_* in set.h): the host side.
//
// Per lane: a non-blocking stream, one graph WHILE { fetch -> SWITCH { blur | scan } } built and
// uploaded once, a ring of descriptors and a completion word per entry in page-locked host memory,
// a control line (done counter and loop exits written by the GPU, stop flag written by the host)
// and the lane's device block (fetched arguments, scan look-back state).
//
// Submit plans the job's single stage kernel with the same planners as the executor, writes the
// argument struct into the lane's next ring entry and publishes it with a release store of the
// entry's sequence word.  Ring entries are reused only after the completion thread has handled
// the job that used them.  The completion thread reads each lane's done counter, completes the
// jobs behind it (status from the completion word, latency) and relaunches lanes whose loop has
// ended while descriptors are waiting; submitters relaunch too, under the lane's mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../kernels/dev_dispatch.h"
#include "../kernels/stages.h"
#include "executor.h"
#include "layout.h"
#include "set.h"
#include "sync.h"
#include "thread_error.h"

namespace setrt {
namespace {

#define DD_CK(call)                                                               \
  do {                                                                            \
    const cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                      \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return SET_ECUDA;                                                           \
    }                                                                             \
  } while (0)

constexpr uint64_t kPollSleepNs = 5000;

struct DdInfo {
  uint64_t id = 0;
  volatile int32_t* status = nullptr;
  uint64_t t_arrival = 0;
};

struct DdLane {
  std::mutex mu;  // writers of this lane's ring and graph launches
  cudaStream_t stream = nullptr;
  cudaEvent_t ended = nullptr;  // recorded behind each launch of the lane's graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  setk::DdEntry* ring = nullptr;  // host view
  setk::DdCtl* ctl = nullptr;
  uint32_t* cmpl = nullptr;
  setk::DdLaneDev* dev = nullptr;  // device memory
  void* scan_scratch = nullptr;
  std::unique_ptr<DdInfo[]> info;
  std::atomic<uint64_t> seq{0};       // descriptors published
  std::atomic<uint64_t> reaped{0};    // completions handled
  std::atomic<uint32_t> launches{0};  // graph launches (changed under mu)
};

inline uint32_t load_acq32(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
inline uint64_t load_acq64(const uint64_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// Device memory of `device` (the lanes' kernels read and write the job's buffers in place).
bool device_memory(const void* p, int device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

class DevDispatch {
 public:
  ~DevDispatch() { release(); }
  set_status init(const set_dd_config& cfg, std::string* err);
  set_status submit(const set_job_desc* d, uint64_t* id_out);
  set_status wait_all(int64_t timeout_us);
  set_status stats(set_stats_t* out, uint64_t* launches);
  set_status reset_stats();
  set_status shutdown();
  const char* last_error() {
    std::lock_guard<std::mutex> g(err_mu_);
    err_copy_ = err_;
    return err_copy_.c_str();
  }
  set_status fail(set_status st, const std::string& why) {
    {
      std::lock_guard<std::mutex> g(err_mu_);
      err_ = why;
    }
    if (st == SET_ECUDA) sticky_.store(SET_ECUDA);
    return st;
  }

 private:
  set_status build_lane(uint32_t i, std::string* err);
  set_status launch_locked(DdLane& l);
  bool maybe_relaunch_locked(DdLane& l);
  uint32_t pick_lane();
  set_status validate(const set_job_desc& d, setk::JobLayout* L, std::string* why) const;
  void poll_main();
  void reap(DdLane& l, uint64_t upto);
  void release();

  set_dd_config cfg_{};
  uint32_t depth_ = 0, mask_ = 0;
  std::vector<std::unique_ptr<DdLane>> lanes_;
  void* host_block_ = nullptr;
  void* dev_block_ = nullptr;
  bool leak_ = false;  // a lane did not end: keep its memory
  std::atomic<uint64_t> next_id_{1};
  std::atomic<uint64_t> submitted_{0}, completed_{0}, failed_{0}, canary_{0}, ring_waits_{0};
  std::atomic<uint64_t> submit_ns_{0}, t_first_{0}, t_last_{0}, t_reset_{0};
  LogHist lat_;
  Signal done_sig_, work_sig_;
  std::thread poller_;
  std::atomic<bool> stop_{false}, poll_quit_{false};
  std::atomic<int> sticky_{SET_OK};
  std::atomic<uint32_t> rr_{0};
  std::mutex err_mu_;
  std::string err_, err_copy_;
};

set_status DevDispatch::init(const set_dd_config& cfg, std::string* err) {
  cfg_ = cfg;
  if (cfg.num_lanes < 1 || cfg.num_lanes > 256 || cfg.ring_depth < 1 || cfg.ring_depth > (1 << 16) ||
      cfg.scan_max_n < 1 || cfg.scan_max_n > setk::kScanMaxN || cfg.blur_max_w < 1 ||
      cfg.blur_max_w > (uint32_t)setk::kBlurMaxW || cfg.idle_us < 1 || cfg.spin_us < 0) {
    *err = "set_dd_config out of range (lanes 1..256, ring 1..65536, scan_max_n 1..2^26, blur_max_w 1..2048, idle_us >= 1)";
    return SET_EINVAL;
  }
  depth_ = (uint32_t)next_pow2((size_t)cfg.ring_depth);
  mask_ = depth_ - 1;
  DD_CK(cudaSetDevice(cfg.device));
  DD_CK(cudaFree(nullptr));
  DD_CK(setk::kernels_init());

  const uint32_t nl = (uint32_t)cfg.num_lanes;
  const size_t ring_bytes = (size_t)depth_ * sizeof(setk::DdEntry);
  const size_t cmpl_bytes = setk::align256((size_t)depth_ * sizeof(uint32_t));
  const size_t host_lane = ring_bytes + sizeof(setk::DdCtl) + cmpl_bytes;
  const size_t host_total = host_lane * nl;
  if (cudaHostAlloc(&host_block_, host_total, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    host_block_ = nullptr;
    *err = "cudaHostAlloc of the descriptor rings failed (" + std::to_string(host_total) + " bytes)";
    return SET_ENOMEM;
  }
  std::memset(host_block_, 0, host_total);
  void* host_dev = nullptr;
  DD_CK(cudaHostGetDevicePointer(&host_dev, host_block_, 0));

  setk::JobLayout SL;
  const uint32_t sd[4] = {cfg.scan_max_n, 0, 0, 0};
  if (!setk::job_sizes(SET_JOB_SAXPY_SCAN_MAX, sd, &SL)) {
    *err = "scan_max_n rejected by the scan layout";
    return SET_EINVAL;
  }
  const size_t lane_dev = setk::align256(sizeof(setk::DdLaneDev));
  const size_t scratch = setk::align256(SL.persist_bytes);
  const size_t dev_total = (lane_dev + scratch) * nl;
  if (cudaMalloc(&dev_block_, dev_total) != cudaSuccess) {
    cudaGetLastError();
    dev_block_ = nullptr;
    *err = "cudaMalloc of the lane state failed (" + std::to_string(dev_total) + " bytes)";
    return SET_ENOMEM;
  }
  DD_CK(cudaMemset(dev_block_, 0, dev_total));

  for (uint32_t i = 0; i < nl; ++i) {
    auto l = std::make_unique<DdLane>();
    uint8_t* hb = static_cast<uint8_t*>(host_block_) + host_lane * i;
    l->ring = reinterpret_cast<setk::DdEntry*>(hb);
    l->ctl = reinterpret_cast<setk::DdCtl*>(hb + ring_bytes);
    l->cmpl = reinterpret_cast<uint32_t*>(hb + ring_bytes + sizeof(setk::DdCtl));
    uint8_t* db = static_cast<uint8_t*>(dev_block_);
    l->dev = reinterpret_cast<setk::DdLaneDev*>(db + lane_dev * i);
    l->scan_scratch = db + lane_dev * nl + scratch * i;
    l->info.reset(new DdInfo[depth_]);
    lanes_.push_back(std::move(l));
  }
  for (uint32_t i = 0; i < nl; ++i) {
    const set_status st = build_lane(i, err);
    if (st != SET_OK) return st;
  }
  DD_CK(cudaDeviceSynchronize());  // uploads and memsets done before the first descriptor
  t_reset_.store(now_ns());
  poller_ = std::thread([this] { poll_main(); });
  return SET_OK;
}

// WHILE (loop, 1 at each launch) { fetch -> SWITCH (kind) { [0] blur, [1] scan } }
set_status DevDispatch::build_lane(uint32_t i, std::string* err) {
  DdLane& l = *lanes_[i];
  DD_CK(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
  DD_CK(cudaEventCreateWithFlags(&l.ended, cudaEventDisableTiming));
  DD_CK(cudaGraphCreate(&l.graph, 0));
  cudaGraphConditionalHandle hloop = 0, hkind = 0;
  DD_CK(cudaGraphConditionalHandleCreate(&hloop, l.graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn = nullptr;
  DD_CK(cudaGraphAddNode(&wn, l.graph, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  // the fetch kernel sets the selector before the SWITCH node reads it in every iteration
  DD_CK(cudaGraphConditionalHandleCreate(&hkind, body, setk::kDdKindNone, 0));

  // device-usable addresses of this lane's host-side structures
  void* ring_d = nullptr;
  void* ctl_d = nullptr;
  void* cmpl_d = nullptr;
  DD_CK(cudaHostGetDevicePointer(&ring_d, l.ring, 0));
  DD_CK(cudaHostGetDevicePointer(&ctl_d, l.ctl, 0));
  DD_CK(cudaHostGetDevicePointer(&cmpl_d, l.cmpl, 0));
  setk::DdFetchArgs fa{};
  fa.lane = l.dev;
  fa.ring = static_cast<const setk::DdEntry*>(ring_d);
  fa.ctl = static_cast<setk::DdCtl*>(ctl_d);
  fa.cmpl = static_cast<uint32_t*>(cmpl_d);
  fa.depth = depth_;
  fa.idle_ns = (uint64_t)cfg_.idle_us * 1000ull;
  fa.loop = hloop;
  fa.kind = hkind;
  void* fargs[1] = {&fa};
  cudaKernelNodeParams fp{};
  fp.func = const_cast<void*>(setk::dd_fetch_func());
  fp.gridDim = dim3(1);
  fp.blockDim = dim3(32);
  fp.kernelParams = fargs;
  cudaGraphNode_t fn = nullptr;
  DD_CK(cudaGraphAddKernelNode(&fn, body, nullptr, 0, &fp));

  cudaGraphNodeParams sp{};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hkind;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = setk::kDdKinds;
  cudaGraphNode_t sn = nullptr;
  DD_CK(cudaGraphAddNode(&sn, body, &fn, nullptr, 1, &sp));

  const void* blur_args = l.dev->args[setk::kDdKindBlur];
  const void* scan_args = l.dev->args[setk::kDdKindScan];
  void* bargs[1] = {&blur_args};
  void* sargs[1] = {&scan_args};
  cudaKernelNodeParams bp{};
  bp.func = const_cast<void*>(setk::blur_lane_func());
  bp.gridDim = dim3(8);
  bp.blockDim = dim3(256);
  bp.sharedMemBytes = setk::blur_lane_smem(cfg_.blur_max_w);
  bp.kernelParams = bargs;
  cudaGraphNode_t bn = nullptr;
  DD_CK(cudaGraphAddKernelNode(&bn, sp.conditional.phGraph_out[setk::kDdKindBlur], nullptr, 0, &bp));
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(setk::scan_lane_func());
  kp.gridDim = dim3(setk::scan_lane_grid(cfg_.scan_max_n));
  kp.blockDim = dim3(256);
  kp.kernelParams = sargs;
  cudaGraphNode_t kn = nullptr;
  DD_CK(cudaGraphAddKernelNode(&kn, sp.conditional.phGraph_out[setk::kDdKindScan], nullptr, 0, &kp));

  DD_CK(cudaGraphInstantiate(&l.exec, l.graph, 0));
  DD_CK(cudaGraphUpload(l.exec, l.stream));
  return SET_OK;
}

set_status DevDispatch::launch_locked(DdLane& l) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != cfg_.device) cudaSetDevice(cfg_.device);
  cudaError_t e = cudaGraphLaunch(l.exec, l.stream);
  if (e == cudaSuccess) e = cudaEventRecord(l.ended, l.stream);
  if (prev >= 0 && prev != cfg_.device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SET_ECUDA, std::string("lane graph launch: ") + cudaGetErrorString(e));
  }
  l.launches.store(l.launches.load(std::memory_order_relaxed) + 1, std::memory_order_release);
  return SET_OK;
}

// A lane needs a launch when descriptors wait and every loop launched so far has ended: its
// fetch counted the exit, and the graph has completed on the stream (the event behind the last
// launch), so one launch of the lane's graph never waits behind another.
bool DevDispatch::maybe_relaunch_locked(DdLane& l) {
  if (l.seq.load(std::memory_order_acquire) <= load_acq64(&l.ctl->done)) return false;
  if (load_acq32(&l.ctl->exits) != l.launches.load(std::memory_order_acquire)) return false;
  const cudaError_t q = cudaEventQuery(l.ended);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) {
    cudaGetLastError();
    fail(SET_ECUDA, std::string("lane graph: ") + cudaGetErrorString(q));
    return false;
  }
  return launch_locked(l) == SET_OK;
}

// Shortest lane (fewest descriptors not yet handled), scanning from a rotating start so that
// ties spread; the paper's "shortest queue" policy for the submitter.
uint32_t DevDispatch::pick_lane() {
  const uint32_t nl = (uint32_t)lanes_.size();
  const uint32_t start = rr_.fetch_add(1, std::memory_order_relaxed) % nl;
  uint32_t best = start;
  uint64_t best_q = ~0ull;
  for (uint32_t k = 0; k < nl; ++k) {
    const uint32_t i = (start + k) % nl;
    const DdLane& l = *lanes_[i];
    const uint64_t q = l.seq.load(std::memory_order_relaxed) - l.reaped.load(std::memory_order_relaxed);
    if (q < best_q) {
      best_q = q;
      best = i;
      if (q == 0) break;
    }
  }
  return best;
}

set_status DevDispatch::validate(const set_job_desc& d, setk::JobLayout* L, std::string* why) const {
  if (d.type != SET_JOB_BLUR_HIST && d.type != SET_JOB_SAXPY_SCAN_MAX) {
    *why = "set_dd: only SET_JOB_BLUR_HIST and SET_JOB_SAXPY_SCAN_MAX jobs";
    return SET_EINVAL;
  }
  if (!setk::job_sizes(d.type, d.dims, L)) {
    *why = "dims out of range for the job type";
    return SET_EINVAL;
  }
  if (d.type == SET_JOB_SAXPY_SCAN_MAX && d.dims[0] > cfg_.scan_max_n) {
    *why = "scan n larger than set_dd_config.scan_max_n";
    return SET_EINVAL;
  }
  if (d.type == SET_JOB_BLUR_HIST && d.dims[0] > cfg_.blur_max_w) {
    *why = "blur width larger than set_dd_config.blur_max_w";
    return SET_EINVAL;
  }
  if (!d.in || !d.out || d.in_bytes != L->in_bytes || d.out_bytes != L->out_bytes) {
    *why = "null in/out, or in_bytes/out_bytes do not match the job type's layout";
    return SET_EINVAL;
  }
  if (!device_memory(d.in, cfg_.device) || !device_memory(d.out, cfg_.device)) {
    *why = "set_dd: in/out must be device memory of the object's GPU";
    return SET_EINVAL;
  }
  if (((reinterpret_cast<uintptr_t>(d.in) | reinterpret_cast<uintptr_t>(d.out)) & 15u) != 0) {
    *why = "set_dd: in/out must be 16-byte aligned (the kernels use 16-byte accesses in place)";
    return SET_EINVAL;
  }
  return SET_OK;
}

set_status DevDispatch::submit(const set_job_desc* d, uint64_t* id_out) {
  if (!d) return fail(SET_EINVAL, "null descriptor");
  if (stop_.load()) return SET_ESHUTDOWN;
  if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
  const uint64_t t0 = now_ns();
  setk::JobLayout L;
  std::string why;
  const set_status v = validate(*d, &L, &why);
  if (v != SET_OK) return fail(v, why);

  const uint32_t li = pick_lane();
  DdLane& l = *lanes_[li];
  const uint64_t id = next_id_.fetch_add(1);
  setk::JobPlanIn in;
  in.type = d->type;
  in.flags = d->flags;
  std::memcpy(in.dims, d->dims, sizeof in.dims);
  in.scalar = d->scalar;
  in.d_in = d->in;
  in.d_out = d->out;
  in.d_persist = l.scan_scratch;
  in.job_id = id;
  in.slot_gen = li;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  if (!setk::plan_job(in, kl, &nk) || nk != 1 || kl[0].args_size > setk::kDdArgBytes)
    return fail(SET_EINVAL, "set_dd: the job does not plan to one kernel with a small argument struct");

  std::unique_lock<std::mutex> g(l.mu);
  const uint64_t s = l.seq.load(std::memory_order_relaxed);
  if (s - l.reaped.load(std::memory_order_acquire) >= depth_) {
    if (d->flags & SET_F_NONBLOCK) return SET_EAGAIN;
    ring_waits_.fetch_add(1, std::memory_order_relaxed);
    const uint64_t limit = t0 + (uint64_t)cfg_.drain_timeout_ms * 1000000ull;
    while (s - l.reaped.load(std::memory_order_acquire) >= depth_) {
      maybe_relaunch_locked(l);
      if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
      if (now_ns() > limit) return fail(SET_ETIMEDOUT, "set_dd_submit: the lane's ring stayed full");
      std::this_thread::yield();
    }
  }
  const uint32_t k = (uint32_t)(s & mask_);
  DdInfo& inf = l.info[k];
  inf.id = id;
  inf.status = d->status;
  inf.t_arrival = d->t_arrival_ns ? d->t_arrival_ns : t0;
  setk::DdEntry& e = l.ring[k];
  e.kind = d->type == SET_JOB_BLUR_HIST ? setk::kDdKindBlur : setk::kDdKindScan;
  e.args_size = (uint32_t)kl[0].args_size;
  e.job_id = id;
  e.trailer = reinterpret_cast<set_trailer*>(static_cast<uint8_t*>(d->out) + L.out_bytes - sizeof(set_trailer));
  std::memcpy(e.args, kl[0].args, kl[0].args_size);
  __atomic_store_n(&e.seq, s + 1, __ATOMIC_RELEASE);
  l.seq.store(s + 1, std::memory_order_release);
  uint64_t z = 0;
  t_first_.compare_exchange_strong(z, t0);
  submitted_.fetch_add(1);
  maybe_relaunch_locked(l);
  g.unlock();
  work_sig_.notify(1);
  submit_ns_.fetch_add(now_ns() - t0, std::memory_order_relaxed);
  if (id_out) *id_out = id;
  return sticky_.load() == SET_OK ? SET_OK : (set_status)sticky_.load();
}

void DevDispatch::reap(DdLane& l, uint64_t upto) {
  uint64_t r = l.reaped.load(std::memory_order_relaxed);
  const uint64_t t = now_ns();
  for (; r < upto; ++r) {
    const uint32_t k = (uint32_t)(r & mask_);
    const DdInfo inf = l.info[k];
    const uint32_t w = __atomic_load_n(&l.cmpl[k], __ATOMIC_ACQUIRE);
    set_status st = SET_OK;
    if (w == 0u) {
      canary_.fetch_add(1, std::memory_order_relaxed);
      st = SET_EDEVICE;
    } else if (w & 0xFFFFu) {
      st = SET_EDEVICE;
    }
    if (st != SET_OK) failed_.fetch_add(1, std::memory_order_relaxed);
    lat_.record(t > inf.t_arrival ? t - inf.t_arrival : 0);
    if (inf.status) *inf.status = st;
    completed_.fetch_add(1);
  }
  t_last_.store(t);
  l.reaped.store(upto, std::memory_order_release);
}

void DevDispatch::poll_main() {
  cudaSetDevice(cfg_.device);
  uint64_t last_progress = now_ns(), last_check = last_progress;
  for (;;) {
    const uint32_t seen = work_sig_.load();
    bool progress = false, pending = false;
    for (auto& lp : lanes_) {
      DdLane& l = *lp;
      const uint64_t sq = l.seq.load(std::memory_order_acquire);
      const uint64_t done = std::min(load_acq64(&l.ctl->done), sq);
      if (done > l.reaped.load(std::memory_order_relaxed)) {
        reap(l, done);
        progress = true;
      }
      if (sq > done) {
        pending = true;
        if (load_acq32(&l.ctl->exits) == l.launches.load(std::memory_order_acquire)) {
          std::unique_lock<std::mutex> g(l.mu, std::try_to_lock);
          if (g.owns_lock()) maybe_relaunch_locked(l);
        }
      }
    }
    const uint64_t t = now_ns();
    if (progress) {
      done_sig_.notify_all();
      last_progress = t;
      continue;
    }
    if (poll_quit_.load()) return;
    if (!pending) {
      work_sig_.wait(seen, 2 * 1000000ll);
      last_progress = now_ns();
      continue;
    }
    // a lane that stopped making progress: surface a CUDA error of its stream (a failed launch
    // or a fault) instead of waiting for the caller's timeout
    if (t - last_check > 50ull * 1000000ull) {
      last_check = t;
      for (auto& lp : lanes_) {
        const cudaError_t e = cudaStreamQuery(lp->stream);
        if (e != cudaSuccess && e != cudaErrorNotReady) {
          fail(SET_ECUDA, std::string("lane stream: ") + cudaGetErrorString(e));
          done_sig_.notify_all();
        }
      }
    }
    if (t - last_progress < (uint64_t)cfg_.spin_us * 1000ull) continue;
    timespec ts{0, (long)kPollSleepNs};
    nanosleep(&ts, nullptr);
  }
}

set_status DevDispatch::wait_all(int64_t timeout_us) {
  const uint64_t t0 = now_ns();
  for (;;) {
    const uint32_t seen = done_sig_.load();
    if (completed_.load() >= submitted_.load()) return SET_OK;
    if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
    int64_t wait_ns = 10 * 1000000ll;
    if (timeout_us >= 0) {
      const int64_t left = timeout_us * 1000ll - (int64_t)(now_ns() - t0);
      if (left <= 0) return SET_ETIMEDOUT;
      wait_ns = std::min(wait_ns, left);
    }
    done_sig_.wait(seen, wait_ns);
  }
}

set_status DevDispatch::stats(set_stats_t* o, uint64_t* launches) {
  if (!o) return SET_EINVAL;
  std::memset(o, 0, sizeof *o);
  o->submitted = submitted_.load();
  o->completed = completed_.load();
  o->failed = failed_.load();
  o->canary_errors = canary_.load();
  const uint64_t t0 = t_first_.load(), t1 = t_last_.load();
  o->elapsed_s = t0 && t1 > t0 ? (double)(t1 - t0) * 1e-9 : 0.0;
  o->jobs_per_s = o->elapsed_s > 0 ? (double)o->completed / o->elapsed_s : 0.0;
  o->p50_us = lat_.quantile(0.50) * 1e-3;
  o->p99_us = lat_.quantile(0.99) * 1e-3;
  o->max_us = lat_.max() * 1e-3;
  o->mean_update_us = 0.0;
  o->mean_launch_us = o->submitted ? (double)submit_ns_.load() * 1e-3 / (double)o->submitted : 0.0;
  o->mem_waits = ring_waits_.load();
  o->mean_queue_us = NAN;
  o->mean_service_us = NAN;
  double gap = NAN;
  o->mean_kernel_gap_us = last_trace_gap(t_reset_.load(), &gap) ? gap : NAN;
  if (launches) {
    uint64_t n = 0;
    for (auto& l : lanes_) n += l->launches.load();
    *launches = n;
  }
  return SET_OK;
}

set_status DevDispatch::reset_stats() {
  submitted_.store(submitted_.load() - completed_.load());
  completed_.store(0);
  failed_.store(0);
  canary_.store(0);
  ring_waits_.store(0);
  submit_ns_.store(0);
  t_first_.store(0);
  t_last_.store(0);
  t_reset_.store(now_ns());
  lat_.reset();
  return SET_OK;
}

set_status DevDispatch::shutdown() {
  stop_.store(true);
  set_status st = wait_all(cfg_.drain_timeout_ms);
  for (auto& l : lanes_) __atomic_store_n(&l->ctl->stop, 1u, __ATOMIC_RELEASE);
  // each loop ends at its next fetch: wait for the streams, bounded
  const uint64_t limit = now_ns() + ((uint64_t)cfg_.idle_us * 1000ull + 5000000000ull);
  for (auto& l : lanes_) {
    if (!l->stream) continue;
    for (;;) {
      const cudaError_t e = cudaStreamQuery(l->stream);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) {
        cudaGetLastError();
        if (st == SET_OK) st = fail(SET_ECUDA, std::string("lane stream at destroy: ") + cudaGetErrorString(e));
        break;
      }
      if (now_ns() > limit) {
        leak_ = true;
        if (st == SET_OK) st = fail(SET_ETIMEDOUT, "a lane's loop did not end at destroy");
        break;
      }
      std::this_thread::yield();
    }
  }
  poll_quit_.store(true);
  work_sig_.notify_all();
  if (poller_.joinable()) poller_.join();
  release();
  return st;
}

void DevDispatch::release() {
  if (poller_.joinable()) {
    poll_quit_.store(true);
    work_sig_.notify_all();
    poller_.join();
  }
  if (leak_) return;
  for (auto& l : lanes_) {
    if (l->ended) cudaEventDestroy(l->ended);
    l->ended = nullptr;
    if (l->exec) cudaGraphExecDestroy(l->exec);
    if (l->graph) cudaGraphDestroy(l->graph);
    if (l->stream) cudaStreamDestroy(l->stream);
    l->exec = nullptr;
    l->graph = nullptr;
    l->stream = nullptr;
  }
  if (dev_block_) cudaFree(dev_block_);
  if (host_block_) cudaFreeHost(host_block_);
  dev_block_ = nullptr;
  host_block_ = nullptr;
}

}  // namespace setrt

struct set_dd {
  setrt::DevDispatch* dd;
};

namespace {
thread_local std::string g_dd_err;
}

extern "C" {

void set_dd_config_default(set_dd_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->num_lanes = 16;
  c->ring_depth = 64;
  c->device = 0;
  c->scan_max_n = 65536;
  c->blur_max_w = 256;
  c->idle_us = 2000;
  c->spin_us = 50;
  c->drain_timeout_ms = 30000;
}

set_status set_dd_create(const set_dd_config* cfg, set_dd** out) {
  if (!out) return SET_EINVAL;
  *out = nullptr;
  set_dd_config c;
  if (cfg)
    c = *cfg;
  else
    set_dd_config_default(&c);
  auto* d = new setrt::DevDispatch();
  std::string err;
  const set_status st = d->init(c, &err);
  if (st != SET_OK) {
    g_dd_err = err;
    setrt::set_thread_error(err.c_str());
    d->shutdown();
    delete d;
    return st;
  }
  *out = new set_dd{d};
  return SET_OK;
}

set_status set_dd_submit(set_dd* dd, const set_job_desc* job, uint64_t* job_id) {
  if (!dd) return SET_EINVAL;
  return dd->dd->submit(job, job_id);
}

set_status set_dd_submit_many(set_dd* dd, const set_job_desc* jobs, size_t n, uint64_t* first_id, size_t* n_done) {
  if (!dd || (n && !jobs)) return SET_EINVAL;
  size_t k = 0;
  set_status st = SET_OK;
  for (; k < n; ++k) {
    uint64_t id = 0;
    st = dd->dd->submit(&jobs[k], &id);
    if (st != SET_OK) break;
    if (k == 0 && first_id) *first_id = id;
  }
  if (n_done) *n_done = k;
  return st;
}

set_status set_dd_wait_all(set_dd* dd, int64_t timeout_us) {
  if (!dd) return SET_EINVAL;
  return dd->dd->wait_all(timeout_us);
}

set_status set_dd_stats(set_dd* dd, set_stats_t* out, uint64_t* graph_launches) {
  if (!dd) return SET_EINVAL;
  return dd->dd->stats(out, graph_launches);
}

set_status set_dd_reset_stats(set_dd* dd) {
  if (!dd) return SET_EINVAL;
  return dd->dd->reset_stats();
}

set_status set_dd_destroy(set_dd* dd) {
  if (!dd) return SET_EINVAL;
  const set_status st = dd->dd->shutdown();
  delete dd->dd;
  delete dd;
  return st;
}

const char* set_dd_last_error(set_dd* dd) {
  if (!dd) return g_dd_err.c_str();
  return dd->dd->last_error();
}

}  // extern "C"
