// dev_dispatch.cpp -- device-dispatch lanes (set_dd_* in set.h): the host protocol.
//
// Per lane: a ring of descriptors and a completion word per entry, a control line (done counter
// and loop exits written by the device, stop flag written by the host) and the lane's loop, all
// owned by a backend (dd_backend.h: the CUDA graphs of dd_cuda.cpp, or the test library's
// simulated device).  This file makes no CUDA call.
//
// Submit plans the job's single stage kernel with the same planners as the executor, writes the
// argument struct into the lane's next ring entry and publishes it with a release store of the
// entry's sequence word; set_dd_submit_many does this for groups of up to kDdBatch
// consecutive jobs on one lane (one lane choice and lock per group, sequence words stored last
// entry first).  Ring entries are reused only after the completion thread has handled
// the job that used them.  The completion thread reads each lane's done counter, completes the
// jobs behind it (status from the completion word, latency) and relaunches lanes whose loop has
// ended while descriptors are waiting; submitters relaunch too, under the lane's mutex.
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
#include "../kernels/params.h"
#include "dd_backend.h"
#include "executor.h"
#include "layout.h"
#include "set.h"
#include "sync.h"
#include "thread_error.h"

namespace setrt {
namespace {

constexpr uint64_t kPollSleepNs = 5000;

struct DdInfo {
  uint64_t id = 0;
  volatile int32_t* status = nullptr;
  uint64_t t_arrival = 0;
};

struct DdLane {
  std::mutex mu;  // writers of this lane's ring and launches of its loop
  DdLaneMem m;    // ring, control line, completion words, scan scratch (from the backend)
  std::unique_ptr<DdInfo[]> info;
  std::atomic<uint64_t> seq{0};       // descriptors published
  std::atomic<uint64_t> reaped{0};    // completions handled
  std::atomic<uint32_t> launches{0};  // loop launches (changed under mu)
};

inline uint32_t load_acq32(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
inline uint64_t load_acq64(const uint64_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

}  // namespace

class DevDispatch {
 public:
  ~DevDispatch() { release(); }
  set_status init(const set_dd_config& cfg, std::string* err);
  // Submits a group of up to min(n, kDdBatch, ring depth) jobs d[0..) to one lane: the prefix
  // that validates; *n_done = jobs published (their ids *first_id, consecutive).  Returns the
  // first job's error when no job was published, else the error of the job after the group (if
  // one stopped it) or SET_OK.
  set_status submit(const set_job_desc* d, uint32_t n, uint64_t* first_id, uint32_t* n_done, DdRangeCache* cache);
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
  set_status launch_locked(uint32_t i);
  bool maybe_relaunch_locked(uint32_t i);
  uint32_t pick_lane();
  set_status validate(const set_job_desc& d, setk::JobLayout* L, std::string* why, DdRangeCache* cache) const;
  void poll_main();
  void reap(DdLane& l, uint64_t upto);
  void release();

  set_dd_config cfg_{};
  uint32_t depth_ = 0, mask_ = 0;
  std::unique_ptr<DdBackend> be_;
  std::vector<std::unique_ptr<DdLane>> lanes_;
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
  be_ = make_dd_backend();
  std::vector<DdLaneMem> mem;
  const set_status st = be_->init(cfg, depth_, &mem, err);
  if (st != SET_OK) return st;
  for (const DdLaneMem& m : mem) {
    auto l = std::make_unique<DdLane>();
    l->m = m;
    l->info.reset(new DdInfo[depth_]);
    lanes_.push_back(std::move(l));
  }
  t_reset_.store(now_ns());
  poller_ = std::thread([this] { poll_main(); });
  return SET_OK;
}

set_status DevDispatch::launch_locked(uint32_t i) {
  DdLane& l = *lanes_[i];
  std::string why;
  if (be_->launch(i, &why) != SET_OK) return fail(SET_ECUDA, why);
  l.launches.store(l.launches.load(std::memory_order_relaxed) + 1, std::memory_order_release);
  return SET_OK;
}

// A lane needs a launch when descriptors wait and every loop launched so far has ended: its
// fetch counted the exit, and the backend reports the last launch complete (for CUDA: the event
// behind it), so one launch of a lane's loop never waits behind another.
bool DevDispatch::maybe_relaunch_locked(uint32_t i) {
  DdLane& l = *lanes_[i];
  if (l.seq.load(std::memory_order_acquire) <= load_acq64(&l.m.ctl->done)) return false;
  if (load_acq32(&l.m.ctl->exits) != l.launches.load(std::memory_order_acquire)) return false;
  std::string why;
  const int e = be_->ended(i, &why);
  if (e == 0) return false;
  if (e < 0) {
    fail(SET_ECUDA, why);
    return false;
  }
  return launch_locked(i) == SET_OK;
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

set_status DevDispatch::validate(const set_job_desc& d, setk::JobLayout* L, std::string* why,
                                 DdRangeCache* cache) const {
  if (d.type != SET_JOB_BLUR_HIST && d.type != SET_JOB_SAXPY_SCAN_MAX && d.type != SET_JOB_IMG_SOBEL_HIST) {
    *why = "set_dd: only SET_JOB_BLUR_HIST, SET_JOB_SAXPY_SCAN_MAX and SET_JOB_IMG_SOBEL_HIST jobs";
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
  if (!be_->buffer_ok(d.in, d.in_bytes, cache) || !be_->buffer_ok(d.out, d.out_bytes, cache)) {
    *why = "set_dd: in/out must be device memory of the object's GPU, each inside one allocation";
    return SET_EINVAL;
  }
  if (((reinterpret_cast<uintptr_t>(d.in) | reinterpret_cast<uintptr_t>(d.out)) & 15u) != 0) {
    *why = "set_dd: in/out must be 16-byte aligned (the kernels use 16-byte accesses in place)";
    return SET_EINVAL;
  }
  return SET_OK;
}

set_status DevDispatch::submit(const set_job_desc* d, uint32_t n, uint64_t* first_id, uint32_t* n_done,
                               DdRangeCache* cache) {
  *n_done = 0;
  if (!d) return fail(SET_EINVAL, "null descriptor");
  if (stop_.load()) return SET_ESHUTDOWN;
  if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
  const uint64_t t0 = now_ns();
  // the group: the prefix of d[0..n) that validates and shares d[0]'s SET_F_NONBLOCK, at most the
  // ring's depth; a job that does not validate is reported after the jobs before it are published
  n = std::min(n, std::min(depth_, setk::kDdBatch));
  setk::JobLayout L[setk::kDdBatch];
  uint32_t g = 0;
  set_status bad = SET_OK;
  std::string why;
  for (; g < n; ++g) {
    if ((d[g].flags ^ d[0].flags) & SET_F_NONBLOCK) break;
    bad = validate(d[g], &L[g], &why, cache);
    if (bad != SET_OK) break;
  }
  if (g == 0) return fail(bad, why);

  const uint32_t li = pick_lane();
  DdLane& l = *lanes_[li];
  std::unique_lock<std::mutex> gl(l.mu);
  const uint64_t s = l.seq.load(std::memory_order_relaxed);
  if (s + g - l.reaped.load(std::memory_order_acquire) > depth_) {
    if (d[0].flags & SET_F_NONBLOCK) {  // publish what fits now
      const uint64_t room = depth_ - (s - l.reaped.load(std::memory_order_acquire));
      if (room == 0) return SET_EAGAIN;
      g = (uint32_t)std::min<uint64_t>(g, room);
      bad = SET_OK;
    } else {
      ring_waits_.fetch_add(1, std::memory_order_relaxed);
      const uint64_t limit = t0 + (uint64_t)cfg_.drain_timeout_ms * 1000000ull;
      while (s + g - l.reaped.load(std::memory_order_acquire) > depth_) {
        maybe_relaunch_locked(li);
        if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
        if (now_ns() > limit) return fail(SET_ETIMEDOUT, "set_dd_submit: the lane's ring stayed full");
        std::this_thread::yield();
      }
    }
  }
  // ids and argument structs under the lane's lock, so that one submitter's ids stay consecutive
  const uint64_t id0 = next_id_.fetch_add(g);
  alignas(16) unsigned char args[setk::kDdBatch][setk::kDdArgBytes];
  uint32_t args_size[setk::kDdBatch];
  for (uint32_t k = 0; k < g; ++k)
    if (!be_->plan(d[k], id0 + k, li, args[k], &args_size[k])) {
      if (k == 0) return fail(SET_EINVAL, "set_dd: the job does not plan to one kernel with a small argument struct");
      g = k;  // the ids after it are skipped
      bad = SET_EINVAL;
      why = "set_dd: the job does not plan to one kernel with a small argument struct";
      break;
    }
  for (uint32_t k = 0; k < g; ++k) {
    const uint32_t slot = (uint32_t)((s + k) & mask_);
    DdInfo& inf = l.info[slot];
    inf.id = id0 + k;
    inf.status = d[k].status;
    inf.t_arrival = d[k].t_arrival_ns ? d[k].t_arrival_ns : t0;
    setk::DdEntry& e = l.m.ring[slot];
    e.kind = d[k].type == SET_JOB_BLUR_HIST        ? setk::kDdKindBlur
             : d[k].type == SET_JOB_SAXPY_SCAN_MAX ? setk::kDdKindScan
                                                   : setk::kDdKindImg;
    e.args_size = args_size[k];
    e.job_id = id0 + k;
    e.trailer = reinterpret_cast<set_trailer*>(static_cast<uint8_t*>(d[k].out) + L[k].out_bytes - sizeof(set_trailer));
    std::memcpy(e.args, args[k], args_size[k]);
  }
  // Publish the group's sequence words last entry first: the lane's fetch waits on the first, and
  // when it sees it the others are already complete, so a group's queued blur or scan jobs run as
  // one batch.
  for (uint32_t k = g; k-- > 0;) __atomic_store_n(&l.m.ring[(s + k) & mask_].seq, s + k + 1, __ATOMIC_RELEASE);
  l.seq.store(s + g, std::memory_order_release);
  uint64_t z = 0;
  t_first_.compare_exchange_strong(z, t0);
  submitted_.fetch_add(g);
  maybe_relaunch_locked(li);
  gl.unlock();
  work_sig_.notify(1);
  submit_ns_.fetch_add(now_ns() - t0, std::memory_order_relaxed);
  if (first_id) *first_id = id0;
  *n_done = g;
  if (bad != SET_OK) return fail(bad, why);
  return sticky_.load() == SET_OK ? SET_OK : (set_status)sticky_.load();
}

void DevDispatch::reap(DdLane& l, uint64_t upto) {
  uint64_t r = l.reaped.load(std::memory_order_relaxed);
  const uint64_t t = now_ns();
  for (; r < upto; ++r) {
    const uint32_t k = (uint32_t)(r & mask_);
    const DdInfo inf = l.info[k];
    const uint32_t w = __atomic_load_n(&l.m.cmpl[k], __ATOMIC_ACQUIRE);
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
  be_->bind_thread();
  uint64_t last_progress = now_ns(), last_check = last_progress;
  for (;;) {
    const uint32_t seen = work_sig_.load();
    bool progress = false, pending = false;
    for (uint32_t i = 0; i < (uint32_t)lanes_.size(); ++i) {
      DdLane& l = *lanes_[i];
      const uint64_t sq = l.seq.load(std::memory_order_acquire);
      const uint64_t done = std::min(load_acq64(&l.m.ctl->done), sq);
      if (done > l.reaped.load(std::memory_order_relaxed)) {
        reap(l, done);
        progress = true;
      }
      if (sq > done) {
        pending = true;
        if (load_acq32(&l.m.ctl->exits) == l.launches.load(std::memory_order_acquire)) {
          std::unique_lock<std::mutex> g(l.mu, std::try_to_lock);
          if (g.owns_lock()) maybe_relaunch_locked(i);
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
    // a lane that stopped making progress: surface an error of its loop (a failed launch or a
    // fault) instead of waiting for the caller's timeout
    if (t - last_check > 50ull * 1000000ull) {
      last_check = t;
      for (uint32_t i = 0; i < (uint32_t)lanes_.size(); ++i) {
        std::string why;
        if (be_->ended(i, &why) < 0) {
          fail(SET_ECUDA, why);
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
  for (auto& l : lanes_) __atomic_store_n(&l->m.ctl->stop, 1u, __ATOMIC_RELEASE);
  // each loop ends at its next fetch: wait for every lane's last launch, bounded
  const uint64_t limit = now_ns() + ((uint64_t)cfg_.idle_us * 1000ull + 5000000000ull);
  for (uint32_t i = 0; i < (uint32_t)lanes_.size(); ++i) {
    for (;;) {
      std::string why;
      const int e = be_->ended(i, &why);
      if (e == 1) break;
      if (e < 0) {
        if (st == SET_OK) st = fail(SET_ECUDA, why);
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
  if (be_) be_->release(leak_);
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
  uint32_t done = 0;
  setrt::DdRangeCache cache;
  return dd->dd->submit(job, 1, job_id, &done, &cache);
}

set_status set_dd_submit_many(set_dd* dd, const set_job_desc* jobs, size_t n, uint64_t* first_id, size_t* n_done) {
  if (!dd || (n && !jobs)) return SET_EINVAL;
  size_t k = 0;
  set_status st = SET_OK;
  setrt::DdRangeCache cache;  // buffers of this call's jobs usually share a few allocations
  while (k < n) {  // groups of consecutive jobs, one lane each
    uint64_t id = 0;
    uint32_t done = 0;
    st = dd->dd->submit(&jobs[k], (uint32_t)std::min<size_t>(n - k, setk::kDdBatch), &id, &done, &cache);
    if (done && k == 0 && first_id) *first_id = id;
    k += done;
    if (st != SET_OK) break;
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
