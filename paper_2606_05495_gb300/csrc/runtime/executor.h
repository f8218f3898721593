// executor.h -- the SET executor's host runtime (Sec. 4.2, Algorithms 1-3), independent of how a
// job reaches the GPU.  The Device interface owns streams, slot memory and graph execs; the
// Executor owns queues, the free-slot pool, dispatch threads, counters and the completion path.
#pragma once

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "arena.h"
#include "set.h"
#include "sync.h"

namespace setrt {

class Executor;

struct JobRec {
  set_job_desc d{};
  uint64_t id = 0;
  uint64_t t_submit_ns = 0;
  uint32_t queued_lane = 0;
};

// One ring entry of a lane: a device buffer with one graph exec per job type bound to it.
struct Slot {
  uint32_t index = 0, lane = 0, ring = 0;
  uint8_t* dev = nullptr;
  size_t bytes = 0;
  uint32_t gen = 0;       // bumped by every completion of this slot
  JobRec job{};           // job in flight
  uint64_t t_dispatch_ns = 0;  // the dispatcher took the job (written before its launch)
  Executor* ex = nullptr;
  void* dev_state = nullptr;  // owned by the Device
  std::atomic<bool> quiet{false};  // set while a baseline reuses the slot's graphs: no completion path
  uint8_t* job_mem = nullptr;      // arena mode: the job's [in | out | scratch] block
  size_t job_mem_bytes = 0;
  Slot* group_prev = nullptr;      // earlier slot of the same completion group (cb_every > 1)
  std::vector<JobRec> batch;       // batched form: the jobs of this launch (empty: the single `job`)
  volatile uint64_t* stamps = nullptr;  // stamps mode: {entry, exit} per kernel (mapped host memory)
  uint32_t stamp_deps[8] = {};          // dependency mask of each kernel of the launch
  int stamp_nk = 0;
};

struct LaunchCost {
  uint64_t updates = 0;   // node parameter updates issued
  uint64_t update_ns = 0; // host time spent updating
  uint64_t launch_ns = 0; // host time spent launching and chaining the callback
};

class Device {
 public:
  virtual ~Device() = default;
  // Allocates slot memory and per-slot graph execs; fills dev / bytes / dev_state of every slot.
  virtual set_status init(const set_config& cfg, std::vector<Slot>& slots, std::string* err) = 0;
  // UpdateGraphParams(job, slot) + GraphLaunch on the slot's lane, and AddCallback when
  // `callback` is set: the callback, run after the D2H copy, must call
  // Executor::on_complete_group(slot) (the slot and every slot chained through group_prev).
  virtual set_status launch(Slot& s, bool callback, LaunchCost* cost, std::string* err) = 0;
  // UpdateGraphParams alone (bind-at-submit): the slot's graph is rebound to s.job now and a later
  // launch_bound(s) launches it without updating.
  virtual set_status prepare(Slot& s, LaunchCost* cost, std::string* err) = 0;
  virtual set_status launch_bound(Slot& s, bool callback, LaunchCost* cost, std::string* err) = 0;
  // Batched form: one launch of the slot's batch graph over the jobs in s.batch (same type).
  virtual set_status launch_batch(Slot& s, bool callback, LaunchCost* cost, std::string* err) = 0;
  // AddCallback alone: completes the group ending at `s` (already launched) on its lane.
  virtual set_status attach_callback(Slot& s, std::string* err) = 0;
  // Waits for all device work of the context (used at destruction).
  virtual void drain() = 0;
  // Called first on every dispatch thread (makes the context's device current on that thread:
  // driver-API calls such as tensor-map encoding need it before any runtime call has been made).
  virtual void thread_init() = 0;
  // Arena mode: device range the executor's buddy allocator manages (nullptr otherwise).
  virtual uint8_t* arena_base() = 0;
  // True if graphs for jobs of this type were instantiated.
  virtual bool supports(uint32_t type) const = 0;
  // SET_IO_MAPPED and sm_copies: true if p is page-locked host memory the device can address at
  // the same address (device memory is refused: the completion path reads the trailer from the
  // host output).
  virtual bool io_accessible(const void* p) const = 0;
  // SET_IO_DEVICE_INPLACE: true if p is device memory of the context's GPU.
  virtual bool io_device(const void* p) const = 0;
  // Autotuner of the batched form (the context's workers are idle): picks jobs per launch (<=
  // max_batch) and the image kernel's tile / CTAs per SM, applies them to later launches.
  virtual set_status autotune(uint32_t type, const JobRec* sample, size_t n, int max_batch, set_tune_result* out,
                              std::string* err) = 0;
  // Runs a baseline programming model over the same slots (the context's workers are idle).
  virtual set_status run_baseline(int kind, const JobRec* jobs, size_t n, std::vector<Slot>& slots,
                                  BuddyArena* arena, LogHist* lat, LaunchCost* cost, uint64_t* t0_ns,
                                  uint64_t* t1_ns, std::string* err) = 0;
};

// The last CUPTI trace's mean kernel gap (process-wide): written by set_trace_stop, read by the
// contexts' statistics when the trace began after their last reset.
void note_trace_gap(double gap_us, uint64_t t_start_ns);
bool last_trace_gap(uint64_t since_ns, double* gap_us);

// Which side of a job the kernels read / write in host memory themselves (no copy node).
// The stage kernels address the caller's buffer itself (no copy node on that side).
inline bool io_maps_in(int io_mode) {
  return io_mode == SET_IO_MAPPED || io_mode == SET_IO_MAPPED_IN || io_mode == SET_IO_DEVICE_INPLACE;
}
inline bool io_maps_out(int io_mode) {
  return io_mode == SET_IO_MAPPED || io_mode == SET_IO_MAPPED_OUT || io_mode == SET_IO_DEVICE_INPLACE;
}
// The job's output (and its trailer) stays in device memory.
inline bool io_out_on_device(int io_mode) { return io_mode == SET_IO_DEVICE || io_mode == SET_IO_DEVICE_INPLACE; }

// Product CUDA device; the host-simulation test library links its own factory instead.
std::unique_ptr<Device> make_device(const set_config& cfg);

class Executor {
 public:
  static set_status create(const set_config& cfg, Executor** out, std::string* err);
  ~Executor();

  set_status submit(const set_job_desc* d, uint64_t* id);                                    // Alg. 1
  set_status submit_many(const set_job_desc* d, size_t n, uint64_t* first_id, size_t* n_done);
  set_status wait_all(int64_t timeout_us);
  void stats(set_stats_t* s) const;
  void reset_stats();
  set_status run_baseline(int kind, const set_job_desc* jobs, size_t n, set_stats_t* out);
  set_status autotune(uint32_t type, const set_job_desc* sample, size_t n, set_tune_result* out);
  set_status serve(int mode, const set_job_desc* jobs, const uint64_t* arrival_ns, size_t n, set_stats_t* out);
  // Bytes of the arena block a job needs (its in, out and scratch regions), 0 if invalid.
  static size_t job_block_bytes(const set_job_desc& d);
  const char* last_error();

  // Algorithm 3 (asynchronous resource return).  Runs on the device's callback thread after the
  // slot's D2H copy completed: checks the returned trailer, counts the job done, returns the slot
  // to W_pool and wakes one dispatcher.
  void on_complete(Slot& s, int32_t dev_status);
  // Completes `last` and every slot chained before it through group_prev (one callback per group).
  void on_complete_group(Slot& last);

  const set_config& config() const { return cfg_; }

 private:
  explicit Executor(const set_config& cfg);
  void worker_main(int w);
  void flush_groups(std::vector<Slot*>& pending, std::vector<int>& count);
  void launch_slot(Slot& s, bool bound, std::vector<Slot*>& pending, std::vector<int>& count, int every);
  bool find_job(uint32_t lane, JobRec& j, bool& stolen);  // Alg. 2 FindJob
  set_status validate(const set_job_desc& d, std::string* why) const;
  set_status fail(set_status st, const std::string& msg);
  int32_t check_trailer(const Slot& s, const JobRec& j) const;
  void finish_job(Slot& s, const JobRec& j, int32_t dev_status, uint64_t t);
  size_t batch_block_bytes(const std::vector<JobRec>& b, const JobRec* extra) const;
  size_t slot_payload_bytes() const;

  set_config cfg_;
  std::unique_ptr<Device> dev_;
  std::vector<Slot> slots_;
  std::vector<std::unique_ptr<MpmcRing<JobRec>>> queues_;  // Q_i, one per lane
  std::unique_ptr<MpmcRing<uint32_t>> free_;                // W_pool of slot indices
  std::unique_ptr<MpmcRing<uint32_t>> ready_;               // bind-at-submit: slots bound to a job
  std::vector<std::thread> workers_;

  Signal free_sig_, job_sig_, space_sig_, done_sig_;
  std::atomic<bool> stop_{false};
  std::atomic<int> sticky_{SET_OK};

  std::atomic<uint64_t> c_next_{0};       // next job id
  std::atomic<uint64_t> c_submitted_{0};
  std::atomic<uint64_t> c_done_{0};
  std::atomic<uint64_t> c_failed_{0};
  std::atomic<uint64_t> done_target_{~0ull};
  std::atomic<uint64_t> steals_{0}, updates_{0}, canary_errors_{0};
  std::atomic<uint64_t> update_ns_{0}, launch_ns_{0}, launched_{0};
  std::atomic<uint64_t> queue_ns_{0}, service_ns_{0}, timed_jobs_{0};  // latency breakdown
  std::atomic<uint64_t> t_first_ns_{0}, t_last_ns_{0};
  std::atomic<uint64_t> t_reset_ns_{0};  // last reset of the statistics (creation)
  std::atomic<uint64_t> stat_base_submitted_{0}, stat_base_done_{0}, stat_base_failed_{0};
  std::atomic<uint64_t> mem_waits_{0};
  std::atomic<uint64_t> order_errors_{0};
  LogHist lat_;
  BuddyArena arena_;
  bool use_arena_ = false;
  std::atomic<int> batch_limit_{1};  // jobs per batched launch (autotuner may lower it)
  Signal mem_sig_;

  std::mutex err_mu_;
  std::string err_;
  std::string err_copy_;
};

}  // namespace setrt
