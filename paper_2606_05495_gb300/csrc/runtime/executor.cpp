// executor.cpp -- queues, free-slot pool, dispatch workers and the completion path of the SET
// executor (Sec. 4.2; Algorithm 1 = submit, Algorithm 2 = worker_main / find_job,
// Algorithm 3 = on_complete).  Device specifics live behind the Device interface.
#include "executor.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "layout.h"

namespace setrt {

namespace {
std::mutex g_trace_mu;
double g_trace_gap_us = 0.0;
uint64_t g_trace_start_ns = 0;  // 0: no trace yet

void normalize(set_config& c) {
  if (c.ring_depth <= 0) c.ring_depth = 2;
  if (c.queue_capacity <= 0) c.queue_capacity = 4;
  if (c.steal != 0) c.steal = 1;
  if (c.type_mask == 0) c.type_mask = ~0u;
  if (c.drain_timeout_ms <= 0) c.drain_timeout_ms = 30000;
  if (c.spin_us < 0) c.spin_us = 0;
  if (c.batch_max < 1) c.batch_max = 1;
  if (c.batch_max > setk::kMaxBatch) c.batch_max = setk::kMaxBatch;
  if (c.img_ctas_per_sm < 1) c.img_ctas_per_sm = 4;
}

// Spins (plain atomic loads, no system call) for up to spin_ns while `ready` is false.
template <class F>
bool spin_until(F ready, uint64_t spin_ns) {
  if (spin_ns == 0) return ready();
  const uint64_t t_end = now_ns() + spin_ns;
  for (int k = 0;; ++k) {
    if (ready()) return true;
    if ((k & 63) == 63 && now_ns() > t_end) return false;
  }
}

}  // namespace

Executor::Executor(const set_config& cfg) : cfg_(cfg) {}

void note_trace_gap(double gap_us, uint64_t t_start_ns) {
  std::lock_guard<std::mutex> g(g_trace_mu);
  g_trace_gap_us = gap_us;
  g_trace_start_ns = t_start_ns;
}

bool last_trace_gap(uint64_t since_ns, double* gap_us) {
  std::lock_guard<std::mutex> g(g_trace_mu);
  if (g_trace_start_ns == 0 || g_trace_start_ns < since_ns) return false;
  *gap_us = g_trace_gap_us;
  return true;
}

set_status Executor::create(const set_config& cfg_in, Executor** out, std::string* err) {
  set_config cfg = cfg_in;
  normalize(cfg);
  if (!out || cfg.num_streams < 1 || cfg.num_streams > 1024 || cfg.num_workers < 1 || cfg.num_workers > 256 ||
      cfg.ring_depth > 64 || cfg.queue_capacity > (1 << 20) || cfg.slot_bytes < 4096 ||
      cfg.io_mode < SET_IO_HOST || cfg.io_mode > SET_IO_DEVICE_INPLACE || cfg.cb_mode < 0 || cfg.cb_mode > 3 ||
      ((io_maps_in(cfg.io_mode) || io_maps_out(cfg.io_mode)) && cfg.batch_max > 1) ||
      cfg.bind_at_submit < 0 || cfg.bind_at_submit > 2 || (cfg.bind_at_submit && cfg.batch_max > 1) ||
      (cfg.guards && (cfg.arena_bytes || cfg.batch_max > 1 || cfg.io_mode != SET_IO_HOST)) || cfg.sm_copies < 0 ||
      cfg.sm_copies > 1 || (cfg.sm_copies && (cfg.io_mode != SET_IO_HOST || cfg.batch_max > 1))) {
    *err = "invalid set_config (num_streams 1..1024, num_workers 1..256, ring_depth <= 64, slot_bytes >= 4096, "
           "cb_mode 0..3, no batched form with mapped I/O or bind_at_submit; guards only with SET_IO_HOST, "
           "without arena or batches; sm_copies 0/1, only with SET_IO_HOST and without batches)";
    return SET_EINVAL;
  }
  std::unique_ptr<Executor> ex(new Executor(cfg));
  const uint32_t L = (uint32_t)cfg.num_streams, R = (uint32_t)cfg.ring_depth;
  ex->slots_ = std::vector<Slot>((size_t)L * R);
  for (uint32_t i = 0; i < L * R; ++i) {
    Slot& s = ex->slots_[i];
    s.index = i;
    s.lane = i % L;  // interleaved so that the first b tokens cover every lane once
    s.ring = i / L;
    s.ex = ex.get();
  }
  ex->dev_ = make_device(cfg);
  if (!ex->dev_) {
    *err = "no device backend";
    return SET_EINVAL;
  }
  const set_status st = ex->dev_->init(cfg, ex->slots_, err);
  if (st != SET_OK) return st;
  if (cfg.arena_bytes) {
    ex->arena_.init(ex->dev_->arena_base(), cfg.arena_bytes, size_t(64) << 10);
    ex->use_arena_ = true;
  }
  ex->batch_limit_.store(cfg.batch_max);
  ex->t_reset_ns_.store(now_ns());
  for (uint32_t i = 0; i < L; ++i) ex->queues_.emplace_back(new MpmcRing<JobRec>((size_t)cfg.queue_capacity));
  ex->free_.reset(new MpmcRing<uint32_t>((size_t)L * R));
  if (cfg.bind_at_submit) ex->ready_.reset(new MpmcRing<uint32_t>((size_t)L * R));
  for (uint32_t i = 0; i < L * R; ++i) ex->free_->push(i);
  for (int w = 0; w < cfg.num_workers; ++w) ex->workers_.emplace_back(&Executor::worker_main, ex.get(), w);
  *out = ex.release();
  return SET_OK;
}

Executor::~Executor() {
  wait_all((int64_t)cfg_.drain_timeout_ms * 1000);
  stop_.store(true);
  free_sig_.notify_all();
  job_sig_.notify_all();
  space_sig_.notify_all();
  done_sig_.notify_all();
  for (auto& t : workers_) t.join();
  if (dev_) dev_->drain();
  dev_.reset();
}

set_status Executor::fail(set_status st, const std::string& msg) {
  std::lock_guard<std::mutex> g(err_mu_);
  err_ = msg;
  if (st == SET_ECUDA) sticky_.store(SET_ECUDA);
  return st;
}

const char* Executor::last_error() {
  std::lock_guard<std::mutex> g(err_mu_);
  err_copy_ = err_;
  return err_copy_.c_str();
}

set_status Executor::validate(const set_job_desc& d, std::string* why) const {
  setk::JobLayout L;
  if (!setk::job_sizes(d.type, d.dims, &L)) {
    *why = "unknown job type or dims out of range";
    return SET_EINVAL;
  }
  if (!(cfg_.type_mask & (1u << d.type)) || !dev_->supports(d.type)) {
    *why = "job type not instantiated in this context (type_mask)";
    return SET_EINVAL;
  }
  if (!d.in || !d.out) {
    *why = "null in/out";
    return SET_EINVAL;
  }
  if (d.in_bytes != L.in_bytes || d.out_bytes != L.out_bytes) {
    *why = "in_bytes/out_bytes do not match the job type's layout";
    return SET_EINVAL;
  }
  if (d.type == SET_JOB_MLP_LN && (!d.shared[0] || !d.shared[1])) {
    *why = "MLP job needs device weights in shared[0], shared[1]";
    return SET_EINVAL;
  }
  if (cfg_.io_mode == SET_IO_DEVICE_INPLACE) {
    if (d.type == SET_JOB_MLP_LN) {
      *why = "in-place device I/O: not for MLP jobs";
      return SET_EINVAL;
    }
    if (!dev_->io_device(d.in) || !dev_->io_device(d.out) ||
        ((reinterpret_cast<uintptr_t>(d.in) | reinterpret_cast<uintptr_t>(d.out)) & 15u)) {
      *why = "in-place device I/O: in/out must be 16-byte aligned device memory of the context's GPU";
      return SET_EINVAL;
    }
  } else if (io_maps_in(cfg_.io_mode) && d.type == SET_JOB_MLP_LN) {
    *why = "mapped input: MLP inputs feed TMA loads and must be copied into device memory";
    return SET_EINVAL;
  }
  const bool host_mapped = cfg_.io_mode != SET_IO_DEVICE_INPLACE;
  if (host_mapped && ((io_maps_in(cfg_.io_mode) && !dev_->io_accessible(d.in)) ||
                      (io_maps_out(cfg_.io_mode) && !dev_->io_accessible(d.out)))) {
    *why = "mapped I/O: in/out must be page-locked host memory the GPU can address (not device memory)";
    return SET_EINVAL;
  }
  if ((io_maps_in(cfg_.io_mode) && (reinterpret_cast<uintptr_t>(d.in) & 15u)) ||
      (io_maps_out(cfg_.io_mode) && (reinterpret_cast<uintptr_t>(d.out) & 15u))) {
    *why = "mapped I/O: in/out must be 16-byte aligned (the kernels use 16-byte accesses in place)";
    return SET_EINVAL;
  }
  if (cfg_.sm_copies && (!dev_->io_accessible(d.in) || !dev_->io_accessible(d.out) ||
                         ((reinterpret_cast<uintptr_t>(d.in) | reinterpret_cast<uintptr_t>(d.out)) & 15u))) {
    *why = "sm_copies: in/out must be 16-byte aligned page-locked host memory the GPU can address";
    return SET_EINVAL;
  }
  const size_t ctl = setk::slot_control_bytes(cfg_.slot_bytes);
  if (use_arena_) {
    if (job_block_bytes(d) > arena_.max_block() || job_block_bytes(d) > cfg_.slot_bytes ||
        setk::control_offset(d.type) + L.persist_bytes > ctl) {
      *why = "job larger than the arena's largest block or than slot_bytes";
      return SET_ENOMEM;
    }
    return SET_OK;
  }
  if (cfg_.guards)
    setk::place_job_guarded(&L, ctl);
  else
    setk::place_job(&L, ctl);
  if (L.end > cfg_.slot_bytes || setk::control_offset(d.type) + L.persist_bytes > ctl) {
    *why = "job does not fit the slot (slot_bytes too small)";
    return SET_ENOMEM;
  }
  return SET_OK;
}

size_t Executor::job_block_bytes(const set_job_desc& d) {
  setk::JobLayout L;
  if (!setk::job_sizes(d.type, d.dims, &L)) return 0;
  setk::place_job(&L, 0);
  return L.end;
}

// Algorithm 1 (job submitter): claim an id, push to the shortest queue that is not full; with
// bind_at_submit, first try to bind the job to a free slot here (and launch it, mode 2).
set_status Executor::submit(const set_job_desc* d, uint64_t* id_out) {
  if (!d) return SET_EINVAL;
  if (stop_.load()) return SET_ESHUTDOWN;
  if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
  std::string why;
  const set_status v = validate(*d, &why);
  if (v != SET_OK) return fail(v, why);
  JobRec j;
  j.d = *d;
  uint32_t tok = 0;
  bool have_slot = ready_ && free_->pop(tok);
  if (have_slot && use_arena_) {
    // arena mode: the job also needs its device block now; without one it is bound at dispatch
    Slot& s = slots_[tok];
    s.job_mem = arena_.alloc(job_block_bytes(*d), &s.job_mem_bytes);
    if (!s.job_mem) {
      free_->push(tok);
      free_sig_.notify(1);
      have_slot = false;
    }
  }
  if (have_slot) {
    // Algorithm 1 with UpdateGraphParams at submit: bind the job to a free slot now, queue it bound
    Slot& s = slots_[tok];
    j.id = c_next_.fetch_add(1);
    const uint64_t t = now_ns();
    j.t_submit_ns = d->t_arrival_ns ? d->t_arrival_ns : t;
    uint64_t z = 0;
    t_first_ns_.compare_exchange_strong(z, t);
    j.queued_lane = s.lane;
    c_submitted_.fetch_add(1);
    s.job = j;
    s.batch.clear();
    s.t_dispatch_ns = 0;
    s.group_prev = nullptr;
    LaunchCost cost;
    std::string e;
    const set_status st = dev_->prepare(s, &cost, &e);
    updates_.fetch_add(cost.updates, std::memory_order_relaxed);
    update_ns_.fetch_add(cost.update_ns, std::memory_order_relaxed);
    if (st != SET_OK) {
      fail(st, e);
      on_complete(s, st);  // the job is accepted and completes with the error
    } else if (cfg_.bind_at_submit == 2) {
      // launch at submit: the submitting thread is the dispatcher (one callback per job)
      if (sticky_.load() != SET_OK) {
        on_complete(s, sticky_.load());
      } else {
        s.t_dispatch_ns = now_ns();
        LaunchCost lc;
        const set_status ls = dev_->launch_bound(s, true, &lc, &e);
        launch_ns_.fetch_add(lc.launch_ns, std::memory_order_relaxed);
        launched_.fetch_add(1, std::memory_order_relaxed);
        if (ls != SET_OK) {
          fail(ls, e);
          on_complete(s, ls);
        }
      }
    } else {
      ready_->push(tok);  // capacity = all slots: never full
      free_sig_.notify(1);
      job_sig_.notify(1);
    }
    if (id_out) *id_out = j.id;
    return SET_OK;
  }
  bool claimed = false;
  const uint32_t L = (uint32_t)queues_.size();
  for (;;) {
    const uint32_t seen = space_sig_.load();
    int best = -1;
    size_t best_sz = SIZE_MAX;
    for (uint32_t i = 0; i < L; ++i) {
      const size_t sz = queues_[i]->size_approx();
      if (sz < queues_[i]->capacity() && sz < best_sz) {
        best = (int)i;
        best_sz = sz;
      }
    }
    if (best >= 0) {
      if (!claimed) {
        j.id = c_next_.fetch_add(1);
        const uint64_t t = now_ns();
        j.t_submit_ns = d->t_arrival_ns ? d->t_arrival_ns : t;
        uint64_t z = 0;
        t_first_ns_.compare_exchange_strong(z, t);
        claimed = true;
      }
      j.queued_lane = (uint32_t)best;
      c_submitted_.fetch_add(1);
      if (queues_[best]->push(j)) {
        job_sig_.notify(1);
        if (id_out) *id_out = j.id;
        return SET_OK;
      }
      c_submitted_.fetch_sub(1);  // lost the last position to another submitter: retry
      continue;
    }
    if (d->flags & SET_F_NONBLOCK) return SET_EAGAIN;
    if (stop_.load()) return SET_ESHUTDOWN;
    if (spin_until([&] { return space_sig_.load() != seen || stop_.load(); }, (uint64_t)cfg_.spin_us * 1000ull)) continue;
    space_sig_.wait(seen, 50 * 1000000ll);
  }
}

set_status Executor::submit_many(const set_job_desc* d, size_t n, uint64_t* first_id, size_t* n_done) {
  size_t k = 0;
  set_status st = SET_OK;
  for (; k < n; ++k) {
    uint64_t id;
    st = submit(&d[k], &id);
    if (st != SET_OK) break;
    if (k == 0 && first_id) *first_id = id;
  }
  if (n_done) *n_done = k;
  return st;
}

// Algorithm 2, FindJob: the slot's own lane queue first, then lanes (w + k) mod b.
bool Executor::find_job(uint32_t lane, JobRec& j, bool& stolen) {
  if (queues_[lane]->pop(j)) {
    stolen = false;
    return true;
  }
  if (!cfg_.steal) return false;
  const uint32_t L = (uint32_t)queues_.size();
  for (uint32_t k = 1; k < L; ++k) {
    if (queues_[(lane + k) % L]->pop(j)) {
      stolen = true;
      return true;
    }
  }
  return false;
}

// Closes every open completion group of this dispatcher (AddCallback on its last slot): done
// before the dispatcher waits, so that no launched job is left without a completion.
void Executor::flush_groups(std::vector<Slot*>& pending, std::vector<int>& count) {
  for (size_t l = 0; l < pending.size(); ++l) {
    if (!pending[l]) continue;
    std::string e;
    const set_status st = dev_->attach_callback(*pending[l], &e);
    if (st != SET_OK) {
      fail(st, e);
      on_complete_group(*pending[l]);  // no callback will come: complete them here (sticky error)
    }
    pending[l] = nullptr;
    count[l] = 0;
  }
}

// Algorithm 2, dispatcher loop: launch a slot bound at submit if one is ready; else pop a free
// slot (W_pool), FindJob, UpdateGraphParams, LaunchJob.  Waiting is a spin, then a futex sleep on
// the pool / submit signals; the device is never polled here.
void Executor::worker_main(int) {
  dev_->thread_init();
  const uint64_t spin_ns = (uint64_t)cfg_.spin_us * 1000ull;
  const int every = (cfg_.cb_mode == 2 || cfg_.cb_every < 1) ? 1 : cfg_.cb_every;
  std::vector<Slot*> pending(queues_.size(), nullptr);  // open completion group per lane
  std::vector<int> count(queues_.size(), 0);
  JobRec carry;             // batched form: a job popped while filling a batch that did not fit it
  bool have_carry = false;
  for (;;) {
    uint32_t tok = 0;
    bool bound = false;
    for (;;) {
      const uint32_t seen = free_sig_.load();
      if (stop_.load()) {
        flush_groups(pending, count);
        return;
      }
      if (ready_ && ready_->pop(tok)) {  // bound at submit: only the launch is left
        bound = true;
        break;
      }
      if (free_->pop(tok)) break;
      flush_groups(pending, count);  // about to wait: every launched job must own a callback
      if (spin_until([&] { return free_sig_.load() != seen || stop_.load(); }, spin_ns)) continue;
      free_sig_.wait(seen, -1);
    }
    if (bound) {
      launch_slot(slots_[tok], true, pending, count, every);
      continue;
    }
    Slot& s = slots_[tok];
    JobRec j;
    bool stolen = false, got = false, yielded = false;
    for (;;) {
      const uint32_t seen = job_sig_.load();
      if (have_carry) {
        j = carry;
        have_carry = false;
        got = true;
        break;
      }
      if (find_job(s.lane, j, stolen)) {
        got = true;
        break;
      }
      if (ready_ && ready_->size_approx() > 0) {  // a bound job waits for a launcher: give the slot back
        free_->push(tok);
        free_sig_.notify(1);
        yielded = true;
        break;
      }
      flush_groups(pending, count);
      if (stop_.load()) break;
      if (!cfg_.steal) {
        // without stealing, a slot whose lane has no work goes back to the pool so that a
        // slot of a lane with queued jobs can be taken
        free_->push(tok);
        free_sig_.notify(1);
        job_sig_.wait(seen, 200 * 1000ll);
        break;
      }
      if (spin_until([&] { return job_sig_.load() != seen || stop_.load(); }, spin_ns)) continue;
      job_sig_.wait(seen, -1);
    }
    if (!got) {
      if (yielded) continue;
      if (stop_.load() && cfg_.steal) {
        free_->push(tok);
        return;
      }
      continue;
    }
    space_sig_.notify(1);
    if (stolen) steals_.fetch_add(1, std::memory_order_relaxed);
    s.t_dispatch_ns = 0;
    s.job = j;
    s.batch.clear();
    const int blim = batch_limit_.load(std::memory_order_relaxed);
    if (blim > 1 && setk::batchable(j.d.type)) {
      // batched form: take what is queued now (no waiting), same type, while it fits one block
      s.batch.push_back(j);
      while ((int)s.batch.size() < blim) {
        JobRec k;
        bool st2 = false;
        if (!find_job(s.lane, k, st2)) break;
        space_sig_.notify(1);
        if (k.d.type != j.d.type || batch_block_bytes(s.batch, &k) > slot_payload_bytes()) {
          carry = k;
          have_carry = true;
          break;
        }
        s.batch.push_back(k);
      }
      if (s.batch.size() == 1) s.batch.clear();  // a batch of one runs the single-job graph
    }
    if (use_arena_) {
      // admission by free device memory: wait (in arrival order of this worker) for a block
      const size_t need = s.batch.empty() ? job_block_bytes(j.d) : batch_block_bytes(s.batch, nullptr);
      bool waited = false;
      for (;;) {
        const uint32_t seen = mem_sig_.load();
        s.job_mem = arena_.alloc(need, &s.job_mem_bytes);
        if (s.job_mem || stop_.load()) break;
        waited = true;
        if (spin_until([&] { return mem_sig_.load() != seen || stop_.load(); }, spin_ns)) continue;
        mem_sig_.wait(seen, 100 * 1000000ll);
      }
      if (waited) mem_waits_.fetch_add(1, std::memory_order_relaxed);
      if (!s.job_mem) {
        on_complete(s, SET_ESHUTDOWN);
        continue;
      }
    }
    launch_slot(s, false, pending, count, every);
  }
}

// LaunchJob + AddCallback for a slot that holds its job (bound: its graph was already rebound at
// submit).  The slot joins its lane's open completion group, which closes every `every` launches.
void Executor::launch_slot(Slot& s, bool bound, std::vector<Slot*>& pending, std::vector<int>& count, int every) {
  if (sticky_.load() != SET_OK) {
    s.group_prev = nullptr;
    on_complete(s, sticky_.load());
    return;
  }
  s.t_dispatch_ns = now_ns();  // admitted: from here on the job is being launched
  LaunchCost cost;
  std::string e;
  s.group_prev = pending[s.lane];
  const bool close = ++count[s.lane] >= every;
  const set_status st = bound            ? dev_->launch_bound(s, close, &cost, &e)
                        : s.batch.empty() ? dev_->launch(s, close, &cost, &e)
                                          : dev_->launch_batch(s, close, &cost, &e);
  if (st == SET_OK) {
    pending[s.lane] = close ? nullptr : &s;
    if (close) count[s.lane] = 0;
  } else {
    count[s.lane] -= 1;
  }
  updates_.fetch_add(cost.updates, std::memory_order_relaxed);
  update_ns_.fetch_add(cost.update_ns, std::memory_order_relaxed);
  launch_ns_.fetch_add(cost.launch_ns, std::memory_order_relaxed);
  launched_.fetch_add(1, std::memory_order_relaxed);
  if (st != SET_OK) {
    fail(st, e);
    s.group_prev = nullptr;
    on_complete(s, st);
  }
}

void Executor::on_complete_group(Slot& last) {
  // completing a slot hands it back to W_pool, so read each link before completing its slot
  Slot* s = &last;
  while (s) {
    Slot* prev = s->group_prev;
    s->group_prev = nullptr;
    on_complete(*s, SET_OK);
    s = prev;
  }
}

int32_t Executor::check_trailer(const Slot& s, const JobRec& j) const {
  if (io_out_on_device(cfg_.io_mode)) return SET_OK;  // the trailer stays in device memory
  set_trailer t;
  std::memcpy(&t, static_cast<const uint8_t*>(j.d.out) + j.d.out_bytes - sizeof(set_trailer), sizeof t);
  if (t.job_id != j.id || t.slot_gen != s.gen || (t.word >> 16) != SET_TRAILER_MAGIC) return -1000;
  if (t.word & 0xFFFFu) return SET_EDEVICE;
  return SET_OK;
}

size_t Executor::slot_payload_bytes() const {
  if (use_arena_) return const_cast<BuddyArena&>(arena_).max_block();
  const size_t ctl = setk::slot_control_bytes(cfg_.slot_bytes);
  return cfg_.slot_bytes > ctl ? cfg_.slot_bytes - ctl : 0;
}

size_t Executor::batch_block_bytes(const std::vector<JobRec>& b, const JobRec* extra) const {
  setk::BatchItem items[setk::kMaxBatch];
  int nb = 0;
  for (const auto& j : b) {
    std::memcpy(items[nb].dims, j.d.dims, sizeof items[nb].dims);
    items[nb++].job_id = j.id;
  }
  if (extra) {
    if (nb >= setk::kMaxBatch) return ~size_t(0);
    std::memcpy(items[nb].dims, extra->d.dims, sizeof items[nb].dims);
    items[nb++].job_id = extra->id;
  }
  setk::BatchLayout L;
  if (!setk::batch_layout(b.empty() ? extra->d.type : b[0].d.type, items, nb, &L)) return ~size_t(0);
  return L.block_bytes;
}

void Executor::finish_job(Slot& s, const JobRec& j, int32_t dev_status, uint64_t t) {
  int32_t st = dev_status;
  if (st == SET_OK) {
    st = check_trailer(s, j);
    if (st == -1000) {
      canary_errors_.fetch_add(1, std::memory_order_relaxed);
      st = SET_EDEVICE;
    }
  }
  lat_.record(t > j.t_submit_ns ? t - j.t_submit_ns : 0);
  if (s.t_dispatch_ns) {
    queue_ns_.fetch_add(s.t_dispatch_ns > j.t_submit_ns ? s.t_dispatch_ns - j.t_submit_ns : 0,
                        std::memory_order_relaxed);
    service_ns_.fetch_add(t > s.t_dispatch_ns ? t - s.t_dispatch_ns : 0, std::memory_order_relaxed);
    timed_jobs_.fetch_add(1, std::memory_order_relaxed);
  }
  if (st != SET_OK) c_failed_.fetch_add(1, std::memory_order_relaxed);
  if (j.d.status) *j.d.status = st;
}

// Algorithm 3: ++c_done (per job of the slot), return the slot to W_pool, wake one dispatcher.
void Executor::on_complete(Slot& s, int32_t dev_status) {
  const uint64_t t = now_ns();
  if (cfg_.stamps && s.stamps && dev_status == SET_OK && s.stamp_nk > 0) {
    // per-job stage order: every kernel started after each kernel it depends on had finished
    bool ok = true;
    for (int k = 0; k < s.stamp_nk; ++k) {
      const uint64_t entry = s.stamps[2 * k], exit = s.stamps[2 * k + 1];
      if (entry == 0 || exit == 0 || entry > exit) ok = false;
      for (int q = 0; q < k; ++q)
        if ((s.stamp_deps[k] >> q) & 1u) ok = ok && s.stamps[2 * q + 1] < entry;
    }
    if (!ok) {
      order_errors_.fetch_add(s.batch.empty() ? 1 : s.batch.size(), std::memory_order_relaxed);
      dev_status = SET_EDEVICE;
    }
  }
  uint64_t n = 1;
  if (s.batch.empty()) {
    finish_job(s, s.job, dev_status, t);
  } else {
    for (const auto& j : s.batch) finish_job(s, j, dev_status, t);
    n = s.batch.size();
  }
  uint64_t last = t_last_ns_.load(std::memory_order_relaxed);
  while (t > last && !t_last_ns_.compare_exchange_weak(last, t)) {
  }
  s.gen += 1;
  if (s.job_mem) {
    arena_.free(s.job_mem, s.job_mem_bytes);
    s.job_mem = nullptr;
    mem_sig_.notify(1);
  }
  const uint64_t d = c_done_.fetch_add(n) + n;
  free_->push(s.index);  // nothing of `s` is touched after this point
  free_sig_.notify(1);
  if (d >= done_target_.load()) done_sig_.notify_all();
}

set_status Executor::wait_all(int64_t timeout_us) {
  const uint64_t t_end = timeout_us < 0 ? ~0ull : now_ns() + (uint64_t)timeout_us * 1000ull;
  for (;;) {
    const uint32_t seen = done_sig_.load();
    const uint64_t target = c_submitted_.load();
    uint64_t cur = done_target_.load();
    while (target < cur && !done_target_.compare_exchange_weak(cur, target)) {
    }
    if (c_done_.load() >= target) {
      done_target_.store(~0ull);
      return (set_status)sticky_.load();
    }
    const uint64_t now = now_ns();
    if (now >= t_end) return SET_ETIMEDOUT;
    const uint64_t rem = t_end - now;
    done_sig_.wait(seen, rem > 100000000ull ? 100000000ll : (int64_t)rem);
  }
}

void Executor::stats(set_stats_t* s) const {
  std::memset(s, 0, sizeof *s);
  s->submitted = c_submitted_.load() - stat_base_submitted_.load();
  s->completed = c_done_.load() - stat_base_done_.load();
  s->failed = c_failed_.load() - stat_base_failed_.load();
  s->steals = steals_.load();
  s->updates = updates_.load();
  s->canary_errors = canary_errors_.load();
  const uint64_t t0 = t_first_ns_.load(), t1 = t_last_ns_.load();
  s->elapsed_s = (t0 && t1 > t0) ? (double)(t1 - t0) * 1e-9 : 0.0;
  s->jobs_per_s = s->elapsed_s > 0 ? (double)s->completed / s->elapsed_s : 0.0;
  s->p50_us = lat_.quantile(0.50) * 1e-3;
  s->p99_us = lat_.quantile(0.99) * 1e-3;
  s->max_us = lat_.max() * 1e-3;
  const uint64_t nl = launched_.load();
  s->mean_update_us = nl ? (double)update_ns_.load() * 1e-3 / (double)nl : 0.0;
  s->mean_launch_us = nl ? (double)launch_ns_.load() * 1e-3 / (double)nl : 0.0;
  s->mem_waits = mem_waits_.load();
  s->order_errors = order_errors_.load();
  s->arena_peak_bytes = use_arena_ ? const_cast<BuddyArena&>(arena_).peak() : 0;
  const uint64_t nt = timed_jobs_.load();
  s->mean_queue_us = nt ? (double)queue_ns_.load() * 1e-3 / (double)nt : 0.0;
  s->mean_service_us = nt ? (double)service_ns_.load() * 1e-3 / (double)nt : 0.0;
  double gap = 0.0;
  s->mean_kernel_gap_us = last_trace_gap(t_reset_ns_.load(), &gap) ? gap : std::nan("");
}

void Executor::reset_stats() {
  stat_base_submitted_.store(c_submitted_.load());
  stat_base_done_.store(c_done_.load());
  stat_base_failed_.store(c_failed_.load());
  steals_.store(0);
  updates_.store(0);
  canary_errors_.store(0);
  update_ns_.store(0);
  launch_ns_.store(0);
  launched_.store(0);
  mem_waits_.store(0);
  queue_ns_.store(0);
  service_ns_.store(0);
  timed_jobs_.store(0);
  order_errors_.store(0);
  t_first_ns_.store(0);
  t_reset_ns_.store(now_ns());
  t_last_ns_.store(0);
  lat_.reset();
}

set_status Executor::run_baseline(int kind, const set_job_desc* jobs, size_t n, set_stats_t* out) {
  if (!jobs || !out) return SET_EINVAL;
  if (io_maps_in(cfg_.io_mode) || io_maps_out(cfg_.io_mode))
    return fail(SET_EINVAL, "baselines copy with cudaMemcpyAsync: use SET_IO_HOST");
  if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
  const set_status w = wait_all(60 * 1000000ll);
  if (w != SET_OK) return w;
  std::vector<JobRec> recs(n);
  std::string why;
  for (size_t i = 0; i < n; ++i) {
    const set_status v = validate(jobs[i], &why);
    if (v != SET_OK) return fail(v, why);
    recs[i].d = jobs[i];
    recs[i].id = c_next_.fetch_add(1);
  }
  LogHist* lat = new LogHist();
  LaunchCost cost;
  uint64_t t0 = 0, t1 = 0;
  std::string e;
  for (auto& s : slots_) s.quiet.store(true);
  const set_status st =
      dev_->run_baseline(kind, recs.data(), n, slots_, use_arena_ ? &arena_ : nullptr, lat, &cost, &t0, &t1, &e);
  for (auto& s : slots_) s.quiet.store(false);
  std::memset(out, 0, sizeof *out);
  if (st == SET_OK) {
    out->submitted = out->completed = n;
    out->updates = cost.updates;
    out->elapsed_s = (double)(t1 - t0) * 1e-9;
    out->jobs_per_s = out->elapsed_s > 0 ? (double)n / out->elapsed_s : 0.0;
    out->p50_us = lat->quantile(0.50) * 1e-3;
    out->p99_us = lat->quantile(0.99) * 1e-3;
    out->max_us = lat->max() * 1e-3;
    out->mean_update_us = n ? (double)cost.update_ns * 1e-3 / (double)n : 0.0;
    out->mean_launch_us = n ? (double)cost.launch_ns * 1e-3 / (double)n : 0.0;
  } else {
    fail(st, e);
  }
  delete lat;
  return st;
}

// Request loop of the serving form: arrivals at start + arrival_ns[i].  Under SET the jobs enter
// through Algorithm 1 as they arrive and overlap with the ones already on the device; under the
// batch-synchronous baseline the same arrivals are batched by what has arrived.
set_status Executor::serve(int mode, const set_job_desc* jobs, const uint64_t* arrival_ns, size_t n, set_stats_t* out) {
  if (!jobs || !arrival_ns || !out || n == 0) return SET_EINVAL;
  for (size_t i = 1; i < n; ++i)
    if (arrival_ns[i] < arrival_ns[i - 1]) return fail(SET_EINVAL, "arrival times must be ascending");
  const set_status w = wait_all(60 * 1000000ll);
  if (w != SET_OK) return w;
  const uint64_t t0 = now_ns() + 1000000ull;  // first arrival 1 ms from now
  if (mode == SET_SERVE_BATCH_SYNC) {
    std::vector<set_job_desc> d(jobs, jobs + n);
    for (size_t i = 0; i < n; ++i) d[i].t_arrival_ns = t0 + arrival_ns[i];
    return run_baseline(SET_BASE_BATCH_SYNC, d.data(), n, out);
  }
  if (mode != SET_SERVE_SET) return SET_EINVAL;
  reset_stats();
  for (size_t i = 0; i < n; ++i) {
    const uint64_t target = t0 + arrival_ns[i];
    wait_until_ns(target);
    set_job_desc d = jobs[i];
    d.t_arrival_ns = target;
    d.flags &= ~SET_F_NONBLOCK;
    const set_status st = submit(&d, nullptr);
    if (st != SET_OK) return st;
  }
  const set_status st = wait_all(600 * 1000000ll);
  stats(out);
  if (out->elapsed_s > 0) out->jobs_per_s = (double)out->completed / out->elapsed_s;
  return st;
}

set_status Executor::autotune(uint32_t type, const set_job_desc* sample, size_t n, set_tune_result* out) {
  if (!sample || !out || n == 0 || !setk::batchable(type)) return SET_EINVAL;
  const set_status w = wait_all(60 * 1000000ll);
  if (w != SET_OK) return w;
  std::vector<JobRec> recs(n);
  std::string why;
  for (size_t i = 0; i < n; ++i) {
    if (sample[i].type != type) return fail(SET_EINVAL, "autotune: sample jobs must all have the given type");
    const set_status v = validate(sample[i], &why);
    if (v != SET_OK) return fail(v, why);
    recs[i].d = sample[i];
    recs[i].id = c_next_.fetch_add(1);
  }
  std::string e;
  for (auto& s : slots_) s.quiet.store(true);
  const set_status st = dev_->autotune(type, recs.data(), n, cfg_.batch_max, out, &e);
  for (auto& s : slots_) s.quiet.store(false);
  if (st != SET_OK) return fail(st, e);
  batch_limit_.store(out->batch_max);
  return SET_OK;
}

}  // namespace setrt
