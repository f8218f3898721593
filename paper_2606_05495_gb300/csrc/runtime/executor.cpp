// executor.cpp -- queues, free-slot pool, dispatch workers and the completion path of the SET
// executor (Sec. 4.2; Algorithm 1 = submit, Algorithm 2 = worker_main / find_job,
// Algorithm 3 = on_complete).  Device specifics live behind the Device interface.
#include "executor.h"

#include <algorithm>
#include <cstring>

#include "layout.h"

namespace setrt {

namespace {

void normalize(set_config& c) {
  if (c.ring_depth <= 0) c.ring_depth = 2;
  if (c.queue_capacity <= 0) c.queue_capacity = 4;
  if (c.steal != 0) c.steal = 1;
  if (c.type_mask == 0) c.type_mask = ~0u;
  if (c.drain_timeout_ms <= 0) c.drain_timeout_ms = 30000;
  if (c.spin_us < 0) c.spin_us = 0;
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

set_status Executor::create(const set_config& cfg_in, Executor** out, std::string* err) {
  set_config cfg = cfg_in;
  normalize(cfg);
  if (!out || cfg.num_streams < 1 || cfg.num_streams > 1024 || cfg.num_workers < 1 || cfg.num_workers > 256 ||
      cfg.ring_depth > 64 || cfg.queue_capacity > (1 << 20) || cfg.slot_bytes < 4096 ||
      (cfg.io_mode != SET_IO_HOST && cfg.io_mode != SET_IO_DEVICE)) {
    *err = "invalid set_config (num_streams 1..1024, num_workers 1..256, ring_depth <= 64, slot_bytes >= 4096)";
    return SET_EINVAL;
  }
  std::unique_ptr<Executor> ex(new Executor(cfg));
  const uint32_t L = (uint32_t)cfg.num_streams, R = (uint32_t)cfg.ring_depth;
  ex->slots_.resize((size_t)L * R);
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
  for (uint32_t i = 0; i < L; ++i) ex->queues_.emplace_back(new MpmcRing<JobRec>((size_t)cfg.queue_capacity));
  ex->free_.reset(new MpmcRing<uint32_t>((size_t)L * R));
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
  const size_t ctl = setk::slot_control_bytes(cfg_.slot_bytes);
  setk::place_job(&L, ctl);
  if (L.end > cfg_.slot_bytes || setk::control_offset(d.type) + L.persist_bytes > ctl) {
    *why = "job does not fit the slot (slot_bytes too small)";
    return SET_ENOMEM;
  }
  return SET_OK;
}

// Algorithm 1 (job submitter): claim an id, push to the shortest queue that is not full.
set_status Executor::submit(const set_job_desc* d, uint64_t* id_out) {
  if (!d) return SET_EINVAL;
  if (stop_.load()) return SET_ESHUTDOWN;
  if (sticky_.load() != SET_OK) return (set_status)sticky_.load();
  std::string why;
  const set_status v = validate(*d, &why);
  if (v != SET_OK) return fail(v, why);
  JobRec j;
  j.d = *d;
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

// Algorithm 2, dispatcher loop: pop a free slot (W_pool), FindJob, LaunchJob.  Waiting is a
// futex sleep on the pool / submit signals, never a poll.
void Executor::worker_main(int) {
  const uint64_t spin_ns = (uint64_t)cfg_.spin_us * 1000ull;
  for (;;) {
    uint32_t tok = 0;
    for (;;) {
      const uint32_t seen = free_sig_.load();
      if (stop_.load()) return;
      if (free_->pop(tok)) break;
      if (spin_until([&] { return free_sig_.load() != seen || stop_.load(); }, spin_ns)) continue;
      free_sig_.wait(seen, -1);
    }
    Slot& s = slots_[tok];
    JobRec j;
    bool stolen = false, got = false;
    for (;;) {
      const uint32_t seen = job_sig_.load();
      if (find_job(s.lane, j, stolen)) {
        got = true;
        break;
      }
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
      if (stop_.load() && cfg_.steal) {
        free_->push(tok);
        return;
      }
      continue;
    }
    space_sig_.notify(1);
    if (stolen) steals_.fetch_add(1, std::memory_order_relaxed);
    s.job = j;
    if (sticky_.load() != SET_OK) {
      on_complete(s, sticky_.load());
      continue;
    }
    LaunchCost cost;
    std::string e;
    const set_status st = dev_->launch(s, &cost, &e);
    updates_.fetch_add(cost.updates, std::memory_order_relaxed);
    update_ns_.fetch_add(cost.update_ns, std::memory_order_relaxed);
    launch_ns_.fetch_add(cost.launch_ns, std::memory_order_relaxed);
    launched_.fetch_add(1, std::memory_order_relaxed);
    if (st != SET_OK) {
      fail(st, e);
      on_complete(s, st);
    }
  }
}

int32_t Executor::check_trailer(const Slot& s) const {
  if (cfg_.io_mode != SET_IO_HOST) return SET_OK;
  set_trailer t;
  std::memcpy(&t, static_cast<const uint8_t*>(s.job.d.out) + s.job.d.out_bytes - sizeof(set_trailer), sizeof t);
  if (t.job_id != s.job.id || t.slot_gen != s.gen || (t.word >> 16) != SET_TRAILER_MAGIC) return -1000;
  if (t.word & 0xFFFFu) return SET_EDEVICE;
  return SET_OK;
}

// Algorithm 3: ++c_done, return the slot to W_pool, wake one dispatcher.
void Executor::on_complete(Slot& s, int32_t dev_status) {
  int32_t st = dev_status;
  if (st == SET_OK) {
    st = check_trailer(s);
    if (st == -1000) {
      canary_errors_.fetch_add(1, std::memory_order_relaxed);
      st = SET_EDEVICE;
    }
  }
  const uint64_t t = now_ns();
  lat_.record(t - s.job.t_submit_ns);
  uint64_t last = t_last_ns_.load(std::memory_order_relaxed);
  while (t > last && !t_last_ns_.compare_exchange_weak(last, t)) {
  }
  if (st != SET_OK) c_failed_.fetch_add(1, std::memory_order_relaxed);
  if (s.job.d.status) *s.job.d.status = st;
  s.gen += 1;
  const uint64_t d = c_done_.fetch_add(1) + 1;
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
  t_first_ns_.store(0);
  t_last_ns_.store(0);
  lat_.reset();
}

set_status Executor::run_baseline(int kind, const set_job_desc* jobs, size_t n, set_stats_t* out) {
  if (!jobs || !out) return SET_EINVAL;
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
  const set_status st = dev_->run_baseline(kind, recs.data(), n, slots_, lat, &cost, &t0, &t1, &e);
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

}  // namespace setrt
