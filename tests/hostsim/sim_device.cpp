// sim_device.cpp -- TEST DOUBLE of the executor's Device: no GPU, no arithmetic.
//
// Compiled only into the test library libset_hostsim.so (never into libset.so).  A "launch" is
// queued to its lane's host thread, which waits a seeded random delay (the job's "device
// time"), writes the job's trailer {job id, slot generation, magic} into the caller's output
// buffer (the only byte it writes) and hands the slot to a single callback thread that calls
// Executor::on_complete, as the CUDA driver's host-function thread does.  Lane threads run
// their launches in FIFO order like a stream.
//
// Fault injection (environment, read at context creation):
//   SET_SIM_DELAY_US=lo,hi   per-launch delay range (default 5,50)
//   SET_SIM_DROP_EVERY=k     every k-th launch never completes (a lost callback)
//   SET_SIM_BADGEN_EVERY=k   every k-th launch writes a wrong slot generation (stale slot)
//   SET_SIM_FAIL_EVERY=k     every k-th launch fails with SET_ECUDA at launch time
//   SET_SIM_SLOW_LANE=i,f    lane i's delays are f times longer (a lane that falls behind)
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "executor.h"
#include "layout.h"

namespace setrt {
namespace {

long env_long(const char* name, long dflt) {
  const char* v = std::getenv(name);
  return v ? std::strtol(v, nullptr, 10) : dflt;
}

class SimDevice final : public Device {
 public:
  explicit SimDevice(const set_config&) {}
  ~SimDevice() override { stop(); }

  set_status init(const set_config& cfg, std::vector<Slot>& slots, std::string*) override {
    const char* d = std::getenv("SET_SIM_DELAY_US");
    if (d) std::sscanf(d, "%ld,%ld", &lo_, &hi_);
    drop_ = env_long("SET_SIM_DROP_EVERY", 0);
    badgen_ = env_long("SET_SIM_BADGEN_EVERY", 0);
    fail_ = env_long("SET_SIM_FAIL_EVERY", 0);
    if (const char* sl = std::getenv("SET_SIM_SLOW_LANE")) std::sscanf(sl, "%ld,%ld", &slow_lane_, &slow_factor_);
    for (auto& s : slots) s.bytes = cfg.slot_bytes;
    dropped_.assign(slots.size(), 0);
    // arena mode: host bytes stand in for the device range (the simulation never touches them)
    if (cfg.arena_bytes) arena_.resize(cfg.arena_bytes > (64u << 20) ? (64u << 20) : cfg.arena_bytes);
    for (int i = 0; i < cfg.num_streams; ++i) lanes_.emplace_back(new Lane);
    for (int i = 0; i < cfg.num_streams; ++i) lanes_[i]->th = std::thread(&SimDevice::lane_main, this, i);
    cb_th_ = std::thread(&SimDevice::cb_main, this);
    return SET_OK;
  }

  bool supports(uint32_t type) const override { return type >= 1 && type <= SET_NUM_JOB_TYPES; }
  bool io_accessible(const void*) const override { return true; }
  bool io_device(const void*) const override { return true; }

  set_status launch(Slot& s, bool callback, LaunchCost* cost, std::string* err) override {
    const uint64_t k = ++launches_;
    cost->updates += 3;
    if (fail_ && k % fail_ == 0) {
      *err = "simulated launch failure";
      return SET_ECUDA;
    }
    enqueue(&s, k, false);
    if (callback) enqueue(&s, 0, true);
    return SET_OK;
  }

  set_status launch_batch(Slot& s, bool callback, LaunchCost* cost, std::string* err) override {
    return launch(s, callback, cost, err);
  }

  set_status prepare(Slot&, LaunchCost* cost, std::string*) override {
    cost->updates += 3;
    return SET_OK;
  }

  set_status launch_bound(Slot& s, bool callback, LaunchCost*, std::string* err) override {
    const uint64_t k = ++launches_;
    if (fail_ && k % fail_ == 0) {
      *err = "simulated launch failure";
      return SET_ECUDA;
    }
    enqueue(&s, k, false);
    if (callback) enqueue(&s, 0, true);
    return SET_OK;
  }

  set_status autotune(uint32_t, const JobRec*, size_t, int, set_tune_result*, std::string* err) override {
    *err = "the autotuner needs the CUDA device";
    return SET_EINVAL;
  }

  set_status attach_callback(Slot& s, std::string*) override {
    enqueue(&s, 0, true);
    return SET_OK;
  }

  void drain() override {
    for (;;) {
      bool idle = true;
      for (auto& L : lanes_) {
        std::lock_guard<std::mutex> g(L->mu);
        idle = idle && L->q.empty() && !L->busy;
      }
      {
        std::lock_guard<std::mutex> g(cb_mu_);
        idle = idle && cb_q_.empty() && !cb_busy_;
      }
      if (idle) return;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }

  uint8_t* arena_base() override { return arena_.data(); }
  void thread_init() override {}

  set_status run_baseline(int, const JobRec*, size_t, std::vector<Slot>&, BuddyArena*, LogHist*, LaunchCost*,
                          uint64_t*, uint64_t*, std::string* err) override {
    *err = "baselines need the CUDA device";
    return SET_EINVAL;
  }

 private:
  struct Item {
    Slot* s;
    uint64_t k;
    bool cb;  // a completion callback for the group ending at s (runs after earlier items)
  };

  void enqueue(Slot* s, uint64_t k, bool cb) {
    Lane& L = *lanes_[s->lane];
    {
      std::lock_guard<std::mutex> g(L.mu);
      L.q.push_back({s, k, cb});
    }
    L.cv.notify_one();
  }
  struct Lane {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Item> q;
    bool busy = false;
    std::thread th;
  };

  void lane_main(int i) {
    Lane& L = *lanes_[i];
    std::mt19937_64 rng(1234 + i);
    for (;;) {
      Item it;
      {
        std::unique_lock<std::mutex> g(L.mu);
        L.cv.wait(g, [&] { return stop_ || !L.q.empty(); });
        if (stop_ && L.q.empty()) return;
        it = L.q.front();
        L.q.pop_front();
        L.busy = true;
      }
      Slot& s = *it.s;
      if (it.cb) {
        // callbacks are the only way slots come back; a dropped one strands its whole group
        if (!dropped_[s.index]) {
          std::lock_guard<std::mutex> g(cb_mu_);
          cb_q_.push_back(&s);
          cb_cv_.notify_one();
        }
      } else {
        const long us = (lo_ + (long)(rng() % (uint64_t)(hi_ - lo_ + 1))) * (i == slow_lane_ ? slow_factor_ : 1);
        std::this_thread::sleep_for(std::chrono::microseconds(us));
        auto write = [&](const JobRec& j) {
          set_trailer t;
          t.job_id = j.id;
          t.slot_gen = (badgen_ && it.k % badgen_ == 0) ? s.gen + 7 : s.gen;
          t.word = SET_TRAILER_MAGIC << 16;
          std::memcpy(static_cast<uint8_t*>(j.d.out) + j.d.out_bytes - sizeof t, &t, sizeof t);
        };
        if (s.batch.empty()) write(s.job);
        for (const auto& j : s.batch) write(j);
        dropped_[s.index] = drop_ && it.k % drop_ == 0;
      }
      std::lock_guard<std::mutex> g(L.mu);
      L.busy = false;
    }
  }

  void cb_main() {
    for (;;) {
      Slot* s;
      {
        std::unique_lock<std::mutex> g(cb_mu_);
        cb_cv_.wait(g, [&] { return stop_ || !cb_q_.empty(); });
        if (stop_ && cb_q_.empty()) return;
        s = cb_q_.front();
        cb_q_.pop_front();
        cb_busy_ = true;
      }
      s->ex->on_complete_group(*s);
      std::lock_guard<std::mutex> g(cb_mu_);
      cb_busy_ = false;
    }
  }

  void stop() {
    {
      std::lock_guard<std::mutex> g(cb_mu_);
      stop_ = true;
    }
    for (auto& L : lanes_) {
      {
        std::lock_guard<std::mutex> g(L->mu);
      }
      L->cv.notify_all();
    }
    cb_cv_.notify_all();
    for (auto& L : lanes_)
      if (L->th.joinable()) L->th.join();
    if (cb_th_.joinable()) cb_th_.join();
  }

  long lo_ = 5, hi_ = 50, drop_ = 0, badgen_ = 0, fail_ = 0, slow_lane_ = -1, slow_factor_ = 1;
  std::vector<uint8_t> arena_;
  std::vector<char> dropped_;  // per slot: its last job "lost" its callback
  std::atomic<uint64_t> launches_{0};
  std::vector<std::unique_ptr<Lane>> lanes_;
  std::mutex cb_mu_;
  std::condition_variable cb_cv_;
  std::deque<Slot*> cb_q_;
  bool cb_busy_ = false;
  std::atomic<bool> stop_{false};
  std::thread cb_th_;
};

}  // namespace

std::unique_ptr<Device> make_device(const set_config& cfg) { return std::unique_ptr<Device>(new SimDevice(cfg)); }

}  // namespace setrt
