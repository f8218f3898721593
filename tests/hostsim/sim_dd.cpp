// sim_dd.cpp -- TEST DOUBLE of the device-dispatch backend (dd_backend.h): no GPU, no arithmetic.
//
// Compiled only into the test library libset_hostsim.so (never into libset.so).  A launch of a
// lane's loop starts a host thread that follows the fetch kernel's protocol on the same memory
// layout: retire the jobs the previous iteration ran (their completion words, then the done
// counter with release order), poll the next ring entry's sequence word with acquire order for at
// most idle_us (or until the stop word is set), take the job -- a blur or scan job together with
// the entries of the same kind directly behind it that are already complete, up to kDdBatch, as
// the fetch kernel does -- and "run" them: wait a seeded random delay and write each trailer {job
// id, lane, magic}, the only bytes of a job it touches.  With no descriptor the loop counts an
// exit (release order)
// and ends; the backend reports the launch ended only after the thread's last access, as a stream
// reports a graph complete.
//
// Fault injection (environment, read at set_dd_create):
//   SET_SIM_DD_DELAY_US=lo,hi     per-job delay range (default 2,20)
//   SET_SIM_DD_BADTRAILER_EVERY=k every k-th job writes a wrong job id (a canary error)
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <random>
#include <thread>
#include <vector>

#include "dd_backend.h"
#include "sync.h"

namespace setrt {
namespace {

std::atomic<uint64_t> g_batched_jobs{0};  // jobs that ran in batches of two or more (all objects)

struct SimLane {
  // state the device keeps across launches (DdLaneDev's fields the protocol uses)
  uint64_t head = 0, cur_first = 0;
  uint32_t cur_count = 0, exits = 0;
  uint64_t cur_job[setk::kDdBatch] = {};
  set_trailer* cur_trailer[setk::kDdBatch] = {};
  std::thread th;
  std::atomic<bool> running{false};
  std::mt19937_64 rng;
};

class SimDdBackend final : public DdBackend {
 public:
  ~SimDdBackend() override { release(false); }

  set_status init(const set_dd_config& cfg, uint32_t depth, std::vector<DdLaneMem>* lanes, std::string*) override {
    cfg_ = cfg;
    depth_ = depth;
    if (const char* d = std::getenv("SET_SIM_DD_DELAY_US")) std::sscanf(d, "%ld,%ld", &lo_, &hi_);
    if (const char* b = std::getenv("SET_SIM_DD_BADTRAILER_EVERY")) bad_every_ = std::strtol(b, nullptr, 10);
    const uint32_t nl = (uint32_t)cfg.num_lanes;
    lanes->assign(nl, DdLaneMem{});
    for (uint32_t i = 0; i < nl; ++i) {
      rings_.emplace_back(new setk::DdEntry[depth]());
      ctls_.emplace_back(new setk::DdCtl[1]());
      cmpls_.emplace_back(new uint32_t[depth]());
      scratch_.emplace_back(new uint8_t[64]());
      (*lanes)[i] = DdLaneMem{rings_[i].get(), ctls_[i].get(), cmpls_[i].get(), scratch_[i].get(), scratch_[i].get()};
      lanes_.emplace_back(new SimLane);
      lanes_[i]->rng.seed(0x5E7Dull * (i + 1));
    }
    return SET_OK;
  }

  bool plan(const set_job_desc&, uint64_t, uint32_t, unsigned char*, uint32_t* args_size) override {
    *args_size = 0;  // the simulated loop needs only the entry's job id and trailer
    return true;
  }
  bool buffer_ok(const void* p, size_t, DdRangeCache*) const override { return p != nullptr; }

  set_status launch(uint32_t lane, std::string*) override {
    SimLane& l = *lanes_[lane];
    if (l.th.joinable()) l.th.join();  // the previous launch has ended (the protocol checked)
    l.running.store(true, std::memory_order_release);
    l.th = std::thread(&SimDdBackend::loop, this, lane);
    return SET_OK;
  }
  int ended(uint32_t lane, std::string*) override { return lanes_[lane]->running.load(std::memory_order_acquire) ? 0 : 1; }
  void bind_thread() override {}
  void release(bool leak) override {
    if (leak) leaked_ = true;
    for (auto& l : lanes_)
      if (l->th.joinable()) l->th.join();  // a simulated loop always ends (bounded poll)
  }

 private:
  void loop(uint32_t lane) {
    SimLane& l = *lanes_[lane];
    setk::DdEntry* ring = rings_[lane].get();
    setk::DdCtl* ctl = ctls_[lane].get();
    uint32_t* cmpl = cmpls_[lane].get();
    const uint32_t mask = depth_ - 1;
    for (;;) {
      for (uint32_t i = 0; i < l.cur_count; ++i) {  // retire the previous batch
        set_trailer t;
        std::memcpy(&t, l.cur_trailer[i], sizeof t);
        uint32_t word = t.word;
        if (t.job_id != l.cur_job[i] || (word >> 16) != SET_TRAILER_MAGIC) word = 0u;
        __atomic_store_n(&cmpl[(l.cur_first - 1 + i) & mask], word, __ATOMIC_RELAXED);
      }
      if (l.cur_count != 0) __atomic_store_n(&ctl->done, l.cur_first + l.cur_count - 1, __ATOMIC_RELEASE);
      l.cur_count = 0;
      const uint64_t want = l.head + 1;
      setk::DdEntry& e = ring[l.head & mask];
      const uint64_t t0 = now_ns();
      bool found = false;
      for (uint32_t it = 0;; ++it) {
        if (__atomic_load_n(&e.seq, __ATOMIC_ACQUIRE) == want) {
          found = true;
          break;
        }
        if (__atomic_load_n(&ctl->stop, __ATOMIC_ACQUIRE) || now_ns() - t0 > (uint64_t)cfg_.idle_us * 1000ull) break;
        if (it > 64) std::this_thread::yield();
      }
      if (!found) {
        l.exits += 1;
        __atomic_store_n(&ctl->exits, l.exits, __ATOMIC_RELEASE);
        break;
      }
      uint32_t count = 1;
      l.cur_job[0] = e.job_id;
      l.cur_trailer[0] = e.trailer;
      if (e.kind == setk::kDdKindScan || e.kind == setk::kDdKindBlur)
        for (; count < setk::kDdBatch; ++count) {
          setk::DdEntry& f = ring[(l.head + count) & mask];
          if (__atomic_load_n(&f.seq, __ATOMIC_ACQUIRE) != want + count || f.kind != e.kind) break;
          l.cur_job[count] = f.job_id;
          l.cur_trailer[count] = f.trailer;
        }
      l.head += count;
      l.cur_first = want;
      l.cur_count = count;
      if (count > 1) g_batched_jobs.fetch_add(count);
      // the jobs: a delay, then their trailers
      const long us = lo_ + (hi_ > lo_ ? (long)(l.rng() % (uint64_t)(hi_ - lo_ + 1)) : 0);
      if (us > 0) std::this_thread::sleep_for(std::chrono::microseconds(us));
      for (uint32_t i = 0; i < count; ++i) {
        const uint64_t k = jobs_.fetch_add(1) + 1;
        set_trailer t;
        t.job_id = (bad_every_ > 0 && k % (uint64_t)bad_every_ == 0) ? l.cur_job[i] + 1000000007ull : l.cur_job[i];
        t.slot_gen = lane;
        t.word = (uint32_t)SET_TRAILER_MAGIC << 16;
        std::memcpy(l.cur_trailer[i], &t, sizeof t);
      }
    }
    l.running.store(false, std::memory_order_release);
  }

  set_dd_config cfg_{};
  uint32_t depth_ = 0;
  long lo_ = 2, hi_ = 20, bad_every_ = 0;
  bool leaked_ = false;
  std::atomic<uint64_t> jobs_{0};
  std::vector<std::unique_ptr<setk::DdEntry[]>> rings_;
  std::vector<std::unique_ptr<setk::DdCtl[]>> ctls_;
  std::vector<std::unique_ptr<uint32_t[]>> cmpls_;
  std::vector<std::unique_ptr<uint8_t[]>> scratch_;
  std::vector<std::unique_ptr<SimLane>> lanes_;
};

}  // namespace

std::unique_ptr<DdBackend> make_dd_backend() { return std::make_unique<SimDdBackend>(); }

}  // namespace setrt

// Test probe: jobs the simulated loops have run in batches of two or more since the library loaded.
extern "C" uint64_t set_sim_dd_batched_jobs() { return setrt::g_batched_jobs.load(); }

// Test probe: DdRangeCache (the per-call memory of accepted allocations) on fixed cases; returns
// the bit mask of the cases that came out wrong (0 = all right).
extern "C" uint32_t set_sim_dd_range_cache_check() {
  uint32_t bad = 0;
  setrt::DdRangeCache c;
  if (c.has(0x1000, 1)) bad |= 1u << 0;  // empty
  c.add(0x1000, 0x2000);
  if (!c.has(0x1000, 0x1000)) bad |= 1u << 1;  // the whole allocation
  if (!c.has(0x1ff0, 0x10)) bad |= 1u << 2;    // ends exactly at its end
  if (c.has(0x1ff0, 0x11)) bad |= 1u << 3;     // one byte past it
  if (c.has(0x0fff, 1)) bad |= 1u << 4;        // starts before it
  if (c.has(0x3000, 0)) bad |= 1u << 5;        // starts past its end (no wrap-around)
  if (c.has(0x2001, 1)) bad |= 1u << 6;
  for (uintptr_t k = 1; k <= 4; ++k) c.add(0x10000 * k, 0x10000 * k + 0x100);  // evicts the first
  if (c.has(0x1000, 1)) bad |= 1u << 7;
  for (uintptr_t k = 1; k <= 4; ++k)
    if (!c.has(0x10000 * k + 0x80, 0x80)) bad |= 1u << 8;
  if (c.n != setrt::DdRangeCache::kN) bad |= 1u << 9;
  return bad;
}
