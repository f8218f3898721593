// sync.h -- lock-free queues and futex-backed signals for the executor's host side.
//
// MpmcRing is Vyukov's bounded multi-producer / multi-consumer queue (a ring of cells, each with
// a sequence number; push and pop claim a position with one CAS).  It holds the per-lane job
// queues Q_i and the free-slot pool W_pool (Sec. 4.2).  Signal is a sequence word that waiters
// sleep on with futex(2) instead of polling; notifiers bump it and only enter the kernel when
// someone is asleep.  Waiters read the sequence, re-check their condition, then sleep only if the
// sequence is unchanged, so no wake-up is lost.
#pragma once

#include <linux/futex.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <atomic>
#include <cerrno>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <ctime>
#include <memory>
#include <new>

namespace setrt {

inline uint64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

// Request loops: returns at `target` (CLOCK_MONOTONIC ns).  Sleeps while more than 150 us remain,
// then spins, so a loop waiting for sparse arrivals does not hold a core.
inline void wait_until_ns(uint64_t target) {
  for (uint64_t t = now_ns(); t + 150000ull < target; t = now_ns()) {
    const uint64_t d = target - t - 100000ull;
    timespec ts;
    ts.tv_sec = (time_t)(d / 1000000000ull);
    ts.tv_nsec = (long)(d % 1000000000ull);
    nanosleep(&ts, nullptr);
  }
  while (now_ns() < target) {
  }
}

class Signal {
 public:
  uint32_t load() const { return seq_.load(std::memory_order_seq_cst); }

  void notify(int n) {
    seq_.fetch_add(1, std::memory_order_seq_cst);
    if (waiters_.load(std::memory_order_seq_cst) > 0) futex_wake(n);
  }
  void notify_all() { notify(INT_MAX); }

  // Sleeps while the sequence still equals `seen`.  timeout_ns < 0 waits without limit.
  // Returns false only when the timeout expired.
  bool wait(uint32_t seen, int64_t timeout_ns) {
    waiters_.fetch_add(1, std::memory_order_seq_cst);
    bool ok = true;
    if (seq_.load(std::memory_order_seq_cst) == seen) {
      timespec ts, *tsp = nullptr;
      if (timeout_ns >= 0) {
        ts.tv_sec = timeout_ns / 1000000000;
        ts.tv_nsec = timeout_ns % 1000000000;
        tsp = &ts;
      }
      const long r = syscall(SYS_futex, reinterpret_cast<uint32_t*>(&seq_), FUTEX_WAIT_PRIVATE, seen, tsp,
                             nullptr, 0);
      if (r != 0 && errno == ETIMEDOUT) ok = false;
    }
    waiters_.fetch_sub(1, std::memory_order_seq_cst);
    return ok;
  }

 private:
  void futex_wake(int n) {
    syscall(SYS_futex, reinterpret_cast<uint32_t*>(&seq_), FUTEX_WAKE_PRIVATE, n, nullptr, nullptr, 0);
  }
  alignas(64) std::atomic<uint32_t> seq_{0};
  alignas(64) std::atomic<int32_t> waiters_{0};
};
static_assert(sizeof(std::atomic<uint32_t>) == 4, "futex word must be 32 bits");

inline size_t next_pow2(size_t v) {
  size_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

template <class T>
class MpmcRing {
 public:
  explicit MpmcRing(size_t capacity) : cap_(next_pow2(capacity < 2 ? 2 : capacity)), mask_(cap_ - 1) {
    cells_.reset(new Cell[cap_]);
    for (size_t i = 0; i < cap_; ++i) cells_[i].seq.store(i, std::memory_order_relaxed);
  }

  bool push(const T& v) {
    size_t pos = enq_.load(std::memory_order_relaxed);
    for (;;) {
      Cell& c = cells_[pos & mask_];
      const size_t seq = c.seq.load(std::memory_order_acquire);
      const intptr_t dif = (intptr_t)seq - (intptr_t)pos;
      if (dif == 0) {
        if (enq_.compare_exchange_weak(pos, pos + 1, std::memory_order_relaxed)) {
          c.val = v;
          c.seq.store(pos + 1, std::memory_order_release);
          return true;
        }
      } else if (dif < 0) {
        return false;  // full
      } else {
        pos = enq_.load(std::memory_order_relaxed);
      }
    }
  }

  bool pop(T& v) {
    size_t pos = deq_.load(std::memory_order_relaxed);
    for (;;) {
      Cell& c = cells_[pos & mask_];
      const size_t seq = c.seq.load(std::memory_order_acquire);
      const intptr_t dif = (intptr_t)seq - (intptr_t)(pos + 1);
      if (dif == 0) {
        if (deq_.compare_exchange_weak(pos, pos + 1, std::memory_order_relaxed)) {
          v = c.val;
          c.seq.store(pos + mask_ + 1, std::memory_order_release);
          return true;
        }
      } else if (dif < 0) {
        return false;  // empty
      } else {
        pos = deq_.load(std::memory_order_relaxed);
      }
    }
  }

  size_t size_approx() const {
    const size_t e = enq_.load(std::memory_order_relaxed), d = deq_.load(std::memory_order_relaxed);
    return e > d ? e - d : 0;
  }
  size_t capacity() const { return cap_; }

 private:
  struct alignas(64) Cell {
    std::atomic<size_t> seq;
    T val;
  };
  const size_t cap_, mask_;
  std::unique_ptr<Cell[]> cells_;
  alignas(64) std::atomic<size_t> enq_{0};
  alignas(64) std::atomic<size_t> deq_{0};
};

// Log-bucketed latency histogram: 64 sub-buckets per octave (about 1.1 % resolution).
class LogHist {
 public:
  static constexpr int kSub = 64, kOct = 44, kN = kSub * kOct;
  void record(uint64_t ns) {
    counts_[index(ns)].fetch_add(1, std::memory_order_relaxed);
    uint64_t m = max_.load(std::memory_order_relaxed);
    while (ns > m && !max_.compare_exchange_weak(m, ns, std::memory_order_relaxed)) {
    }
  }
  void reset() {
    for (auto& c : counts_) c.store(0, std::memory_order_relaxed);
    max_.store(0, std::memory_order_relaxed);
  }
  // Value (ns) at quantile q in [0, 1]: midpoint of the bucket that holds it.
  double quantile(double q) const {
    uint64_t total = 0;
    for (const auto& c : counts_) total += c.load(std::memory_order_relaxed);
    if (total == 0) return 0.0;
    const uint64_t rank = (uint64_t)(q * (double)(total - 1));
    uint64_t run = 0;
    for (int i = 0; i < kN; ++i) {
      run += counts_[i].load(std::memory_order_relaxed);
      if (run > rank) return midpoint(i);
    }
    return (double)max_.load();
  }
  double max() const { return (double)max_.load(std::memory_order_relaxed); }

 private:
  static int index(uint64_t v) {
    if (v < (uint64_t)kSub) return (int)v;
    const int e = 63 - __builtin_clzll(v);  // v in [2^e, 2^(e+1)), e >= 6
    const int sub = (int)((v >> (e - 6)) & (kSub - 1));
    const int i = (e - 5) * kSub + sub;
    return i < kN ? i : kN - 1;
  }
  static double midpoint(int i) {
    if (i < kSub) return (double)i;
    const int e = i / kSub + 5, sub = i % kSub;
    const double lo = (double)(((uint64_t)kSub + sub) << (e - 6));
    return lo + (double)(1ull << (e - 6)) * 0.5;
  }
  std::atomic<uint64_t> counts_[kN] = {};
  std::atomic<uint64_t> max_{0};
};

}  // namespace setrt
