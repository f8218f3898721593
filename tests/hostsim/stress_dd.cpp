// stress_dd.cpp -- TEST DRIVER: submitter threads against the device-dispatch lanes on the
// simulated backend; run under ThreadSanitizer or AddressSanitizer.  Exit 0 when every job
// completed exactly once with its own trailer and the counters agree.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "set.h"

int main(int argc, char** argv) {
  const int njobs = argc > 1 ? std::atoi(argv[1]) : 20000;
  const int nthreads = 4;
  set_dd_config cfg;
  set_dd_config_default(&cfg);
  cfg.num_lanes = argc > 2 ? std::atoi(argv[2]) : 5;
  cfg.ring_depth = argc > 3 ? std::atoi(argv[3]) : 4;
  cfg.idle_us = argc > 4 ? std::atoi(argv[4]) : 200;  // short: loops end and relaunch often
  set_dd* dd = nullptr;
  if (set_dd_create(&cfg, &dd) != SET_OK) {
    std::fprintf(stderr, "create failed: %s\n", set_dd_last_error(nullptr));
    return 2;
  }
  const uint32_t dims[4] = {4096, 0, 0, 0};
  const size_t in_b = set_job_in_bytes(SET_JOB_SAXPY_SCAN_MAX, dims);
  const size_t out_b = set_job_out_bytes(SET_JOB_SAXPY_SCAN_MAX, dims);
  std::vector<uint8_t> in(in_b + 16, 1);
  std::vector<std::vector<uint8_t>> outs(njobs, std::vector<uint8_t>(out_b + 16, 0));
  std::vector<int32_t> status(njobs, 99);
  std::vector<uint64_t> ids(njobs, ~0ull);
  std::vector<std::thread> th;
  std::atomic<int> errors{0};
  // threads 0 and 1 submit one job at a time (ids recorded), threads 2 and 3 their shares with
  // set_dd_submit_many in chunks of 1..19 jobs (groups of up to 8 per lane; ids then come from the
  // trailers, checked for uniqueness below)
  auto desc = [&](int j) {
    set_job_desc d;
    std::memset(&d, 0, sizeof d);
    d.type = SET_JOB_SAXPY_SCAN_MAX;
    std::memcpy(d.dims, dims, sizeof dims);
    d.in = in.data();
    d.in_bytes = in_b;
    d.out = outs[j].data();
    d.out_bytes = out_b;
    d.status = &status[j];
    return d;
  };
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      const int lo = (int)((int64_t)njobs * t / nthreads), hi = (int)((int64_t)njobs * (t + 1) / nthreads);
      if (t < 2) {
        for (int j = lo; j < hi; ++j) {
          if (j % 97 == 3) {  // a pause now and then: idle loops end and are relaunched
            std::this_thread::sleep_for(std::chrono::microseconds(400));
          }
          set_job_desc d = desc(j);
          if (set_dd_submit(dd, &d, &ids[j]) != SET_OK) errors++;
        }
        return;
      }
      std::vector<set_job_desc> ds;
      for (int j = lo; j < hi;) {
        const int k = std::min(hi - j, 1 + (j * 7 + t) % 19);
        ds.clear();
        for (int q = 0; q < k; ++q) ds.push_back(desc(j + q));
        size_t done = 0;
        if (set_dd_submit_many(dd, ds.data(), ds.size(), nullptr, &done) != SET_OK || done != ds.size()) errors++;
        if (j % 11 == 5) std::this_thread::sleep_for(std::chrono::microseconds(300));
        j += k;
      }
    });
  for (auto& x : th) x.join();
  if (set_dd_wait_all(dd, 120 * 1000000ll) != SET_OK) {
    std::fprintf(stderr, "wait_all failed: %s\n", set_dd_last_error(dd));
    return 3;
  }
  set_stats_t st;
  uint64_t launches = 0;
  set_dd_stats(dd, &st, &launches);
  int bad = errors.load();
  std::vector<uint64_t> seen;
  for (int j = 0; j < njobs; ++j) {
    set_trailer t;
    std::memcpy(&t, outs[j].data() + out_b - sizeof t, sizeof t);
    const bool own = ids[j] == ~0ull || t.job_id == ids[j];  // ids known for threads 0 and 1
    if (status[j] != SET_OK || !own || (t.word >> 16) != SET_TRAILER_MAGIC) ++bad;
    seen.push_back(t.job_id);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) ++bad;  // every id once
  if (st.completed != (uint64_t)njobs || st.submitted != (uint64_t)njobs || st.failed || st.canary_errors) ++bad;
  if (set_dd_destroy(dd) != SET_OK) ++bad;
  std::printf("jobs %d bad %d launches %llu\n", njobs, bad, (unsigned long long)launches);
  return bad ? 1 : 0;
}
