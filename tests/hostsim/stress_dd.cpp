// stress_dd.cpp -- TEST DRIVER: submitter threads against the device-dispatch lanes on the
// simulated backend; run under ThreadSanitizer or AddressSanitizer.  Exit 0 when every job
// completed exactly once with its own trailer and the counters agree.
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
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      for (int j = t; j < njobs; j += nthreads) {
        set_job_desc d;
        std::memset(&d, 0, sizeof d);
        d.type = SET_JOB_SAXPY_SCAN_MAX;
        std::memcpy(d.dims, dims, sizeof dims);
        d.in = in.data();
        d.in_bytes = in_b;
        d.out = outs[j].data();
        d.out_bytes = out_b;
        d.status = &status[j];
        if (j % 97 == 3) {  // a pause now and then: idle loops end and are relaunched
          std::this_thread::sleep_for(std::chrono::microseconds(400));
        }
        if (set_dd_submit(dd, &d, &ids[j]) != SET_OK) errors++;
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
  for (int j = 0; j < njobs; ++j) {
    set_trailer t;
    std::memcpy(&t, outs[j].data() + out_b - sizeof t, sizeof t);
    if (status[j] != SET_OK || t.job_id != ids[j] || (t.word >> 16) != SET_TRAILER_MAGIC) ++bad;
  }
  if (st.completed != (uint64_t)njobs || st.submitted != (uint64_t)njobs || st.failed || st.canary_errors) ++bad;
  if (set_dd_destroy(dd) != SET_OK) ++bad;
  std::printf("jobs %d bad %d launches %llu\n", njobs, bad, (unsigned long long)launches);
  return bad ? 1 : 0;
}
