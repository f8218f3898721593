// stress.cpp -- TEST DRIVER: many submitter threads against the executor on the simulated
// device; run under ThreadSanitizer or AddressSanitizer.  Exit 0 when every job completed
// exactly once with its own trailer and the counters agree.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "set.h"

int main(int argc, char** argv) {
  const int njobs = argc > 1 ? std::atoi(argv[1]) : 20000;
  const int nthreads = 4;
  set_config cfg;
  set_config_default(&cfg);
  cfg.num_streams = 6;
  cfg.num_workers = 5;
  cfg.ring_depth = 2;
  cfg.queue_capacity = 2;
  cfg.slot_bytes = 1 << 20;
  cfg.cb_every = argc > 2 ? std::atoi(argv[2]) : 1;
  cfg.bind_at_submit = argc > 3 ? std::atoi(argv[3]) : 0;
  set_ctx* ctx = nullptr;
  if (set_create_ex(&cfg, &ctx) != SET_OK) {
    std::fprintf(stderr, "create failed: %s\n", set_last_error(nullptr));
    return 2;
  }
  const uint32_t dims[4] = {16, 16, 0, 0};
  const size_t in_b = set_job_in_bytes(SET_JOB_BLUR_HIST, dims), out_b = set_job_out_bytes(SET_JOB_BLUR_HIST, dims);
  std::vector<uint8_t> in(in_b, 1);
  std::vector<std::vector<uint8_t>> outs(njobs, std::vector<uint8_t>(out_b, 0));
  std::vector<int32_t> status(njobs, 99);
  std::vector<uint64_t> ids(njobs, ~0ull);
  std::vector<std::thread> th;
  std::atomic<int> errors{0};
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      for (int j = t; j < njobs; j += nthreads) {
        set_job_desc d;
        std::memset(&d, 0, sizeof d);
        d.type = SET_JOB_BLUR_HIST;
        std::memcpy(d.dims, dims, sizeof dims);
        d.in = in.data();
        d.in_bytes = in_b;
        d.out = outs[j].data();
        d.out_bytes = out_b;
        d.status = &status[j];
        if (set_submit(ctx, &d, &ids[j]) != SET_OK) errors++;
      }
    });
  for (auto& x : th) x.join();
  if (set_wait_all(ctx, 60 * 1000000ll) != SET_OK) {
    std::fprintf(stderr, "wait_all failed\n");
    return 3;
  }
  set_stats_t st;
  set_stats(ctx, &st);
  int bad = errors.load();
  for (int j = 0; j < njobs; ++j) {
    set_trailer t;
    std::memcpy(&t, outs[j].data() + out_b - sizeof t, sizeof t);
    if (status[j] != SET_OK || t.job_id != ids[j] || (t.word >> 16) != SET_TRAILER_MAGIC) ++bad;
  }
  if (st.completed != (uint64_t)njobs || st.submitted != (uint64_t)njobs || st.failed || st.canary_errors) ++bad;
  set_destroy(ctx);
  std::printf("jobs %d bad %d steals %llu\n", njobs, bad, (unsigned long long)st.steals);
  return bad ? 1 : 0;
}
