// trace.cpp -- CUPTI activity trace of kernels and copies (measurement helper of set.h).
//
// The paper locates the scheduling overhead in gaps of the device timeline (Sec. 3.2: t_in-in,
// t_in-k, delta t_k, t_k-out inside a batch, t_inter between batches; Eq. 4 t_schedule =
// T_measured - T_ideal).  This module records every kernel and memcpy with CUPTI's activity API
// (device timestamps) and reduces them to: mean / max idle gap between consecutive kernels on the
// device timeline, busy time of kernels, copies and either, and the idle fraction of the span.
// libcupti is opened with dlopen on first use, so the library does not depend on it otherwise.
#include <cupti.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "executor.h"
#include "set.h"
#include "thread_error.h"

namespace {

struct Rec {
  uint64_t start, end;
  int kernel;  // 1 kernel, 0 copy
  std::string name;
};

struct Cupti {
  CUptiResult (*enable)(CUpti_ActivityKind) = nullptr;
  CUptiResult (*disable)(CUpti_ActivityKind) = nullptr;
  CUptiResult (*reg)(CUpti_BuffersCallbackRequestFunc, CUpti_BuffersCallbackCompleteFunc) = nullptr;
  CUptiResult (*flush)(uint32_t) = nullptr;
  CUptiResult (*next)(uint8_t*, size_t, CUpti_Activity**) = nullptr;
  bool ok = false;
};

std::mutex g_mu;
Cupti g_c;
std::vector<Rec> g_recs;
bool g_on = false;
uint64_t g_start_ns = 0;  // host clock at set_trace_start

bool load_cupti() {
  if (g_c.ok) return true;
  const char* home = std::getenv("CUDA_HOME");
  std::vector<std::string> cands = {"libcupti.so.13", "libcupti.so"};
  for (const char* base : {home, "/usr/local/cuda"}) {
    if (!base) continue;
    cands.push_back(std::string(base) + "/lib64/libcupti.so.13");
    cands.push_back(std::string(base) + "/extras/CUPTI/lib64/libcupti.so.13");
    cands.push_back(std::string(base) + "/targets/sbsa-linux/lib/libcupti.so.13");
    cands.push_back(std::string(base) + "/targets/x86_64-linux/lib/libcupti.so.13");
  }
  void* h = nullptr;
  for (const auto& c : cands)
    if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) return false;
  g_c.enable = reinterpret_cast<decltype(g_c.enable)>(dlsym(h, "cuptiActivityEnable"));
  g_c.disable = reinterpret_cast<decltype(g_c.disable)>(dlsym(h, "cuptiActivityDisable"));
  g_c.reg = reinterpret_cast<decltype(g_c.reg)>(dlsym(h, "cuptiActivityRegisterCallbacks"));
  g_c.flush = reinterpret_cast<decltype(g_c.flush)>(dlsym(h, "cuptiActivityFlushAll"));
  g_c.next = reinterpret_cast<decltype(g_c.next)>(dlsym(h, "cuptiActivityGetNextRecord"));
  g_c.ok = g_c.enable && g_c.disable && g_c.reg && g_c.flush && g_c.next;
  return g_c.ok;
}

void CUPTIAPI buffer_requested(uint8_t** buf, size_t* size, size_t* max_records) {
  *size = 8u << 20;
  *buf = static_cast<uint8_t*>(std::aligned_alloc(8, *size));
  *max_records = 0;
}

void CUPTIAPI buffer_completed(CUcontext, uint32_t, uint8_t* buf, size_t, size_t valid) {
  CUpti_Activity* r = nullptr;
  std::vector<Rec> local;
  while (g_c.next(buf, valid, &r) == CUPTI_SUCCESS) {
    if (r->kind == CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL || r->kind == CUPTI_ACTIVITY_KIND_KERNEL) {
      const auto* k = reinterpret_cast<const CUpti_ActivityKernel10*>(r);
      local.push_back({k->start, k->end, 1, k->name ? k->name : "?"});
    } else if (r->kind == CUPTI_ACTIVITY_KIND_MEMCPY) {
      const auto* m = reinterpret_cast<const CUpti_ActivityMemcpy6*>(r);
      local.push_back({m->start, m->end, 0, std::string()});
    }
  }
  std::free(buf);
  std::lock_guard<std::mutex> g(g_mu);
  g_recs.insert(g_recs.end(), local.begin(), local.end());
}

// Length of the union of [start, end) intervals.
double union_ns(std::vector<std::pair<uint64_t, uint64_t>> iv) {
  std::sort(iv.begin(), iv.end());
  double total = 0;
  uint64_t s = 0, e = 0;
  bool open = false;
  for (auto& p : iv) {
    if (!open || p.first > e) {
      if (open) total += (double)(e - s);
      s = p.first;
      e = p.second;
      open = true;
    } else {
      e = std::max(e, p.second);
    }
  }
  if (open) total += (double)(e - s);
  return total;
}

}  // namespace

extern "C" set_status set_trace_start(void) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!load_cupti()) {
    setrt::set_thread_error("set_trace_start: libcupti could not be loaded");
    return SET_EINVAL;
  }
  g_recs.clear();
  if (g_c.reg(buffer_requested, buffer_completed) != CUPTI_SUCCESS ||
      g_c.enable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL) != CUPTI_SUCCESS ||
      g_c.enable(CUPTI_ACTIVITY_KIND_MEMCPY) != CUPTI_SUCCESS) {
    setrt::set_thread_error("set_trace_start: CUPTI activity tracing could not be enabled");
    return SET_ECUDA;
  }
  g_on = true;
  g_start_ns = setrt::now_ns();
  return SET_OK;
}

extern "C" set_status set_trace_stop(set_trace_summary* out) {
  if (!out) return SET_EINVAL;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_on) return SET_EINVAL;
  }
  g_c.flush(1);  // delivers the remaining buffers through buffer_completed
  g_c.disable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL);
  g_c.disable(CUPTI_ACTIVITY_KIND_MEMCPY);
  g_c.flush(1);
  std::lock_guard<std::mutex> g(g_mu);
  g_on = false;
  std::memset(out, 0, sizeof *out);
  std::vector<Rec>& R = g_recs;
  if (R.empty()) return SET_OK;
  std::vector<std::pair<uint64_t, uint64_t>> kiv, civ, all;
  uint64_t t0 = ~0ull, t1 = 0;
  std::map<std::string, std::pair<double, uint64_t>> per_name;
  for (const auto& r : R) {
    (r.kernel ? kiv : civ).push_back({r.start, r.end});
    all.push_back({r.start, r.end});
    t0 = std::min(t0, r.start);
    t1 = std::max(t1, r.end);
    if (r.kernel) {
      auto& p = per_name[r.name];
      p.first += (double)(r.end - r.start);
      p.second += 1;
    }
  }
  out->kernels = kiv.size();
  out->memcpys = civ.size();
  out->span_us = (double)(t1 - t0) * 1e-3;
  out->kernel_busy_us = union_ns(kiv) * 1e-3;
  out->copy_busy_us = union_ns(civ) * 1e-3;
  out->any_busy_us = union_ns(all) * 1e-3;
  out->idle_frac = out->span_us > 0 ? 1.0 - out->any_busy_us / out->span_us : 0.0;
  std::sort(kiv.begin(), kiv.end());
  double gsum = 0, gmax = 0;
  uint64_t run_end = kiv.empty() ? 0 : kiv[0].second;
  for (size_t i = 1; i < kiv.size(); ++i) {
    const double gap = kiv[i].first > run_end ? (double)(kiv[i].first - run_end) : 0.0;
    gsum += gap;
    gmax = std::max(gmax, gap);
    run_end = std::max(run_end, kiv[i].second);
  }
  out->mean_kernel_gap_us = kiv.size() > 1 ? gsum / (double)(kiv.size() - 1) * 1e-3 : 0.0;
  setrt::note_trace_gap(out->mean_kernel_gap_us, g_start_ns);
  out->max_kernel_gap_us = gmax * 1e-3;
  double best = -1;
  double ksum = 0;
  for (const auto& kv : per_name) ksum += kv.second.first;
  for (const auto& kv : per_name) {
    if (kv.second.first > best) {
      best = kv.second.first;
      std::strncpy(out->top_kernel, kv.first.c_str(), sizeof(out->top_kernel) - 1);
      out->top_kernel_launches = kv.second.second;
      out->top_kernel_mean_us = kv.second.first / (double)kv.second.second * 1e-3;
      out->top_kernel_share = ksum > 0 ? kv.second.first / ksum : 0.0;
    }
  }
  return SET_OK;
}
