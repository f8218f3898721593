// cuda_device.cpp -- the executor's CUDA side: slot pool, lane streams, one graph exec per
// (slot, job type), per-job parameter updates, event-chained completion callbacks, direct
// launches and the two baseline programming models (Sec. 4.1-4.2, Sec. 5.1.3).
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "../kernels/stages.h"
#include "executor.h"

namespace setrt {
namespace {

#define SET_CK(call)                                                              \
  do {                                                                            \
    const cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                      \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return SET_ECUDA;                                                           \
    }                                                                             \
  } while (0)

constexpr size_t kPlaceholderBytes = 1 << 16;

struct GraphInst {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t h2d = nullptr, d2h = nullptr;
  cudaGraphNode_t kn[setk::kMaxKernels] = {};
  int nk = 0;
};

struct SlotState {
  GraphInst gi[SET_NUM_JOB_TYPES + 1];
  cudaEvent_t done = nullptr;
};

// Smallest valid dims of each type: graph templates are built with these and every job
// overwrites all copy and kernel parameters before its launch.
void template_dims(uint32_t type, uint32_t d[4]) {
  d[0] = d[1] = d[2] = d[3] = 0;
  switch (type) {
    case SET_JOB_BLUR_HIST:
    case SET_JOB_IMG_SOBEL_HIST:
      d[0] = d[1] = 16;
      break;
    case SET_JOB_SAXPY_SCAN_MAX:
      d[0] = 256;
      break;
    case SET_JOB_MLP_LN:
      d[0] = 1;
      break;
    default:
      break;
  }
}

void CUDART_CB host_complete(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->ex->on_complete(*s, SET_OK);
}

cudaKernelNodeParams node_params(setk::KernelLaunch& k) {
  cudaKernelNodeParams p{};
  p.func = const_cast<void*>(k.func);
  p.gridDim = k.grid;
  p.blockDim = k.block;
  p.sharedMemBytes = k.smem;
  p.kernelParams = k.params;
  p.extra = nullptr;
  return p;
}

class CudaDevice final : public Device {
 public:
  explicit CudaDevice(const set_config& c) : cfg_(c) {}
  ~CudaDevice() override { release(); }

  set_status init(const set_config& cfg, std::vector<Slot>& slots, std::string* err) override;
  set_status launch(Slot& s, LaunchCost* cost, std::string* err) override;
  void drain() override;
  bool supports(uint32_t type) const override {
    return type >= 1 && type <= SET_NUM_JOB_TYPES && supported_[type];
  }
  set_status run_baseline(int kind, const JobRec* jobs, size_t n, std::vector<Slot>& slots, LogHist* lat,
                          LaunchCost* cost, uint64_t* t0, uint64_t* t1, std::string* err) override;

 private:
  set_status build_graph(Slot& s, uint32_t type, std::string* err);
  bool plan(const Slot& s, const JobRec& j, setk::JobLayout* L, setk::KernelLaunch* kl, int* nk) const;
  set_status update(const Slot& s, const JobRec& j, GraphInst& gi, LaunchCost* cost, std::string* err);
  void release();

  set_config cfg_;
  std::vector<cudaStream_t> lanes_, cbs_;
  std::vector<SlotState> st_;
  void* pool_ = nullptr;
  bool own_pool_ = false;
  void* ph_host_ = nullptr;
  void* ph_dev_ = nullptr;
  size_t ctl_ = 0;
  bool supported_[SET_NUM_JOB_TYPES + 1] = {};
  cudaMemcpyKind kind_in_ = cudaMemcpyHostToDevice, kind_out_ = cudaMemcpyDeviceToHost;
};

set_status CudaDevice::init(const set_config& cfg, std::vector<Slot>& slots, std::string* err) {
  cfg_ = cfg;
  SET_CK(cudaSetDevice(cfg.device));
  SET_CK(cudaFree(nullptr));
  SET_CK(setk::kernels_init());
  const size_t stride = setk::align256(cfg.slot_bytes);
  const size_t need = stride * slots.size();
  if (cfg.pool) {
    if (cfg.pool_bytes < need || (reinterpret_cast<uintptr_t>(cfg.pool) & 255)) {
      *err = "set_config.pool too small or not 256-byte aligned";
      return SET_EINVAL;
    }
    pool_ = cfg.pool;
  } else {
    if (cudaMalloc(&pool_, need) != cudaSuccess) {
      cudaGetLastError();
      *err = "cudaMalloc of the slot pool failed (" + std::to_string(need) + " bytes)";
      pool_ = nullptr;
      return SET_ENOMEM;
    }
    own_pool_ = true;
  }
  SET_CK(cudaMemset(pool_, 0, need));  // control blocks start zeroed
  SET_CK(cudaHostAlloc(&ph_host_, kPlaceholderBytes, cudaHostAllocDefault));
  SET_CK(cudaMalloc(&ph_dev_, kPlaceholderBytes));
  if (cfg.io_mode == SET_IO_DEVICE) {
    kind_in_ = cudaMemcpyDeviceToDevice;
    kind_out_ = cudaMemcpyDeviceToDevice;
  }
  ctl_ = setk::slot_control_bytes(cfg.slot_bytes);
  lanes_.resize(cfg.num_streams);
  cbs_.resize(cfg.num_streams);
  for (int i = 0; i < cfg.num_streams; ++i) {
    SET_CK(cudaStreamCreateWithFlags(&lanes_[i], cudaStreamNonBlocking));
    SET_CK(cudaStreamCreateWithFlags(&cbs_[i], cudaStreamNonBlocking));
  }
  st_.resize(slots.size());
  for (auto& s : slots) {
    s.dev = static_cast<uint8_t*>(pool_) + stride * s.index;
    s.bytes = cfg.slot_bytes;
    s.dev_state = &st_[s.index];
    SET_CK(cudaEventCreateWithFlags(&st_[s.index].done, cudaEventDisableTiming));
    for (uint32_t t = 1; t <= SET_NUM_JOB_TYPES; ++t) {
      if (!(cfg.type_mask & (1u << t))) continue;
      const set_status b = build_graph(s, t, err);
      if (b != SET_OK) return b;
    }
  }
  for (uint32_t t = 1; t <= SET_NUM_JOB_TYPES; ++t) supported_[t] = st_.empty() ? false : st_[0].gi[t].exec != nullptr;
  SET_CK(cudaDeviceSynchronize());
  return SET_OK;
}

bool CudaDevice::plan(const Slot& s, const JobRec& j, setk::JobLayout* L, setk::KernelLaunch* kl, int* nk) const {
  if (!setk::job_sizes(j.d.type, j.d.dims, L)) return false;
  setk::place_job(L, ctl_);
  setk::JobPlanIn in;
  in.type = j.d.type;
  std::memcpy(in.dims, j.d.dims, sizeof in.dims);
  in.scalar = j.d.scalar;
  in.shared[0] = j.d.shared[0];
  in.shared[1] = j.d.shared[1];
  in.d_in = s.dev + L->in_off;
  in.d_out = s.dev + L->out_off;
  in.d_scratch = s.dev + L->scratch_off;
  in.d_persist = s.dev + setk::control_offset(j.d.type);
  in.job_id = j.id;
  in.slot_gen = s.gen;
  in.img_fused = cfg_.img_fused;
  return setk::plan_job(in, kl, nk);
}

// Graph template of one job type bound to one slot (Sec. 4.1): H2D -> kernel DAG -> D2H, built
// once; copy endpoints and kernel arguments are placeholders overwritten per job.
set_status CudaDevice::build_graph(Slot& s, uint32_t type, std::string* err) {
  JobRec rep;
  rep.d.type = type;
  template_dims(type, rep.d.dims);
  rep.d.shared[0] = rep.d.shared[1] = ph_dev_;
  setk::JobLayout L;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  if (!plan(s, rep, &L, kl, &nk)) return SET_OK;  // type not provided by this build: no graph
  if (L.end > s.bytes || L.in_bytes > kPlaceholderBytes || L.out_bytes > kPlaceholderBytes) return SET_OK;
  GraphInst& gi = st_[s.index].gi[type];
  SET_CK(cudaGraphCreate(&gi.graph, 0));
  const void* src_ph = cfg_.io_mode == SET_IO_HOST ? ph_host_ : ph_dev_;
  void* dst_ph = cfg_.io_mode == SET_IO_HOST ? ph_host_ : ph_dev_;
  SET_CK(cudaGraphAddMemcpyNode1D(&gi.h2d, gi.graph, nullptr, 0, s.dev + L.in_off, src_ph, L.in_bytes, kind_in_));
  uint32_t has_dependents = 0;
  for (int k = 0; k < nk; ++k) {
    cudaGraphNode_t deps[setk::kMaxKernels];
    size_t nd = 0;
    if (kl[k].deps == 0) {
      deps[nd++] = gi.h2d;
    } else {
      for (int q = 0; q < k; ++q)
        if (kl[k].deps & (1u << q)) {
          deps[nd++] = gi.kn[q];
          has_dependents |= 1u << q;
        }
    }
    const cudaKernelNodeParams p = node_params(kl[k]);
    SET_CK(cudaGraphAddKernelNode(&gi.kn[k], gi.graph, deps, nd, &p));
  }
  cudaGraphNode_t sinks[setk::kMaxKernels];
  size_t ns = 0;
  for (int k = 0; k < nk; ++k)
    if (!(has_dependents & (1u << k))) sinks[ns++] = gi.kn[k];
  SET_CK(cudaGraphAddMemcpyNode1D(&gi.d2h, gi.graph, sinks, ns, dst_ph, s.dev + L.out_off, L.out_bytes, kind_out_));
  gi.nk = nk;
  SET_CK(cudaGraphInstantiate(&gi.exec, gi.graph, 0));
  return SET_OK;
}

// UpdateGraphParams (Algorithms 1-2): rebind the exec's copies and kernels to this job.
set_status CudaDevice::update(const Slot& s, const JobRec& j, GraphInst& gi, LaunchCost* cost, std::string* err) {
  setk::JobLayout L;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  if (!plan(s, j, &L, kl, &nk) || nk != gi.nk) {
    *err = "job does not match its graph template";
    return SET_EINVAL;
  }
  const uint64_t t0 = now_ns();
  cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(gi.exec, gi.h2d, s.dev + L.in_off, j.d.in, L.in_bytes, kind_in_);
  if (e == cudaSuccess)
    for (int k = 0; k < nk && e == cudaSuccess; ++k) {
      const cudaKernelNodeParams p = node_params(kl[k]);
      e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.kn[k], &p);
    }
  if (e == cudaSuccess)
    e = cudaGraphExecMemcpyNodeSetParams1D(gi.exec, gi.d2h, j.d.out, s.dev + L.out_off, L.out_bytes, kind_out_);
  cost->update_ns += now_ns() - t0;
  cost->updates += (uint64_t)nk + 2;
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("graph parameter update rejected (host buffers must be pinned, device buffers must be on "
                       "the context's GPU): ") + cudaGetErrorString(e);
    return SET_EINVAL;
  }
  return SET_OK;
}

// LaunchJob (Algorithm 2) + AddCallback: the callback hangs off a per-lane callback stream that
// waits on an event recorded behind the graph, so the lane stream runs on without a host round
// trip.
set_status CudaDevice::launch(Slot& s, LaunchCost* cost, std::string* err) {
  SlotState& ss = st_[s.index];
  GraphInst& gi = ss.gi[s.job.d.type];
  if (!gi.exec) {
    *err = "job type not instantiated";
    return SET_EINVAL;
  }
  const set_status u = update(s, s.job, gi, cost, err);
  if (u != SET_OK) return u;
  const uint64_t t1 = now_ns();
  cudaStream_t lane = lanes_[s.lane], cb = cbs_[s.lane];
  SET_CK(cudaGraphLaunch(gi.exec, lane));
  if (cfg_.cb_mode == 1) {
    SET_CK(cudaLaunchHostFunc(lane, host_complete, &s));
  } else {
    SET_CK(cudaEventRecord(ss.done, lane));
    SET_CK(cudaStreamWaitEvent(cb, ss.done, 0));
    SET_CK(cudaLaunchHostFunc(cb, host_complete, &s));
  }
  cost->launch_ns += now_ns() - t1;
  return SET_OK;
}

void CudaDevice::drain() {
  for (auto s : lanes_) cudaStreamSynchronize(s);
  for (auto s : cbs_) cudaStreamSynchronize(s);
}

void CudaDevice::release() {
  drain();
  for (auto& ss : st_) {
    for (auto& gi : ss.gi) {
      if (gi.exec) cudaGraphExecDestroy(gi.exec);
      if (gi.graph) cudaGraphDestroy(gi.graph);
    }
    if (ss.done) cudaEventDestroy(ss.done);
  }
  st_.clear();
  for (auto s : lanes_) cudaStreamDestroy(s);
  for (auto s : cbs_) cudaStreamDestroy(s);
  lanes_.clear();
  cbs_.clear();
  if (own_pool_ && pool_) cudaFree(pool_);
  pool_ = nullptr;
  if (ph_host_) cudaFreeHost(ph_host_);
  if (ph_dev_) cudaFree(ph_dev_);
  ph_host_ = ph_dev_ = nullptr;
}

// Baselines of Sec. 5.1.3 on the same kernels and slots.
//  SET_BASE_SYNC: one stream, one slot; per job cudaMemcpyAsync H2D, plain kernel launches,
//    cudaMemcpyAsync D2H, stream-ordered, no host synchronisation between jobs.
//  SET_BASE_BATCH_SYNC: b lanes with one graph exec each (ring entry 0); per batch of b jobs
//    update every exec, launch all, then cudaStreamSynchronize every lane before the next batch.
set_status CudaDevice::run_baseline(int kind, const JobRec* jobs, size_t n, std::vector<Slot>& slots, LogHist* lat,
                                    LaunchCost* cost, uint64_t* t0, uint64_t* t1, std::string* err) {
  const size_t L = lanes_.size();
  if (kind == SET_BASE_SYNC) {
    Slot& s = slots[0];
    cudaStream_t st = lanes_[0];
    *t0 = now_ns();
    for (size_t i = 0; i < n; ++i) {
      const JobRec& j = jobs[i];
      setk::JobLayout Lo;
      setk::KernelLaunch kl[setk::kMaxKernels];
      int nk = 0;
      JobRec jj = j;
      if (!plan(s, jj, &Lo, kl, &nk)) {
        *err = "invalid job";
        return SET_EINVAL;
      }
      const uint64_t ta = now_ns();
      SET_CK(cudaMemcpyAsync(s.dev + Lo.in_off, j.d.in, Lo.in_bytes, kind_in_, st));
      for (int k = 0; k < nk; ++k)
        SET_CK(cudaLaunchKernel(kl[k].func, kl[k].grid, kl[k].block, kl[k].params, kl[k].smem, st));
      SET_CK(cudaMemcpyAsync(j.d.out, s.dev + Lo.out_off, Lo.out_bytes, kind_out_, st));
      cost->launch_ns += now_ns() - ta;
      s.gen += 1;
    }
    SET_CK(cudaStreamSynchronize(st));
    *t1 = now_ns();
    return SET_OK;
  }
  if (kind == SET_BASE_BATCH_SYNC) {
    *t0 = now_ns();
    for (size_t base = 0; base < n; base += L) {
      const size_t nb = std::min(L, n - base);
      for (size_t i = 0; i < nb; ++i) {
        Slot& s = slots[i];  // ring entry 0 of lane i
        const JobRec& j = jobs[base + i];
        GraphInst& gi = st_[s.index].gi[j.d.type];
        if (!gi.exec) {
          *err = "job type not instantiated";
          return SET_EINVAL;
        }
        const set_status u = update(s, j, gi, cost, err);
        if (u != SET_OK) return u;
        const uint64_t ta = now_ns();
        SET_CK(cudaGraphLaunch(gi.exec, lanes_[i]));
        cost->launch_ns += now_ns() - ta;
      }
      for (size_t i = 0; i < nb; ++i) SET_CK(cudaStreamSynchronize(lanes_[i]));
      const uint64_t tb = now_ns();
      for (size_t i = 0; i < nb; ++i) {
        const uint64_t arrival = jobs[base + i].d.t_arrival_ns ? jobs[base + i].d.t_arrival_ns : *t0;
        lat->record(tb > arrival ? tb - arrival : 0);
        slots[i].gen += 1;
      }
    }
    *t1 = now_ns();
    return SET_OK;
  }
  *err = "unknown baseline kind";
  return SET_EINVAL;
}

}  // namespace

std::unique_ptr<Device> make_device(const set_config& cfg) { return std::unique_ptr<Device>(new CudaDevice(cfg)); }

}  // namespace setrt

// ---- direct launches (C ABI) ----
extern "C" set_status set_launch_job(const set_job_desc* job, const void* d_in, void* d_out, void* d_scratch,
                                     uint64_t job_id, uint32_t slot_gen, void* stream) {
  if (!job || !d_in || !d_out) return SET_EINVAL;
  setk::JobLayout L;
  if (!setk::job_sizes(job->type, job->dims, &L)) return SET_EINVAL;
  if ((L.persist_bytes || L.scratch_bytes) && !d_scratch) return SET_EINVAL;
  static thread_local bool inited = false;
  if (!inited) {
    if (setk::kernels_init() != cudaSuccess) return SET_ECUDA;
    inited = true;
  }
  setk::JobPlanIn in;
  in.type = job->type;
  std::memcpy(in.dims, job->dims, sizeof in.dims);
  in.scalar = job->scalar;
  in.shared[0] = job->shared[0];
  in.shared[1] = job->shared[1];
  in.d_in = d_in;
  in.d_out = d_out;
  in.d_persist = d_scratch;
  in.d_scratch = static_cast<uint8_t*>(d_scratch) + setk::align256(L.persist_bytes);
  in.job_id = job_id;
  in.slot_gen = slot_gen;
  in.img_fused = 1;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  if (!setk::plan_job(in, kl, &nk)) return SET_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nk; ++k)
    if (cudaLaunchKernel(kl[k].func, kl[k].grid, kl[k].block, kl[k].params, kl[k].smem, st) != cudaSuccess)
      return SET_ECUDA;
  return SET_OK;
}

extern "C" set_status set_copy_bandwidth(size_t bytes, int streams, int reps, int dir, double* gbs) {
  if (!gbs || bytes == 0 || streams < 1 || reps < 1 || dir < 0 || dir > 2) return SET_EINVAL;
  std::vector<cudaStream_t> ss(streams, nullptr);
  std::vector<void*> h(2 * streams, nullptr), d(2 * streams, nullptr);
  set_status st = SET_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && st == SET_OK) st = SET_ECUDA;
    return e == cudaSuccess;
  };
  for (int i = 0; i < streams && st == SET_OK; ++i) {
    ok(cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
    ok(cudaHostAlloc(&h[2 * i], bytes, cudaHostAllocDefault));
    ok(cudaHostAlloc(&h[2 * i + 1], bytes, cudaHostAllocDefault));
    ok(cudaMalloc(&d[2 * i], bytes));
    ok(cudaMalloc(&d[2 * i + 1], bytes));
  }
  ok(cudaEventCreate(&e0));
  ok(cudaEventCreate(&e1));
  if (st == SET_OK) {
    for (int pass = 0; pass < 2 && st == SET_OK; ++pass) {  // pass 0 warms up
      ok(cudaDeviceSynchronize());
      ok(cudaEventRecord(e0, ss[0]));
      for (int i = 1; i < streams; ++i) ok(cudaStreamWaitEvent(ss[i], e0, 0));
      for (int r = 0; r < reps; ++r) {
        const int i = r % streams;
        if (dir != 1) ok(cudaMemcpyAsync(d[2 * i], h[2 * i], bytes, cudaMemcpyHostToDevice, ss[i]));
        if (dir != 0) ok(cudaMemcpyAsync(h[2 * i + 1], d[2 * i + 1], bytes, cudaMemcpyDeviceToHost, ss[i]));
      }
      for (int i = 1; i < streams; ++i) {
        cudaEvent_t ev;
        ok(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ok(cudaEventRecord(ev, ss[i]));
        ok(cudaStreamWaitEvent(ss[0], ev, 0));
        cudaEventDestroy(ev);
      }
      ok(cudaEventRecord(e1, ss[0]));
      ok(cudaEventSynchronize(e1));
    }
    float ms = 0.f;
    if (ok(cudaEventElapsedTime(&ms, e0, e1)))
      *gbs = (double)bytes * reps * (dir == 2 ? 2.0 : 1.0) / ((double)ms * 1e-3) / 1e9;
  }
  for (int i = 0; i < streams; ++i) {
    if (ss[i]) cudaStreamDestroy(ss[i]);
    if (h[2 * i]) cudaFreeHost(h[2 * i]);
    if (h[2 * i + 1]) cudaFreeHost(h[2 * i + 1]);
    if (d[2 * i]) cudaFree(d[2 * i]);
    if (d[2 * i + 1]) cudaFree(d[2 * i + 1]);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

extern "C" int set_job_kernel_count(uint32_t type, const uint32_t dims[4], int img_fused) {
  setk::JobLayout L;
  if (!setk::job_sizes(type, dims, &L)) return -1;
  setk::JobPlanIn in;
  in.type = type;
  std::memcpy(in.dims, dims, sizeof in.dims);
  in.img_fused = img_fused;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  return setk::plan_job(in, kl, &nk) ? nk : -1;
}
