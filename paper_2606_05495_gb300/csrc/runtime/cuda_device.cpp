// cuda_device.cpp -- the executor's CUDA side: slot pool, lane streams, one graph exec per
// (slot, job type), per-job parameter updates, event-chained completion callbacks, direct
// launches and the two baseline programming models (Sec. 4.1-4.2, Sec. 5.1.3).  cb_mode 3 replaces
// the host-function callback by a completion thread that queries each lane's oldest event.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../kernels/stages.h"
#include "executor.h"
#include "sync.h"
#include "thread_error.h"

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
constexpr size_t kTableStaging = 96 << 10;  // >= the largest batch table (64 image jobs: 82,176 bytes)

struct GraphInst {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t h2d = nullptr, d2h = nullptr;
  cudaGraphNode_t arm = nullptr, check = nullptr;  // set_config.guards: guard bands around the job
  cudaGraphNode_t kn[setk::kMaxKernels] = {};
  int nk = 0;
};

// Batched form: table H2D, kMaxBatch-capable job copy nodes (unused ones disabled per launch),
// the packed kernels, and a D2H node per job.
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t table = nullptr;
  std::vector<cudaGraphNode_t> h2d, d2h;
  std::vector<char> on;  // enabled state of job j's copy nodes in the exec
  cudaGraphNode_t kn[setk::kMaxKernels] = {};
  int nk = 0;
};

struct SlotState {
  GraphInst gi[SET_NUM_JOB_TYPES + 1];
  BatchGraph bg[SET_NUM_JOB_TYPES + 1];
  uint8_t* h_table = nullptr;  // pinned staging of the batch table (written at dispatch)
  uint64_t* h_stamps = nullptr;  // stamps mode: mapped host {entry, exit} x kernels
  uint64_t* d_stamps = nullptr;  // its device alias
  cudaEvent_t done = nullptr;
};

// Smallest valid dims of each type: graph templates are built with these, so that a slot sized
// for any one job of the type holds its template, and every job overwrites all copy and kernel
// parameters before its launch.
void template_dims(uint32_t type, uint32_t d[4]) {
  d[0] = d[1] = d[2] = d[3] = 0;
  switch (type) {
    case SET_JOB_BLUR_HIST:
    case SET_JOB_IMG_SOBEL_HIST:
      d[0] = d[1] = 1;
      break;
    case SET_JOB_SAXPY_SCAN_MAX:
    case SET_JOB_MLP_LN:
      d[0] = 1;
      break;
    case SET_JOB_HOTSPOT:
      d[0] = d[1] = d[2] = 1;
      break;
    default:
      break;
  }
}

void CUDART_CB host_complete(void* p) {
  Slot* s = static_cast<Slot*>(p);
  if (s->quiet.load(std::memory_order_acquire)) return;  // a baseline is reusing the slot's graph
  s->ex->on_complete_group(*s);
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
  set_status launch(Slot& s, bool callback, LaunchCost* cost, std::string* err) override;
  set_status prepare(Slot& s, LaunchCost* cost, std::string* err) override;
  set_status launch_bound(Slot& s, bool callback, LaunchCost* cost, std::string* err) override;
  set_status launch_batch(Slot& s, bool callback, LaunchCost* cost, std::string* err) override;
  set_status autotune(uint32_t type, const JobRec* sample, size_t n, int max_batch, set_tune_result* out,
                      std::string* err) override;
  set_status attach_callback(Slot& s, std::string* err) override;
  void drain() override;
  uint8_t* arena_base() override { return static_cast<uint8_t*>(arena_); }
  void thread_init() override {
    cudaSetDevice(cfg_.device);
    cudaFree(nullptr);  // the primary context is current on this thread from here on
  }
  bool supports(uint32_t type) const override {
    return type >= 1 && type <= SET_NUM_JOB_TYPES && supported_[type];
  }
  bool io_device(const void* p) const override {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == cfg_.device;
  }
  bool io_accessible(const void* p) const override {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    // page-locked host memory mapped at the same address; not device memory, whose trailer the
    // completion path could not read on the host
    return at.type == cudaMemoryTypeHost && at.devicePointer == p;
  }
  set_status run_baseline(int kind, const JobRec* jobs, size_t n, std::vector<Slot>& slots, BuddyArena* arena,
                          LogHist* lat, LaunchCost* cost, uint64_t* t0, uint64_t* t1, std::string* err) override;

 private:
  set_status build_graph(Slot& s, uint32_t type, std::string* err);
  set_status build_batch_graph(Slot& s, uint32_t type, std::string* err);
  bool plan_batch(Slot& s, const setk::BatchItem* items, int nb, const setk::BatchLayout& L, uint8_t* d_block,
                  const void* const shared[2], setk::KernelLaunch* kl, int* nk);
  uint8_t* batch_block(Slot& s) { return s.job_mem ? s.job_mem : s.dev + ctl_; }
  setk::Stamp stamp_base(const Slot& s) const {
    setk::Stamp st;
    if (clock_) {
      st.clock = clock_;
      st.ctr = reinterpret_cast<uint32_t*>(s.dev + setk::kCtlStampOff);
      st.out = st_[s.index].d_stamps;
    }
    return st;
  }
  // Before a launch: clear the slot's stamp array and remember the kernels' dependencies.
  void arm_stamps(Slot& s, const setk::KernelLaunch* kl, int nk) {
    if (!clock_) return;
    for (int k = 0; k < 2 * setk::kMaxKernels; ++k) st_[s.index].h_stamps[k] = 0;
    s.stamp_nk = nk;
    for (int k = 0; k < nk; ++k) s.stamp_deps[k] = kl[k].deps;
  }
  bool plan(const Slot& s, const JobRec& j, setk::JobLayout* L, setk::KernelLaunch* kl, int* nk) const;
  set_status update(const Slot& s, const JobRec& j, GraphInst& gi, LaunchCost* cost, std::string* err);
  void release();

  set_config cfg_;
  std::vector<cudaStream_t> lanes_, cbs_;
  std::vector<SlotState> st_;
  void* pool_ = nullptr;
  bool own_pool_ = false;
  void* arena_ = nullptr;
  void* ph_host_ = nullptr;
  void* ph_dev_ = nullptr;
  size_t ctl_ = 0;
  bool supported_[SET_NUM_JOB_TYPES + 1] = {};
  std::atomic<int> img_ctas_{4}, img_tile_{0};  // batched image kernel launch shape (autotuned)
  unsigned long long* clock_ = nullptr;          // stamps mode: the ticket counter
  cudaMemcpyKind kind_in_ = cudaMemcpyHostToDevice, kind_out_ = cudaMemcpyDeviceToHost;

  // cb_mode 3: completion thread.  Dispatchers hand it (slot, event recorded behind the graph);
  // it polls the oldest event of every lane (a lane's events complete in stream order) and runs
  // the completion path itself, sleeping on a futex while nothing is in flight.
  void poll_main();
  void poll_push(Slot* s);
  std::thread poller_;
  std::atomic<bool> poll_stop_{false};
  std::atomic<int64_t> poll_pending_{0};
  Signal poll_sig_;
  std::mutex poll_mu_;
  std::vector<Slot*> poll_in_;
};

void CudaDevice::poll_push(Slot* s) {
  poll_pending_.fetch_add(1);
  {
    std::lock_guard<std::mutex> g(poll_mu_);
    poll_in_.push_back(s);
  }
  poll_sig_.notify(1);
}

void CudaDevice::poll_main() {
  thread_init();
  std::vector<std::deque<Slot*>> fifo(lanes_.size());
  std::vector<Slot*> got;
  int idle_rounds = 0;
  for (;;) {
    const uint32_t seen = poll_sig_.load();
    {
      std::lock_guard<std::mutex> g(poll_mu_);
      got.swap(poll_in_);
    }
    for (Slot* s : got) fifo[s->lane].push_back(s);
    got.clear();
    bool waiting = false, progressed = false;
    for (auto& q : fifo) {
      while (!q.empty()) {
        Slot* s = q.front();
        const cudaError_t e = cudaEventQuery(st_[s->index].done);
        if (e == cudaErrorNotReady) {
          waiting = true;
          break;
        }
        if (e != cudaSuccess) cudaGetLastError();  // the job's trailer check reports the failure
        q.pop_front();
        progressed = true;
        host_complete(s);
        poll_pending_.fetch_sub(1);
      }
    }
    if (waiting) {
      // jobs in flight: after a round without a completion, pause 2 us (a plain clock spin, no
      // driver call) before querying again, so the queries do not contend with the dispatch
      // threads' launches for the driver; yield the core after a run of empty rounds
      idle_rounds = progressed ? 0 : idle_rounds + 1;
      if (!progressed) {
        const uint64_t t_next = now_ns() + 2000ull;
        while (now_ns() < t_next && poll_sig_.load() == seen) {
        }
      }
      if (idle_rounds > 64) std::this_thread::yield();
      continue;
    }
    if (poll_stop_.load()) return;
    // idle: spin spin_us on the signal first (a job launched meanwhile needs no futex wake), then sleep
    const uint64_t t_end = now_ns() + (uint64_t)(cfg_.spin_us > 0 ? cfg_.spin_us : 0) * 1000ull;
    while (poll_sig_.load() == seen && !poll_stop_.load() && now_ns() < t_end) {
    }
    if (poll_sig_.load() == seen) poll_sig_.wait(seen, 100 * 1000000ll);
  }
}

set_status CudaDevice::init(const set_config& cfg, std::vector<Slot>& slots, std::string* err) {
  cfg_ = cfg;
  img_ctas_.store(cfg.img_ctas_per_sm > 0 ? cfg.img_ctas_per_sm : 4);
  img_tile_.store(cfg.img_tile >= 0 && cfg.img_tile <= 2 ? cfg.img_tile : 0);
  SET_CK(cudaSetDevice(cfg.device));
  SET_CK(cudaFree(nullptr));
  SET_CK(setk::kernels_init());
  ctl_ = setk::slot_control_bytes(cfg.slot_bytes);
  if (cfg.stamps) {
    SET_CK(cudaMalloc(&clock_, sizeof(unsigned long long)));
    SET_CK(cudaMemset(clock_, 0, sizeof(unsigned long long)));
  }
  // arena mode: slots keep only the kernels' control state; payloads live in the arena
  const size_t stride = cfg.arena_bytes ? setk::align256(ctl_) : setk::align256(cfg.slot_bytes);
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
  if (cfg.arena_bytes) {
    if (cudaMalloc(&arena_, cfg.arena_bytes) != cudaSuccess) {
      cudaGetLastError();
      arena_ = nullptr;
      *err = "cudaMalloc of the arena failed (" + std::to_string(cfg.arena_bytes) + " bytes)";
      return SET_ENOMEM;
    }
  }
  SET_CK(cudaHostAlloc(&ph_host_, kPlaceholderBytes, cudaHostAllocDefault));
  SET_CK(cudaMalloc(&ph_dev_, kPlaceholderBytes));
  if (cfg.io_mode == SET_IO_DEVICE) {
    kind_in_ = cudaMemcpyDeviceToDevice;
    kind_out_ = cudaMemcpyDeviceToDevice;
  }
  lanes_.resize(cfg.num_streams);
  cbs_.resize(cfg.num_streams);
  for (int i = 0; i < cfg.num_streams; ++i) {
    SET_CK(cudaStreamCreateWithFlags(&lanes_[i], cudaStreamNonBlocking));
    SET_CK(cudaStreamCreateWithFlags(&cbs_[i], cudaStreamNonBlocking));
  }
  st_.resize(slots.size());
  for (auto& s : slots) {
    s.dev = static_cast<uint8_t*>(pool_) + stride * s.index;
    s.bytes = cfg.arena_bytes ? stride : cfg.slot_bytes;
    s.dev_state = &st_[s.index];
    SET_CK(cudaEventCreateWithFlags(&st_[s.index].done, cudaEventDisableTiming));
    if (cfg.stamps) {
      SlotState& ss = st_[s.index];
      SET_CK(cudaHostAlloc(reinterpret_cast<void**>(&ss.h_stamps), 2 * setk::kMaxKernels * sizeof(uint64_t),
                           cudaHostAllocMapped));
      SET_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ss.d_stamps), ss.h_stamps, 0));
      std::memset(ss.h_stamps, 0, 2 * setk::kMaxKernels * sizeof(uint64_t));
      s.stamps = ss.h_stamps;
    }
    s.job_mem = static_cast<uint8_t*>(arena_);  // templates point into the arena (never launched as built)
    for (uint32_t t = 1; t <= SET_NUM_JOB_TYPES; ++t) {
      if (!(cfg.type_mask & (1u << t))) continue;
      const set_status b = build_graph(s, t, err);
      if (b != SET_OK) return b;
    }
    if (cfg.batch_max > 1) {
      SET_CK(cudaHostAlloc(reinterpret_cast<void**>(&st_[s.index].h_table), kTableStaging, cudaHostAllocDefault));
      std::memset(st_[s.index].h_table, 0, kTableStaging);
      for (uint32_t t = 1; t <= SET_NUM_JOB_TYPES; ++t) {
        if (!(cfg.type_mask & (1u << t)) || !setk::batchable(t)) continue;
        const set_status b = build_batch_graph(s, t, err);
        if (b != SET_OK) return b;
      }
    }
    s.job_mem = nullptr;
  }
  for (uint32_t t = 1; t <= SET_NUM_JOB_TYPES; ++t) supported_[t] = st_.empty() ? false : st_[0].gi[t].exec != nullptr;
  SET_CK(cudaDeviceSynchronize());
  if (cfg.cb_mode == 3) poller_ = std::thread([this] { poll_main(); });
  return SET_OK;
}

bool CudaDevice::plan(const Slot& s, const JobRec& j, setk::JobLayout* L, setk::KernelLaunch* kl, int* nk) const {
  if (!setk::job_sizes(j.d.type, j.d.dims, L)) return false;
  uint8_t* base = s.job_mem ? s.job_mem : s.dev;
  if (cfg_.guards)
    setk::place_job_guarded(L, s.job_mem ? 0 : ctl_);
  else
    setk::place_job(L, s.job_mem ? 0 : ctl_);
  setk::JobPlanIn in;
  in.type = j.d.type;
  in.flags = j.d.flags;
  std::memcpy(in.dims, j.d.dims, sizeof in.dims);
  in.scalar = j.d.scalar;
  in.shared[0] = j.d.shared[0];
  in.shared[1] = j.d.shared[1];
  // mapped sides: the kernels address the job's host buffer directly
  in.d_in = io_maps_in(cfg_.io_mode) ? (j.d.in ? j.d.in : ph_dev_) : base + L->in_off;
  in.d_out = io_maps_out(cfg_.io_mode) ? (j.d.out ? j.d.out : ph_dev_) : base + L->out_off;
  in.d_scratch = base + L->scratch_off;
  in.d_persist = s.dev + setk::control_offset(j.d.type);
  in.job_id = j.id;
  in.slot_gen = s.gen;
  in.img_fused = cfg_.img_fused;
  in.stamps = stamp_base(s);
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
  if (!plan(s, rep, &L, kl, &nk)) return SET_OK;  // type without a planner in this library: no graph
  if ((!s.job_mem && L.end > s.bytes) || L.in_bytes > kPlaceholderBytes || L.out_bytes > kPlaceholderBytes)
    return SET_OK;
  uint8_t* base = s.job_mem ? s.job_mem : s.dev;
  GraphInst& gi = st_[s.index].gi[type];
  SET_CK(cudaGraphCreate(&gi.graph, 0));
  const bool copy_in = !io_maps_in(cfg_.io_mode), copy_out = !io_maps_out(cfg_.io_mode);
  const void* src_ph = cfg_.io_mode == SET_IO_DEVICE ? ph_dev_ : ph_host_;
  void* dst_ph = cfg_.io_mode == SET_IO_DEVICE ? ph_dev_ : ph_host_;
  setk::KernelLaunch gk[2];
  if (cfg_.guards) {  // arm the bands first: the H2D copy must not touch them either
    setk::plan_guards(base, L, false, &gk[0], &gk[1]);
    const cudaKernelNodeParams p = node_params(gk[0]);
    SET_CK(cudaGraphAddKernelNode(&gi.arm, gi.graph, nullptr, 0, &p));
  }
  if (copy_in && cfg_.sm_copies) {  // copy kernel over NVLink-C2C (set_config.sm_copies)
    setk::KernelLaunch ck;
    setk::plan_copy(base + L.in_off, ph_host_, L.in_bytes, &ck);
    const cudaKernelNodeParams p = node_params(ck);
    SET_CK(cudaGraphAddKernelNode(&gi.h2d, gi.graph, gi.arm ? &gi.arm : nullptr, gi.arm ? 1 : 0, &p));
  } else if (copy_in) {
    SET_CK(cudaGraphAddMemcpyNode1D(&gi.h2d, gi.graph, gi.arm ? &gi.arm : nullptr, gi.arm ? 1 : 0, base + L.in_off,
                                    src_ph, L.in_bytes, kind_in_));
  }
  uint32_t has_dependents = 0;
  for (int k = 0; k < nk; ++k) {
    cudaGraphNode_t deps[setk::kMaxKernels];
    size_t nd = 0;
    if (kl[k].deps == 0) {
      if (copy_in)
        deps[nd++] = gi.h2d;
      else if (gi.arm)
        deps[nd++] = gi.arm;
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
  if (cfg_.guards) {  // check after every stage kernel, before the D2H copy returns the trailer
    const cudaKernelNodeParams p = node_params(gk[1]);
    SET_CK(cudaGraphAddKernelNode(&gi.check, gi.graph, sinks, ns, &p));
    sinks[0] = gi.check;
    ns = 1;
  }
  if (copy_out && cfg_.sm_copies) {
    setk::KernelLaunch ck;
    setk::plan_copy(ph_host_, base + L.out_off, L.out_bytes, &ck);
    const cudaKernelNodeParams p = node_params(ck);
    SET_CK(cudaGraphAddKernelNode(&gi.d2h, gi.graph, sinks, ns, &p));
  } else if (copy_out) {
    SET_CK(cudaGraphAddMemcpyNode1D(&gi.d2h, gi.graph, sinks, ns, dst_ph, base + L.out_off, L.out_bytes, kind_out_));
  }
  if (cfg_.cb_mode == 2) {  // Algorithm 3's callback as the graph's last node, bound to this slot
    cudaHostNodeParams hp{};
    hp.fn = host_complete;
    hp.userData = &s;
    cudaGraphNode_t hn;
    if (copy_out)
      SET_CK(cudaGraphAddHostNode(&hn, gi.graph, &gi.d2h, 1, &hp));
    else
      SET_CK(cudaGraphAddHostNode(&hn, gi.graph, sinks, ns, &hp));
  }
  gi.nk = nk;
  SET_CK(cudaGraphInstantiate(&gi.exec, gi.graph, 0));
  SET_CK(cudaGraphUpload(gi.exec, lanes_[s.lane]));  // device-side setup now, not at the first job
  return SET_OK;
}

// UpdateGraphParams (Algorithms 1-2): rebind the exec's copies and kernels to this job.
set_status CudaDevice::update(const Slot& s, const JobRec& j, GraphInst& gi, LaunchCost* cost, std::string* err) {
  setk::JobLayout L;
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  setrt::set_thread_error("");
  const bool planned = plan(s, j, &L, kl, &nk);
  if (!planned || nk != gi.nk) {
    *err = std::string("job does not match its graph template (planned=") + (planned ? "1" : "0") +
           " nk=" + std::to_string(nk) + " template=" + std::to_string(gi.nk) + "): " + setrt::thread_error_text();
    return SET_EINVAL;
  }
  uint8_t* base = s.job_mem ? s.job_mem : s.dev;
  const uint64_t t0 = now_ns();
  arm_stamps(const_cast<Slot&>(s), kl, nk);
  const bool copy_in = !io_maps_in(cfg_.io_mode), copy_out = !io_maps_out(cfg_.io_mode);
  cudaError_t e = cudaSuccess;
  setk::KernelLaunch ck;
  if (copy_in && cfg_.sm_copies) {
    setk::plan_copy(base + L.in_off, j.d.in, L.in_bytes, &ck);
    const cudaKernelNodeParams p = node_params(ck);
    e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.h2d, &p);
  } else if (copy_in) {
    e = cudaGraphExecMemcpyNodeSetParams1D(gi.exec, gi.h2d, base + L.in_off, j.d.in, L.in_bytes, kind_in_);
  }
  if (e == cudaSuccess)
    for (int k = 0; k < nk && e == cudaSuccess; ++k) {
      const cudaKernelNodeParams p = node_params(kl[k]);
      e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.kn[k], &p);
    }
  if (e == cudaSuccess && copy_out && cfg_.sm_copies) {
    setk::plan_copy(j.d.out, base + L.out_off, L.out_bytes, &ck);
    const cudaKernelNodeParams p = node_params(ck);
    e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.d2h, &p);
  } else if (e == cudaSuccess && copy_out) {
    e = cudaGraphExecMemcpyNodeSetParams1D(gi.exec, gi.d2h, j.d.out, base + L.out_off, L.out_bytes, kind_out_);
  }
  if (e == cudaSuccess && gi.arm) {
    setk::KernelLaunch gk[2];
    setk::plan_guards(base, L, (j.d.flags & SET_F_TEST_GUARD) != 0, &gk[0], &gk[1]);
    cudaKernelNodeParams p = node_params(gk[0]);
    e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.arm, &p);
    if (e == cudaSuccess) {
      p = node_params(gk[1]);
      e = cudaGraphExecKernelNodeSetParams(gi.exec, gi.check, &p);
    }
    cost->updates += 2;
  }
  cost->update_ns += now_ns() - t0;
  cost->updates += (uint64_t)nk + (copy_in ? 1 : 0) + (copy_out ? 1 : 0);
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
set_status CudaDevice::attach_callback(Slot& s, std::string* err) {
  SlotState& ss = st_[s.index];
  cudaStream_t lane = lanes_[s.lane], cb = cbs_[s.lane];
  if (cfg_.cb_mode == 1) {
    SET_CK(cudaLaunchHostFunc(lane, host_complete, &s));
  } else if (cfg_.cb_mode == 3) {
    SET_CK(cudaEventRecord(ss.done, lane));
    poll_push(&s);
  } else {
    SET_CK(cudaEventRecord(ss.done, lane));
    SET_CK(cudaStreamWaitEvent(cb, ss.done, 0));
    SET_CK(cudaLaunchHostFunc(cb, host_complete, &s));
  }
  return SET_OK;
}

set_status CudaDevice::launch(Slot& s, bool callback, LaunchCost* cost, std::string* err) {
  GraphInst& gi = st_[s.index].gi[s.job.d.type];
  if (!gi.exec) {
    *err = "job type not instantiated";
    return SET_EINVAL;
  }
  const set_status u = update(s, s.job, gi, cost, err);
  if (u != SET_OK) return u;
  return launch_bound(s, callback, cost, err);
}

// Bind-at-submit: UpdateGraphParams on the submitting thread (its current device is kept).
set_status CudaDevice::prepare(Slot& s, LaunchCost* cost, std::string* err) {
  GraphInst& gi = st_[s.index].gi[s.job.d.type];
  if (!gi.exec) {
    *err = "job type not instantiated";
    return SET_EINVAL;
  }
  int old = -1;
  if (cudaGetDevice(&old) != cudaSuccess) cudaGetLastError();
  SET_CK(cudaSetDevice(cfg_.device));  // makes the context current for driver calls of the planners
  const set_status u = update(s, s.job, gi, cost, err);
  if (old >= 0 && old != cfg_.device) cudaSetDevice(old);
  return u;
}

// GraphLaunch of the slot's (already rebound) graph on its lane, and AddCallback.
set_status CudaDevice::launch_bound(Slot& s, bool callback, LaunchCost* cost, std::string* err) {
  GraphInst& gi = st_[s.index].gi[s.job.d.type];
  const uint64_t t1 = now_ns();
  SET_CK(cudaGraphLaunch(gi.exec, lanes_[s.lane]));
  // cb_mode 2: the graph's own host node runs the completion path
  if (cfg_.cb_mode != 2 && callback) {
    const set_status a = attach_callback(s, err);
    if (a != SET_OK) return a;
  }
  cost->launch_ns += now_ns() - t1;
  return SET_OK;
}

bool CudaDevice::plan_batch(Slot& s, const setk::BatchItem* items, int nb, const setk::BatchLayout& L,
                            uint8_t* d_block, const void* const shared[2], setk::KernelLaunch* kl, int* nk) {
  SlotState& ss = st_[s.index];
  if (L.table_bytes > kTableStaging) return false;
  if (items && nb > 0 && L.nb == nb) {
    // the type was fixed when the layout was made: image and MLP tables differ in shape
    const bool ok =
        L.rows ? setk::plan_mlp_batch(items, nb, L, d_block, ss.h_table, s.gen, shared[0], shared[1], kl, nk)
               : setk::plan_img_batch(items, nb, L, d_block, ss.h_table, s.gen, img_ctas_.load(), img_tile_.load(), kl,
                                      nk);
    if (ok)
      for (int k = 0; k < *nk; ++k) setk::attach_stamp(kl[k], stamp_base(s), k);
    return ok;
  }
  return false;
}

// Batch graph of one type bound to one slot: table -> {job H2D x kMaxBatch} -> packed kernels ->
// {job D2H x kMaxBatch}.  Built with placeholders; every launch rebinds the used positions and
// disables the rest.
set_status CudaDevice::build_batch_graph(Slot& s, uint32_t type, std::string* err) {
  SlotState& ss = st_[s.index];
  BatchGraph& bg = ss.bg[type];
  setk::BatchItem it{};
  uint32_t d[4];
  template_dims(type, d);
  std::memcpy(it.dims, d, sizeof d);
  setk::BatchLayout L;
  if (!setk::batch_layout(type, &it, 1, &L)) return SET_OK;
  uint8_t* d_block = s.job_mem ? s.job_mem : s.dev + ctl_;
  if (!s.job_mem && ctl_ + L.block_bytes > s.bytes) return SET_OK;  // slot too small for any batch
  const void* shared[2] = {ph_dev_, ph_dev_};
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  if (!plan_batch(s, &it, 1, L, d_block, shared, kl, &nk)) return SET_OK;
  const int B = cfg_.batch_max;
  SET_CK(cudaGraphCreate(&bg.graph, 0));
  SET_CK(cudaGraphAddMemcpyNode1D(&bg.table, bg.graph, nullptr, 0, d_block, ss.h_table, L.table_bytes,
                                  cudaMemcpyHostToDevice));
  const void* src_ph = cfg_.io_mode == SET_IO_HOST ? ph_host_ : ph_dev_;
  void* dst_ph = cfg_.io_mode == SET_IO_HOST ? ph_host_ : ph_dev_;
  bg.h2d.assign(B, nullptr);
  bg.d2h.assign(B, nullptr);
  bg.on.assign(B, 1);
  for (int j = 0; j < B; ++j)
    SET_CK(cudaGraphAddMemcpyNode1D(&bg.h2d[j], bg.graph, nullptr, 0, d_block + L.in_off[0], src_ph, 256, kind_in_));
  std::vector<cudaGraphNode_t> roots(bg.h2d);
  roots.push_back(bg.table);
  uint32_t has_dependents = 0;
  for (int k = 0; k < nk; ++k) {
    std::vector<cudaGraphNode_t> deps;
    if (kl[k].deps == 0) {
      deps = roots;
    } else {
      for (int q = 0; q < k; ++q)
        if (kl[k].deps & (1u << q)) {
          deps.push_back(bg.kn[q]);
          has_dependents |= 1u << q;
        }
    }
    const cudaKernelNodeParams p = node_params(kl[k]);
    SET_CK(cudaGraphAddKernelNode(&bg.kn[k], bg.graph, deps.data(), deps.size(), &p));
  }
  std::vector<cudaGraphNode_t> sinks;
  for (int k = 0; k < nk; ++k)
    if (!(has_dependents & (1u << k))) sinks.push_back(bg.kn[k]);
  for (int j = 0; j < B; ++j)
    SET_CK(cudaGraphAddMemcpyNode1D(&bg.d2h[j], bg.graph, sinks.data(), sinks.size(), dst_ph, d_block + L.out_off[0],
                                    256, kind_out_));
  bg.nk = nk;
  SET_CK(cudaGraphInstantiate(&bg.exec, bg.graph, 0));
  SET_CK(cudaGraphUpload(bg.exec, lanes_[s.lane]));
  return SET_OK;
}

set_status CudaDevice::launch_batch(Slot& s, bool callback, LaunchCost* cost, std::string* err) {
  SlotState& ss = st_[s.index];
  const uint32_t type = s.batch[0].d.type;
  BatchGraph& bg = ss.bg[type];
  const int nb = (int)s.batch.size();
  if (!bg.exec || nb > (int)bg.h2d.size()) {
    *err = "no batch graph for this job type (batch_max, slot_bytes)";
    return SET_EINVAL;
  }
  setk::BatchItem items[setk::kMaxBatch];
  for (int j = 0; j < nb; ++j) {
    std::memcpy(items[j].dims, s.batch[j].d.dims, sizeof items[j].dims);
    items[j].job_id = s.batch[j].id;
  }
  setk::BatchLayout L;
  uint8_t* d_block = batch_block(s);
  setk::KernelLaunch kl[setk::kMaxKernels];
  int nk = 0;
  const uint64_t t0 = now_ns();
  if (!setk::batch_layout(type, items, nb, &L) ||
      !plan_batch(s, items, nb, L, d_block, s.batch[0].d.shared, kl, &nk) || nk != bg.nk) {
    *err = std::string("batch does not match its graph template: ") + setrt::thread_error_text();
    return SET_EINVAL;
  }
  arm_stamps(s, kl, nk);
  cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(bg.exec, bg.table, d_block, ss.h_table, L.table_bytes,
                                                     cudaMemcpyHostToDevice);
  for (int j = 0; j < (int)bg.h2d.size() && e == cudaSuccess; ++j) {
    const bool use = j < nb;
    if (use) {
      const JobRec& jr = s.batch[j];
      e = cudaGraphExecMemcpyNodeSetParams1D(bg.exec, bg.h2d[j], d_block + L.in_off[j], jr.d.in, L.in_bytes[j], kind_in_);
      if (e == cudaSuccess)
        e = cudaGraphExecMemcpyNodeSetParams1D(bg.exec, bg.d2h[j], jr.d.out, d_block + L.out_off[j], L.out_bytes[j],
                                               kind_out_);
      cost->updates += 2;
    }
    if (e == cudaSuccess && bg.on[j] != (char)use) {
      e = cudaGraphNodeSetEnabled(bg.exec, bg.h2d[j], use);
      if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(bg.exec, bg.d2h[j], use);
      bg.on[j] = (char)use;
      cost->updates += 2;
    }
  }
  for (int k = 0; k < nk && e == cudaSuccess; ++k) {
    const cudaKernelNodeParams p = node_params(kl[k]);
    e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.kn[k], &p);
    cost->updates += 1;
  }
  cost->update_ns += now_ns() - t0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("batch graph update rejected: ") + cudaGetErrorString(e);
    return SET_EINVAL;
  }
  const uint64_t t1 = now_ns();
  SET_CK(cudaGraphLaunch(bg.exec, lanes_[s.lane]));
  if (callback) {
    const set_status a = attach_callback(s, err);
    if (a != SET_OK) return a;
  }
  cost->launch_ns += now_ns() - t1;
  return SET_OK;
}

// Autotuner: every candidate runs the whole sample in batches of B consecutive jobs; per batch the
// inputs and the table are copied in untimed, and CUDA events bracket the packed kernels only.
set_status CudaDevice::autotune(uint32_t type, const JobRec* sample, size_t n, int max_batch, set_tune_result* out,
                                std::string* err) {
  if (st_.empty() || !st_[0].h_table) {
    *err = "autotune needs a context created with batch_max > 1";
    return SET_EINVAL;
  }
  Slot probe;  // a stand-in slot: generation 0, staging of slot 0 (the context is idle)
  probe.index = 0;
  std::vector<int> Bs;
  for (int b = 1; b <= max_batch && b <= (int)n; b *= 2) Bs.push_back(b);
  std::vector<int> tiles = {0}, ctas = {img_ctas_.load()};
  if (type == SET_JOB_IMG_SOBEL_HIST) {
    tiles = {0, 1, 2};
    ctas = {1, 2, 4, 8};
  }
  // scratch block: the largest batch of any candidate
  size_t need = 0;
  std::vector<setk::BatchItem> items(n);
  for (size_t i = 0; i < n; ++i) {
    std::memcpy(items[i].dims, sample[i].d.dims, sizeof items[i].dims);
    items[i].job_id = sample[i].id;
  }
  for (int B : Bs)
    for (size_t b0 = 0; b0 < n; b0 += B) {
      setk::BatchLayout L;
      if (!setk::batch_layout(type, &items[b0], (int)std::min<size_t>(B, n - b0), &L)) {
        *err = "autotune: invalid sample";
        return SET_EINVAL;
      }
      need = std::max(need, L.block_bytes);
    }
  uint8_t* blk = nullptr;
  SET_CK(cudaMalloc(&blk, need));
  cudaStream_t st = lanes_[0];
  cudaEvent_t e0, e1;
  SET_CK(cudaEventCreate(&e0));
  SET_CK(cudaEventCreate(&e1));
  const int tile0 = img_tile_.load(), cta0 = img_ctas_.load();
  double best = 0, single = 0;
  int cands = 0;
  set_tune_result res{};
  set_status rs = SET_OK;
  std::vector<double> by_b(Bs.size(), 0.0);
  std::vector<set_tune_result> best_of_b(Bs.size());
  for (size_t bi = 0; bi < Bs.size() && rs == SET_OK; ++bi) {
    const int B = Bs[bi];
    for (int tile : tiles)
      for (int c : ctas) {
        img_tile_.store(tile);
        img_ctas_.store(c);
        double best_ms = 1e30;
        for (int rep = 0; rep < 2 && rs == SET_OK; ++rep) {
          double ms_total = 0;
          for (size_t b0 = 0; b0 < n && rs == SET_OK; b0 += B) {
            const int nb = (int)std::min<size_t>(B, n - b0);
            setk::BatchLayout L;
            setk::batch_layout(type, &items[b0], nb, &L);
            setk::KernelLaunch kl[setk::kMaxKernels];
            int nk = 0;
            if (!plan_batch(probe, &items[b0], nb, L, blk, sample[b0].d.shared, kl, &nk)) {
              *err = std::string("autotune: plan failed: ") + setrt::thread_error_text();
              rs = SET_EINVAL;
              break;
            }
            cudaError_t ce = cudaMemcpyAsync(blk, st_[0].h_table, L.table_bytes, cudaMemcpyHostToDevice, st);
            for (int j = 0; j < nb && ce == cudaSuccess; ++j)
              ce = cudaMemcpyAsync(blk + L.in_off[j], sample[b0 + j].d.in, L.in_bytes[j], cudaMemcpyDefault, st);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
            for (int k = 0; k < nk && ce == cudaSuccess; ++k)
              ce = cudaLaunchKernel(kl[k].func, kl[k].grid, kl[k].block, kl[k].params, kl[k].smem, st);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) {
              *err = std::string("autotune: ") + cudaGetErrorString(ce);
              rs = SET_ECUDA;
              break;
            }
            ms_total += ms;
          }
          best_ms = std::min(best_ms, ms_total);
        }
        if (rs != SET_OK) break;
        ++cands;
        const double jps = (double)n / (best_ms * 1e-3);
        if (B == 1) single = std::max(single, jps);
        if (jps > by_b[bi]) {
          by_b[bi] = jps;
          best_of_b[bi].batch_max = B;
          best_of_b[bi].img_tile = tile;
          best_of_b[bi].img_ctas_per_sm = c;
          best_of_b[bi].jobs_per_s = jps;
        }
        best = std::max(best, jps);
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(blk);
  if (rs != SET_OK) {
    img_tile_.store(tile0);
    img_ctas_.store(cta0);
    return rs;
  }
  for (size_t bi = 0; bi < Bs.size(); ++bi)  // smallest batch within 5% of the best
    if (by_b[bi] >= 0.95 * best) {
      res = best_of_b[bi];
      break;
    }
  res.candidates = cands;
  res.single_jobs_per_s = single;
  img_tile_.store(res.img_tile);
  img_ctas_.store(res.img_ctas_per_sm);
  *out = res;
  return SET_OK;
}

void CudaDevice::drain() {
  for (auto s : lanes_) cudaStreamSynchronize(s);
  for (auto s : cbs_) cudaStreamSynchronize(s);
  // cb_mode 3: every recorded event has completed; let the completion thread hand them back
  for (int i = 0; i < 100000 && poll_pending_.load() > 0; ++i) std::this_thread::sleep_for(std::chrono::microseconds(100));
}

void CudaDevice::release() {
  drain();
  if (poller_.joinable()) {
    poll_stop_.store(true);
    poll_sig_.notify_all();
    poller_.join();
  }
  for (auto& ss : st_) {
    for (auto& gi : ss.gi) {
      if (gi.exec) cudaGraphExecDestroy(gi.exec);
      if (gi.graph) cudaGraphDestroy(gi.graph);
    }
    for (auto& bg : ss.bg) {
      if (bg.exec) cudaGraphExecDestroy(bg.exec);
      if (bg.graph) cudaGraphDestroy(bg.graph);
    }
    if (ss.h_table) cudaFreeHost(ss.h_table);
    if (ss.h_stamps) cudaFreeHost(ss.h_stamps);
    if (ss.done) cudaEventDestroy(ss.done);
  }
  st_.clear();
  for (auto s : lanes_) cudaStreamDestroy(s);
  for (auto s : cbs_) cudaStreamDestroy(s);
  lanes_.clear();
  cbs_.clear();
  if (own_pool_ && pool_) cudaFree(pool_);
  pool_ = nullptr;
  if (arena_) cudaFree(arena_);
  arena_ = nullptr;
  if (clock_) cudaFree(clock_);
  clock_ = nullptr;
  if (ph_host_) cudaFreeHost(ph_host_);
  if (ph_dev_) cudaFree(ph_dev_);
  ph_host_ = ph_dev_ = nullptr;
}

// Baselines of Sec. 5.1.3 on the same kernels and slots.
//  SET_BASE_SYNC: one stream, one slot; per job cudaMemcpyAsync H2D, plain kernel launches,
//    cudaMemcpyAsync D2H, stream-ordered, no host synchronisation between jobs.
//  SET_BASE_BATCH_SYNC: b lanes with one graph exec each (ring entry 0); per batch of up to b jobs
//    update every exec, launch all, then cudaStreamSynchronize every lane before the next batch.
//    With arrival times, a batch holds the jobs that have arrived when it starts (at least one).
//  In arena mode each lane borrows one arena block sized for the largest job for the whole run.
set_status CudaDevice::run_baseline(int kind, const JobRec* jobs, size_t n, std::vector<Slot>& slots,
                                    BuddyArena* arena, LogHist* lat, LaunchCost* cost, uint64_t* t0, uint64_t* t1,
                                    std::string* err) {
  const size_t L = lanes_.size();
  const size_t nlanes = kind == SET_BASE_SYNC ? 1 : L;
  size_t need = 0;
  for (size_t i = 0; i < n; ++i) need = std::max(need, Executor::job_block_bytes(jobs[i].d));
  std::vector<std::pair<uint8_t*, size_t>> blocks;
  if (arena) {
    for (size_t i = 0; i < nlanes; ++i) {
      size_t bb = 0;
      uint8_t* p = arena->alloc(need, &bb);
      if (!p) {
        for (auto& b : blocks) arena->free(b.first, b.second);
        *err = "baseline: arena too small for one block per lane";
        return SET_ENOMEM;
      }
      blocks.push_back({p, bb});
      slots[i].job_mem = p;
    }
  }
  auto release = [&] {
    for (size_t i = 0; i < blocks.size(); ++i) {
      slots[i].job_mem = nullptr;
      arena->free(blocks[i].first, blocks[i].second);
    }
  };
  set_status result = SET_OK;
  if (kind == SET_BASE_SYNC) {
    Slot& s = slots[0];
    cudaStream_t st = lanes_[0];
    *t0 = now_ns();
    for (size_t i = 0; i < n && result == SET_OK; ++i) {
      const JobRec& j = jobs[i];
      if (j.d.t_arrival_ns) wait_until_ns(j.d.t_arrival_ns);
      setk::JobLayout Lo;
      setk::KernelLaunch kl[setk::kMaxKernels];
      int nk = 0;
      if (!plan(s, j, &Lo, kl, &nk)) {
        *err = "invalid job";
        result = SET_EINVAL;
        break;
      }
      uint8_t* base = s.job_mem ? s.job_mem : s.dev;
      const uint64_t ta = now_ns();
      cudaError_t e = cudaMemcpyAsync(base + Lo.in_off, j.d.in, Lo.in_bytes, kind_in_, st);
      for (int k = 0; k < nk && e == cudaSuccess; ++k)
        e = cudaLaunchKernel(kl[k].func, kl[k].grid, kl[k].block, kl[k].params, kl[k].smem, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(j.d.out, base + Lo.out_off, Lo.out_bytes, kind_out_, st);
      cost->launch_ns += now_ns() - ta;
      if (e != cudaSuccess) {
        *err = std::string("baseline launch: ") + cudaGetErrorString(e);
        result = SET_ECUDA;
      }
      s.gen += 1;
    }
    if (result == SET_OK && cudaStreamSynchronize(st) != cudaSuccess) result = SET_ECUDA;
    *t1 = now_ns();
    if (arena) release();
    return result;
  }
  if (kind == SET_BASE_BATCH_SYNC) {
    *t0 = now_ns();
    size_t base = 0;
    while (base < n && result == SET_OK) {
      const uint64_t first = jobs[base].d.t_arrival_ns;
      if (first) wait_until_ns(first);
      size_t nb = 1;
      const uint64_t now = now_ns();
      while (nb < L && base + nb < n && jobs[base + nb].d.t_arrival_ns <= now) ++nb;
      for (size_t i = 0; i < nb && result == SET_OK; ++i) {
        Slot& s = slots[i];  // ring entry 0 of lane i
        const JobRec& j = jobs[base + i];
        GraphInst& gi = st_[s.index].gi[j.d.type];
        if (!gi.exec) {
          *err = "job type not instantiated";
          result = SET_EINVAL;
          break;
        }
        result = update(s, j, gi, cost, err);
        if (result != SET_OK) break;
        const uint64_t ta = now_ns();
        if (cudaGraphLaunch(gi.exec, lanes_[i]) != cudaSuccess) result = SET_ECUDA;
        cost->launch_ns += now_ns() - ta;
      }
      for (size_t i = 0; i < nb; ++i)
        if (cudaStreamSynchronize(lanes_[i]) != cudaSuccess) result = SET_ECUDA;
      const uint64_t tb = now_ns();
      for (size_t i = 0; i < nb; ++i) {
        const uint64_t arrival = jobs[base + i].d.t_arrival_ns ? jobs[base + i].d.t_arrival_ns : *t0;
        lat->record(tb > arrival ? tb - arrival : 0);
        slots[i].gen += 1;
      }
      base += nb;
    }
    *t1 = now_ns();
    if (arena) release();
    if (result == SET_ECUDA && err->empty()) *err = "baseline: CUDA error";
    return result;
  }
  if (arena) release();
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
    int dev = 0;  // make the current device's context current on this thread (driver calls need it)
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess || cudaFree(nullptr) != cudaSuccess ||
        setk::kernels_init() != cudaSuccess)
      return SET_ECUDA;
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
  in.img_fused = (job->flags & SET_F_PER_STAGE) ? 0 : 1;
  in.flags = job->flags;
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
  if (!gbs || bytes == 0 || streams < 1 || reps < 1 || dir < 0 || dir > 5) return SET_EINVAL;
  const bool sm = dir >= 3;  // copy kernels (set_config.sm_copies) instead of the copy engines
  const int way = dir % 3;
  // successive copies use distinct buffers, up to a working set of 256 MiB per direction (more
  // than L2), so that no copy reads data an earlier one left in the GPU's cache
  const size_t stride = (bytes + 255) & ~size_t(255);
  const size_t nbuf = std::max<size_t>(1, std::min<size_t>((size_t)reps, ((size_t)256 << 20) / stride + 1));
  std::vector<cudaStream_t> ss(streams, nullptr);
  uint8_t *h_in = nullptr, *h_out = nullptr, *d_in = nullptr, *d_out = nullptr;
  set_status st = SET_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && st == SET_OK) st = SET_ECUDA;
    return e == cudaSuccess;
  };
  for (int i = 0; i < streams && st == SET_OK; ++i) ok(cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
  ok(cudaHostAlloc(reinterpret_cast<void**>(&h_in), nbuf * stride, cudaHostAllocDefault));
  ok(cudaHostAlloc(reinterpret_cast<void**>(&h_out), nbuf * stride, cudaHostAllocDefault));
  ok(cudaMalloc(reinterpret_cast<void**>(&d_in), nbuf * stride));
  ok(cudaMalloc(reinterpret_cast<void**>(&d_out), nbuf * stride));
  ok(cudaEventCreate(&e0));
  ok(cudaEventCreate(&e1));
  if (st == SET_OK) {
    for (int pass = 0; pass < 2 && st == SET_OK; ++pass) {  // pass 0 warms up
      ok(cudaDeviceSynchronize());
      ok(cudaEventRecord(e0, ss[0]));
      for (int i = 1; i < streams; ++i) ok(cudaStreamWaitEvent(ss[i], e0, 0));
      for (int r = 0; r < reps; ++r) {
        const int i = r % streams;
        const size_t off = (size_t)(r % nbuf) * stride;
        if (sm) {
          setk::KernelLaunch k;
          if (way != 1) {
            setk::plan_copy(d_in + off, h_in + off, bytes, &k);
            ok(cudaLaunchKernel(k.func, k.grid, k.block, k.params, 0, ss[i]));
          }
          if (way != 0) {
            setk::plan_copy(h_out + off, d_out + off, bytes, &k);
            ok(cudaLaunchKernel(k.func, k.grid, k.block, k.params, 0, ss[i]));
          }
          continue;
        }
        if (way != 1) ok(cudaMemcpyAsync(d_in + off, h_in + off, bytes, cudaMemcpyHostToDevice, ss[i]));
        if (way != 0) ok(cudaMemcpyAsync(h_out + off, d_out + off, bytes, cudaMemcpyDeviceToHost, ss[i]));
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
      *gbs = (double)bytes * reps * (way == 2 ? 2.0 : 1.0) / ((double)ms * 1e-3) / 1e9;
  }
  for (int i = 0; i < streams; ++i)
    if (ss[i]) cudaStreamDestroy(ss[i]);
  if (h_in) cudaFreeHost(h_in);
  if (h_out) cudaFreeHost(h_out);
  if (d_in) cudaFree(d_in);
  if (d_out) cudaFree(d_out);
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
