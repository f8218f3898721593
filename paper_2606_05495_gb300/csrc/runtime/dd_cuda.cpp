// dd_cuda.cpp -- CUDA backend of the device-dispatch lanes (dd_backend.h).
//
// Per lane: a non-blocking stream, an event recorded behind each launch, and one graph built and
// uploaded once:  WHILE(loop, 1 at each launch) { fetch kernel -> SWITCH(kind) { [0] blur lane
// kernel, [1] scan lane kernel (each a batch of up to kDdBatch jobs), [2] image lane kernel } }.
// The rings, control lines and completion words live in one page-locked host block mapped into
// the GPU's address space; the lanes' device blocks (fetched arguments, scan look-back state) in
// one device allocation.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "../kernels/stages.h"
#include "dd_backend.h"
#include "layout.h"

namespace setrt {
namespace {

#define DD_CK(call)                                                               \
  do {                                                                            \
    const cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                      \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return SET_ECUDA;                                                           \
    }                                                                             \
  } while (0)

struct CudaLane {
  cudaStream_t stream = nullptr;
  cudaEvent_t ended = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  setk::DdLaneDev* dev = nullptr;
};

class CudaDdBackend final : public DdBackend {
 public:
  ~CudaDdBackend() override { release(false); }

  set_status init(const set_dd_config& cfg, uint32_t depth, std::vector<DdLaneMem>* lanes, std::string* err) override {
    cfg_ = cfg;
    depth_ = depth;
    DD_CK(cudaSetDevice(cfg.device));
    DD_CK(cudaFree(nullptr));
    DD_CK(setk::kernels_init());
    {
      void* fp = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fp, 12000, cudaEnableDefault, &q) == cudaSuccess &&
          q == cudaDriverEntryPointSuccess)
        range_fn_ = reinterpret_cast<int (*)(unsigned long long*, size_t*, unsigned long long)>(fp);
      else
        cudaGetLastError();
    }
    const uint32_t nl = (uint32_t)cfg.num_lanes;
    const size_t ring_bytes = (size_t)depth * sizeof(setk::DdEntry);
    const size_t cmpl_bytes = setk::align256((size_t)depth * sizeof(uint32_t));
    const size_t host_lane = ring_bytes + sizeof(setk::DdCtl) + cmpl_bytes;
    const size_t host_total = host_lane * nl;
    if (cudaHostAlloc(&host_block_, host_total, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      host_block_ = nullptr;
      *err = "cudaHostAlloc of the descriptor rings failed (" + std::to_string(host_total) + " bytes)";
      return SET_ENOMEM;
    }
    std::memset(host_block_, 0, host_total);
    setk::JobLayout SL;
    const uint32_t sd[4] = {cfg.scan_max_n, 0, 0, 0};
    if (!setk::job_sizes(SET_JOB_SAXPY_SCAN_MAX, sd, &SL)) {
      *err = "scan_max_n rejected by the scan layout";
      return SET_EINVAL;
    }
    setk::JobLayout IL;
    const uint32_t id[4] = {1, 1, 0, 0};
    if (!setk::job_sizes(SET_JOB_IMG_SOBEL_HIST, id, &IL)) {
      *err = "image layout unavailable";
      return SET_EINVAL;
    }
    const size_t lane_dev = setk::align256(sizeof(setk::DdLaneDev));
    // kDdBatch look-back areas: scan job j of a batch uses area j
    scan_stride_ = setk::align256(SL.persist_bytes);
    const size_t scratch = scan_stride_ * setk::kDdBatch;
    const size_t img_state = setk::align256(IL.persist_bytes);
    const size_t dev_total = (lane_dev + scratch + img_state) * nl;
    if (cudaMalloc(&dev_block_, dev_total) != cudaSuccess) {
      cudaGetLastError();
      dev_block_ = nullptr;
      *err = "cudaMalloc of the lane state failed (" + std::to_string(dev_total) + " bytes)";
      return SET_ENOMEM;
    }
    DD_CK(cudaMemset(dev_block_, 0, dev_total));
    lanes->assign(nl, DdLaneMem{});
    lanes_.assign(nl, CudaLane{});
    for (uint32_t i = 0; i < nl; ++i) {
      uint8_t* hb = static_cast<uint8_t*>(host_block_) + host_lane * i;
      uint8_t* db = static_cast<uint8_t*>(dev_block_);
      DdLaneMem& m = (*lanes)[i];
      m.ring = reinterpret_cast<setk::DdEntry*>(hb);
      m.ctl = reinterpret_cast<setk::DdCtl*>(hb + ring_bytes);
      m.cmpl = reinterpret_cast<uint32_t*>(hb + ring_bytes + sizeof(setk::DdCtl));
      m.scan_scratch = db + lane_dev * nl + scratch * i;
      m.img_state = db + (lane_dev + scratch) * nl + img_state * i;
      lanes_[i].dev = reinterpret_cast<setk::DdLaneDev*>(db + lane_dev * i);
      const set_status st = build_lane(i, m, err);
      if (st != SET_OK) return st;
    }
    lane_mem_ = *lanes;
    DD_CK(cudaDeviceSynchronize());  // uploads and memsets done before the first descriptor
    return SET_OK;
  }

  bool plan(const set_job_desc& d, uint64_t job_id, uint32_t lane, unsigned char* args, uint32_t* args_size) override {
    const DdLaneMem& m = lane_mem_[lane];
    setk::JobPlanIn in;
    in.type = d.type;
    in.flags = d.flags;
    std::memcpy(in.dims, d.dims, sizeof in.dims);
    in.scalar = d.scalar;
    in.d_in = d.in;
    in.d_out = d.out;
    in.job_id = job_id;
    in.slot_gen = lane;
    if (d.type == SET_JOB_IMG_SOBEL_HIST) {  // ticket mode over the lane's fixed grid
      in.d_persist = m.img_state;
      return setk::plan_img_lane(in, args, args_size);
    }
    in.d_persist = m.scan_scratch;
    setk::KernelLaunch kl[setk::kMaxKernels];
    int nk = 0;
    if (!setk::plan_job(in, kl, &nk) || nk != 1 || kl[0].args_size > setk::kDdArgBytes) return false;
    std::memcpy(args, kl[0].args, kl[0].args_size);
    *args_size = (uint32_t)kl[0].args_size;
    return true;
  }

  // Device memory of the object's GPU (the lanes' kernels read and write the buffers in place);
  // where the driver reports the allocation's range, the whole buffer must lie inside it, and the
  // range is remembered for the rest of the submit call.
  bool buffer_ok(const void* p, size_t bytes, DdRangeCache* cache) const override {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (cache && cache->has(a, bytes)) return true;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeDevice || at.device != cfg_.device) return false;
    unsigned long long base = 0;
    size_t size = 0;
    if (!range_fn_ || range_fn_(&base, &size, (unsigned long long)a) != 0) return true;  // start checked only
    if (a < base || bytes > base + size - a) return false;  // runs past the end of its allocation
    if (cache) cache->add((uintptr_t)base, (uintptr_t)(base + size));
    return true;
  }

  set_status launch(uint32_t lane, std::string* err) override {
    CudaLane& l = lanes_[lane];
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != cfg_.device) cudaSetDevice(cfg_.device);
    cudaError_t e = cudaGraphLaunch(l.exec, l.stream);
    if (e == cudaSuccess) e = cudaEventRecord(l.ended, l.stream);
    if (prev >= 0 && prev != cfg_.device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("lane graph launch: ") + cudaGetErrorString(e);
      return SET_ECUDA;
    }
    return SET_OK;
  }

  int ended(uint32_t lane, std::string* err) override {
    const cudaError_t q = cudaEventQuery(lanes_[lane].ended);
    if (q == cudaSuccess) return 1;
    if (q == cudaErrorNotReady) return 0;
    cudaGetLastError();
    *err = std::string("lane graph: ") + cudaGetErrorString(q);
    return -1;
  }

  void bind_thread() override { cudaSetDevice(cfg_.device); }

  void release(bool leak) override {
    if (leak) leaked_ = true;
    if (leaked_) return;  // a loop may still use the memory
    for (auto& l : lanes_) {
      if (l.ended) cudaEventDestroy(l.ended);
      if (l.exec) cudaGraphExecDestroy(l.exec);
      if (l.graph) cudaGraphDestroy(l.graph);
      if (l.stream) cudaStreamDestroy(l.stream);
      l = CudaLane{};
    }
    if (dev_block_) cudaFree(dev_block_);
    if (host_block_) cudaFreeHost(host_block_);
    dev_block_ = nullptr;
    host_block_ = nullptr;
  }

 private:
  set_status build_lane(uint32_t i, const DdLaneMem& m, std::string* err) {
    CudaLane& l = lanes_[i];
    DD_CK(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
    DD_CK(cudaEventCreateWithFlags(&l.ended, cudaEventDisableTiming));
    DD_CK(cudaGraphCreate(&l.graph, 0));
    cudaGraphConditionalHandle hloop = 0, hkind = 0;
    DD_CK(cudaGraphConditionalHandleCreate(&hloop, l.graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hloop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    DD_CK(cudaGraphAddNode(&wn, l.graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // the fetch kernel sets the selector before the SWITCH node reads it in every iteration
    DD_CK(cudaGraphConditionalHandleCreate(&hkind, body, setk::kDdKindNone, 0));

    // device-usable addresses of this lane's host-side structures
    void* ring_d = nullptr;
    void* ctl_d = nullptr;
    void* cmpl_d = nullptr;
    DD_CK(cudaHostGetDevicePointer(&ring_d, m.ring, 0));
    DD_CK(cudaHostGetDevicePointer(&ctl_d, m.ctl, 0));
    DD_CK(cudaHostGetDevicePointer(&cmpl_d, m.cmpl, 0));
    setk::DdFetchArgs fa{};
    fa.lane = l.dev;
    fa.ring = static_cast<const setk::DdEntry*>(ring_d);
    fa.ctl = static_cast<setk::DdCtl*>(ctl_d);
    fa.cmpl = static_cast<uint32_t*>(cmpl_d);
    fa.depth = depth_;
    fa.idle_ns = (uint64_t)cfg_.idle_us * 1000ull;
    fa.loop = hloop;
    fa.kind = hkind;
    void* fargs[1] = {&fa};
    cudaKernelNodeParams fp{};
    fp.func = const_cast<void*>(setk::dd_fetch_func());
    fp.gridDim = dim3(1);
    fp.blockDim = dim3(32);
    fp.kernelParams = fargs;
    cudaGraphNode_t fn = nullptr;
    DD_CK(cudaGraphAddKernelNode(&fn, body, nullptr, 0, &fp));

    cudaGraphNodeParams sp{};
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = hkind;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = setk::kDdKinds;
    cudaGraphNode_t sn = nullptr;
    DD_CK(cudaGraphAddNode(&sn, body, &fn, nullptr, 1, &sp));

    // the blur and scan nodes read the batch's argument areas and job count
    const void* batch_args = l.dev->batch_args[0];
    const void* batch_count = &l.dev->batch_count;
    uint32_t scan_tmax = setk::scan_lane_tiles(cfg_.scan_max_n);
    uint64_t scan_stride = scan_stride_;
    void* bargs[2] = {&batch_args, &batch_count};
    void* sargs[4] = {&batch_args, &batch_count, &scan_tmax, &scan_stride};
    cudaKernelNodeParams bp{};
    bp.func = const_cast<void*>(setk::blur_lane_func());
    bp.gridDim = dim3(8 * setk::kDdBatch);  // one 8-CTA cluster per job of a batch
    bp.blockDim = dim3(256);
    bp.sharedMemBytes = setk::blur_lane_smem(cfg_.blur_max_w);
    bp.kernelParams = bargs;
    cudaGraphNode_t bn = nullptr;
    DD_CK(cudaGraphAddKernelNode(&bn, sp.conditional.phGraph_out[setk::kDdKindBlur], nullptr, 0, &bp));
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(setk::scan_lane_func());
    kp.gridDim = dim3(scan_tmax * setk::kDdBatch);
    kp.blockDim = dim3(256);
    kp.kernelParams = sargs;
    cudaGraphNode_t kn = nullptr;
    DD_CK(cudaGraphAddKernelNode(&kn, sp.conditional.phGraph_out[setk::kDdKindScan], nullptr, 0, &kp));
    const void* img_args = l.dev->args[setk::kDdKindImg];
    void* iargs[1] = {&img_args};
    cudaKernelNodeParams ip{};
    ip.func = const_cast<void*>(setk::img_lane_func());
    ip.gridDim = dim3(setk::img_lane_grid());
    ip.blockDim = dim3(256);
    ip.kernelParams = iargs;
    cudaGraphNode_t in_ = nullptr;
    DD_CK(cudaGraphAddKernelNode(&in_, sp.conditional.phGraph_out[setk::kDdKindImg], nullptr, 0, &ip));

    DD_CK(cudaGraphInstantiate(&l.exec, l.graph, 0));
    DD_CK(cudaGraphUpload(l.exec, l.stream));
    return SET_OK;
  }

  set_dd_config cfg_{};
  uint32_t depth_ = 0;
  std::vector<CudaLane> lanes_;
  std::vector<DdLaneMem> lane_mem_;
  void* host_block_ = nullptr;
  void* dev_block_ = nullptr;
  size_t scan_stride_ = 0;  // bytes between the scan look-back areas of one lane
  // the driver's cuMemGetAddressRange (base, size of the allocation holding an address; 0 = found)
  int (*range_fn_)(unsigned long long*, size_t*, unsigned long long) = nullptr;
  bool leaked_ = false;
};

}  // namespace

std::unique_ptr<DdBackend> make_dd_backend() { return std::make_unique<CudaDdBackend>(); }

}  // namespace setrt
