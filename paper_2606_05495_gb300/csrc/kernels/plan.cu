// plan.cu -- maps a job to its stage-kernel launches (the kernel nodes of its graph).
#include "stages.h"

namespace setk {

bool plan_job(const JobPlanIn& in, KernelLaunch* kl, int* nk) {
  JobLayout L;
  if (!job_sizes(in.type, in.dims, &L)) return false;
  bool ok = false;
  switch (in.type) {
    case SET_JOB_BLUR_HIST:
      ok = plan_blur_hist(in, L, kl, nk);
      break;
    case SET_JOB_SAXPY_SCAN_MAX:
      ok = plan_saxpy_scan_max(in, L, kl, nk);
      break;
    case SET_JOB_IMG_SOBEL_HIST:
      ok = plan_img_sobel_hist(in, L, kl, nk);
      break;
    case SET_JOB_MLP_LN:
      ok = plan_mlp_ln(in, L, kl, nk);
      break;
    case SET_JOB_HOTSPOT:
      ok = plan_hotspot(in, L, kl, nk);
      break;
    default:
      return false;
  }
  if (ok)
    for (int k = 0; k < *nk; ++k) attach_stamp(kl[k], in.stamps, k);
  return ok;
}

cudaError_t kernels_init() {
  cudaError_t e = blur_hist_init();
  if (e == cudaSuccess) e = mlp_init();
  if (e == cudaSuccess) e = hotspot_init();
  return e;
}

}  // namespace setk
