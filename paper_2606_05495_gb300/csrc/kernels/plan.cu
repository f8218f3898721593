// plan.cu -- maps a job to its stage-kernel launches (the kernel nodes of its graph).
#include "stages.h"

namespace setk {

bool plan_job(const JobPlanIn& in, KernelLaunch* kl, int* nk) {
  JobLayout L;
  if (!job_sizes(in.type, in.dims, &L)) return false;
  switch (in.type) {
    case SET_JOB_BLUR_HIST:
      return plan_blur_hist(in, L, kl, nk);
    case SET_JOB_SAXPY_SCAN_MAX:
      return plan_saxpy_scan_max(in, L, kl, nk);
    case SET_JOB_IMG_SOBEL_HIST:
      return plan_img_sobel_hist(in, L, kl, nk);
    case SET_JOB_MLP_LN:
      return plan_mlp_ln(in, L, kl, nk);
    default:
      return false;
  }
}

cudaError_t kernels_init() {
  cudaError_t e = blur_hist_init();
  if (e == cudaSuccess) e = mlp_init();
  return e;
}

}  // namespace setk
