// once.cu -- instantiations of the one-exponential GSW step kernels (their own translation
// unit, compiled in parallel with hot.cu); see gsw_kernels.cuh.
#include "once.h"

namespace hot_once {

namespace {

// Raises the dynamic shared-memory limit of a shape's kernels to what they use.
// The forward field of given phases runs on sub-tiles of hot::kOnceFwdRows rows (its own schedule).
constexpr int kFwdRows = hot::kOnceFwdRows;

template <int TMAX, int R>
cudaError_t set_smem() {
  const int smem = hot::once_smem_bytes(R), fsmem = hot::once_smem_bytes(kFwdRows);
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(hot::gsw_once_kernel<true, true, TMAX, R>, at, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hot::gsw_once_kernel<true, false, TMAX, kFwdRows>, at, fsmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hot::gsw_once_kernel<false, true, TMAX, R>, at, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hot::gsw_once_kernel<false, false, TMAX, kFwdRows>, at, fsmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hot::gsw_once_persistent_kernel<true, TMAX, R>, at, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(hot::gsw_once_persistent_kernel<false, TMAX, R>, at, smem);
  return e;
}

template <int TMAX, int R>
cudaError_t occupancy_shape(int *per_sm) {
  int a = 0, b = 0, p = 0, q = 0, f = 0, g = 0;
  const int smem = hot::once_smem_bytes(R), fsmem = hot::once_smem_bytes(kFwdRows);
  *per_sm = 0;
  cudaError_t e = set_smem<TMAX, R>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, hot::gsw_once_kernel<true, true, TMAX, R>, hot::kThreads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hot::gsw_once_kernel<false, true, TMAX, R>, hot::kThreads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, hot::gsw_once_persistent_kernel<true, TMAX, R>, hot::kThreads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, hot::gsw_once_persistent_kernel<false, TMAX, R>, hot::kThreads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, hot::gsw_once_kernel<true, false, TMAX, kFwdRows>, hot::kThreads, fsmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, hot::gsw_once_kernel<false, false, TMAX, kFwdRows>, hot::kThreads, fsmem);
  *per_sm = std::min(std::min(std::min(a, b), std::min(p, q)), std::min(f, g));
  return e;
}

template <int TMAX, int R>
cudaError_t step_shape(bool fast, bool back, cudaLaunchConfig_t cfg, const hot::StepArgs &a) {
  cfg.dynamicSmemBytes = hot::once_smem_bytes(back ? R : kFwdRows);
  if (fast)
    return back ? cudaLaunchKernelEx(&cfg, hot::gsw_once_kernel<true, true, TMAX, R>, a)
                : cudaLaunchKernelEx(&cfg, hot::gsw_once_kernel<true, false, TMAX, kFwdRows>, a);
  return back ? cudaLaunchKernelEx(&cfg, hot::gsw_once_kernel<false, true, TMAX, R>, a)
              : cudaLaunchKernelEx(&cfg, hot::gsw_once_kernel<false, false, TMAX, kFwdRows>, a);
}

template <int TMAX, int R>
cudaError_t persistent_shape(bool fast, cudaLaunchConfig_t cfg, const hot::PersistArgs &p) {
  cfg.dynamicSmemBytes = hot::once_smem_bytes(R);
  return fast ? cudaLaunchKernelEx(&cfg, hot::gsw_once_persistent_kernel<true, TMAX, R>, p)
              : cudaLaunchKernelEx(&cfg, hot::gsw_once_persistent_kernel<false, TMAX, R>, p);
}

}  // namespace

cudaError_t occupancy(int shape, int *per_sm) {
  cudaError_t e = cudaSuccess;
  HOT_WITH_ONCE_SHAPE(shape, (e = occupancy_shape<TMAX, R>(per_sm)));
  return e;
}

cudaError_t launch_step(int shape, bool fast, bool back, cudaLaunchConfig_t cfg, const hot::StepArgs &a) {
  cudaError_t e = cudaSuccess;
  HOT_WITH_ONCE_SHAPE(shape, (e = step_shape<TMAX, R>(fast, back, cfg, a)));
  return e;
}

cudaError_t launch_persistent(int shape, bool fast, cudaLaunchConfig_t cfg, const hot::PersistArgs &p) {
  cudaError_t e = cudaSuccess;
  HOT_WITH_ONCE_SHAPE(shape, (e = persistent_shape<TMAX, R>(fast, cfg, p)));
  return e;
}

}  // namespace hot_once
