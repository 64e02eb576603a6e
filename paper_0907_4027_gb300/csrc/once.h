// once.h -- host interface (internal to the library) of the one-exponential GSW step kernels
// (hot::gsw_once_kernel, hot::gsw_once_persistent_kernel): once.cu instantiates them for every
// shape, hot.cu drives them.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "gsw_kernels.cuh"

namespace hot_once {

// Blocks per SM that every kernel of a shape (hot::once_shape) keeps resident.
cudaError_t occupancy(int shape, int *per_sm);

// One launch of the per-iteration kernel (BACK: the GSW step; otherwise the forward field of
// given phases) or of the persistent form, with the grid, block, stream and attributes of cfg
// (its dynamic shared memory is set here).
cudaError_t launch_step(int shape, bool fast, bool back, cudaLaunchConfig_t cfg, const hot::StepArgs &a);
cudaError_t launch_persistent(int shape, bool fast, cudaLaunchConfig_t cfg, const hot::PersistArgs &p);

}  // namespace hot_once
