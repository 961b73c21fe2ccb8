// rsv_ess.cuh -- launcher of the per-site effective-sample-size kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsv {
cudaError_t launch_ess(const float* x, int64_t n, int64_t T, float* ess, cudaStream_t st);
}  // namespace rsv
