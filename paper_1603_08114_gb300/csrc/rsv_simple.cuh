// rsv_simple.cuh -- launchers of the stand-alone S(h), dS/dh and draw kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {

int action_grid(int64_t T);
cudaError_t launch_force(const double* h, const double* y, const double* lnrv, int64_t T,
                         ThetaD th, double* F, cudaStream_t st);
cudaError_t launch_action(const double* h, const double* y, const double* lnrv, int64_t T,
                          ThetaD th, double* partials, unsigned* counter, double* S_out,
                          cudaStream_t st);
cudaError_t launch_draw_momenta(uint64_t seed, uint64_t series, uint64_t traj, int64_t T,
                                const float* minv, int bits, double* p, cudaStream_t st);

}  // namespace rsv
