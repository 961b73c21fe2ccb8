// rsv_mlp.cuh -- launchers of the learned-mass kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {

int mlp_nparam();
int mlp_sites_per_block();
int feat_grid(int64_t T);
cudaError_t launch_mlp_step(const float* feat, const float* target, int64_t T, float* params,
                            float* adam_m, float* adam_v, float* grad_out, float* partials,
                            unsigned* counter, uint64_t seed, uint64_t step, int64_t adam_t,
                            float lr, float b1, float b2, float eps, int batch, int update,
                            float* loss_out, const float* log_scale, cudaStream_t st);
cudaError_t launch_mlp_mass(const float* feat, int64_t T, const float* params, const double* y,
                            const double* hbar, ThetaD th, const float* log_scale, float* minv,
                            float* m_out, cudaStream_t st);
cudaError_t launch_welford(const float* x, int64_t n, int64_t T, int64_t count, double* mean,
                           double* m2, cudaStream_t st);
cudaError_t launch_welford_target(const double* mean, const double* m2, int64_t T, int64_t count,
                                  double* hbar, float* target, float* log_scale, cudaStream_t st);
cudaError_t launch_features(const double* y, const double* lnrv, const double* hbar, int64_t T,
                            ThetaD th, float* F, float* stats, double* partials, unsigned* counter,
                            double* acc, cudaStream_t st);

}  // namespace rsv
