// rsv_gibbs.cuh -- launcher of the theta Gibbs sweep.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rsv_traj.cuh"

namespace rsv {

struct GibbsArgs {
    const double* h0d;   // FP64 state double buffer (FP64 path)
    const double* h1d;
    const float2* h0f;   // (hi, lo) state double buffer (mixed path)
    const float2* h1f;
    const int* cur;      // buffer selector, NULL = buffer 0
    const double* lnrv;  // FP64 path
    const float2* lr_f;  // mixed path: lnRV as (hi, lo)
    int64_t T;
    double* theta;       // device [5], in/out
    double* theta_out;   // optional record [5]
    uint64_t seed, series, traj;
    int mask;            // components updated: bit 0 xi .. bit 4 phi
    double* partials;    // [grid * 8]
    unsigned* counter;
    int* phi_acc;        // optional
    MixedTheta* theta_f; // mixed path: the current theta's constants, read and refreshed
    float* snap_out;     // mixed path, optional: h (FP32) of the state the sweep reads
    // mixed path, optional: [2] statistics of the state in each buffer (see
    // StateStats); when set the sweep takes its sums from the current
    // buffer's record and reads no site (snap_out is then not written)
    const StatsRec* rstats;
};

int gibbs_grid(int64_t T);
cudaError_t launch_gibbs(const GibbsArgs& a, bool mixed, cudaStream_t st);

}  // namespace rsv
