// rsv_chain.cuh -- the persistent chain kernel (rsv_chain.cu), host side.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "rsv_traj.cuh"

namespace rsv {

// A chain of n_traj mixed-precision trajectories of one series (model without
// leverage) with the theta sweep after each, in one cooperative launch.
struct ChainArgs {
    TrajArgs A;           // trajectory arguments (state buffers, per-site constants,
                          // plan, scheme; A.theta_f: constants of the starting theta;
                          // A.rstats[0]: statistics of buffer 0, the starting state)
    int64_t n_traj;
    uint64_t traj0;
    int update_theta;
    double* theta;        // device [5] in/out
    double* theta_out;    // [n_traj][5] or NULL
    float* snaps;         // [n_traj / thin][T] or NULL
    int64_t thin;
    double* dH_out;       // [n_traj] or NULL
    int* acc_out;         // [n_traj] or NULL
    double* partials;     // 2 x nsegs x kPartialWords doubles (parity double buffer)
    int64_t nsegs;
    unsigned* bar;        // grid barrier counter, zero at launch
    long long wait_limit; // clock cycles a barrier wait may take before ST_TIMEOUT
    int fallback_window;  // mass fallback window (0: none)
    int* mass_on_out;     // final mass flag, or NULL
    int* ser_cur_out;     // [1] final state buffer
};

// True if the plan can run as one persistent chain (mixed, no leverage, one
// series, every bin on its own block, an instantiated block shape).
bool chain_supported(const Plan& p);
// *fits: the plan is supported and all its blocks can be resident at once.
cudaError_t chain_fits(const Plan& p, int num_sms, bool* fits);
// Launch the chain cooperatively; *launched is false (and nothing is
// launched) if the plan's blocks cannot all be resident at once.
cudaError_t launch_chain(const ChainArgs& c, const Plan& p, int num_sms, cudaStream_t st,
                         bool* launched);

}  // namespace rsv
