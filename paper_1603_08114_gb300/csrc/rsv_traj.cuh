// rsv_traj.cuh -- launch interface of the trajectory kernels (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {

// Arguments of one HMC trajectory over one series, split into tiles.  Tile b
// owns sites [b*tile, min(T,(b+1)*tile)) and integrates the window extended by
// K = n_md + 1 sites on each side (left edge rounded down to a multiple of 4),
// so that its owned sites (and the right neighbour needed by dH) are exact
// after n_md steps without any exchange between tiles.
struct TrajArgs {
    // FP64 state (FP64 path): h0/h1 double buffer; cur selects the input.
    const double* h0d;
    double* h1d;
    // double-float state (mixed path): (hi, lo) of h.
    const float2* h0f;
    float2* h1f;
    int* cur;                 // device: 0 -> read buffer 0, write buffer 1; NULL = 0 always
    const double* p_in;       // optional initial momenta (FP64)
    double* p_out;            // optional p' (FP64), must not alias p_in
    const double* y;          // FP64 path inputs
    const double* lnrv;
    const float* a_f;         // mixed path per-site constants: y^2/2
    const float* b0_f;        //   log2(y^2/2)
    const float2* lr_f;       //   lnRV as (hi, lo)
    const float* minv;        // optional inverse mass (FP32)
    const int* mass_on;       // optional device flag; 0 = use m = 1
    const double* theta;      // device [5], or NULL to use th_inline
    ThetaD th_inline;
    int64_t T;
    int64_t tile;
    int K;
    int n_md;
    double dtau;
    uint64_t seed, series, traj;
    const double* log_u;      // optional device scalar
    double* partials;         // [gridDim.x]
    unsigned* counter;        // zero before launch; last block resets it
    double* dH_out;           // device scalar
    int* acc_out;             // device scalar
    int* status;
    // chain bookkeeping (optional): mass fallback over windows of trajectories
    int* fb_state;            // [2]: accepted count in window, trajectories in window
    int fallback_window;
};

// Kernel configuration: threads per block and sites per thread.
struct TileCfg {
    int nt;
    int j;
    int64_t tile;
    int grid;
    size_t smem;
};

// Choose a tiling for a series of length T (window capacity nt*j per block).
TileCfg plan_tiles(int64_t T, int n_md, bool mixed, bool mass, int num_sms);
// The fixed tiling (nt, j, tile), or nt = 0 if it is not valid for this call.
TileCfg fixed_tiles(int64_t T, int n_md, bool mixed, bool mass, int nt, int j, int64_t tile);

cudaError_t launch_traj(const TrajArgs& a, const TileCfg& c, bool mixed, bool mass,
                        cudaStream_t st);
cudaError_t launch_commit_fp64(double* h, const double* hprop, double* p, const double* pprop,
                               const int* acc, int64_t T, cudaStream_t st);
cudaError_t launch_prep_mixed(const double* y, const double* lnrv, float* a_f, float* b0_f,
                              float2* lr_f, int64_t T, cudaStream_t st);
cudaError_t launch_h_to_ff(const double* h, float2* hf, int64_t T, cudaStream_t st);
cudaError_t launch_ff_to_h(const float2* hf, double* h, const int* acc, int64_t T,
                           cudaStream_t st);
cudaError_t launch_ff_to_h_sel(const float2* b0, const float2* b1, const int* cur, double* h,
                               int64_t T, cudaStream_t st);
cudaError_t launch_d_sel(const double* b0, const double* b1, const int* cur, double* h,
                         int64_t T, cudaStream_t st);
cudaError_t launch_snapshot(const double* b0, const double* b1, const float2* f0,
                            const float2* f1, const int* cur, float* out, int64_t T,
                            cudaStream_t st);

}  // namespace rsv
