// rsv_simple.cu -- stand-alone S(h), dS/dh and momentum draws (FP64).
//
// S(h) and dS/dh of the RSV model (arXiv:1603.08114, Sec. 3 with eqs. (1)-(3));
// both are streaming kernels bound by HBM bandwidth: dS/dh reads h (and its
// two neighbours, served from L1/L2), y and lnRV and writes F, 32 B per site.
// With leverage (th.rho != 0, the RSV model with corr(eps_t, eta_t) = rho of
// the RSV reference cited in Sec. 2) the AR term of site t is
// d_t^2 / (2 s_eta^2 (1 - rho^2)), d_t = x_{t+1} - phi x_t - rho s_eta y_t e^{-h_t/2}.
#include <cmath>

#include "rsv_device.cuh"
#include "rsv_simple.cuh"

namespace rsv {

namespace {

// d_t of the leverage model (t < T-1)
__device__ __forceinline__ double lev_innovation(const double* h, const double* y, int64_t t,
                                                 const ThetaD& th, double rs)
{
    return (h[t + 1] - th.mu) - th.phi * (h[t] - th.mu) - rs * (y[t] * exp(-0.5 * h[t]));
}

__global__ void __launch_bounds__(256) k_force(const double* __restrict__ h,
                                               const double* __restrict__ y,
                                               const double* __restrict__ lnrv, int64_t T,
                                               ThetaD th, double* __restrict__ F)
{
    const double phi = th.phi, mu = th.mu, ie = 1.0 / th.se2, iu = 1.0 / th.su2;
    const double rs = th.rho * sqrt(th.se2), B = 1.0 / (th.se2 * (1.0 - th.rho * th.rho));
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double ht = h[t], x = ht - mu;
        double ar;
        if (th.rho != 0.0) {
            // derivative of the terms of s_t and s_{t-1} that hold h_t
            double g = t == 0 ? (1.0 - phi * phi) * x * ie : 0.0;
            if (t + 1 < T)
                g += B * lev_innovation(h, y, t, th, rs) * (0.5 * rs * y[t] * exp(-0.5 * ht) - phi);
            if (t > 0) g += B * lev_innovation(h, y, t - 1, th, rs);
            const double yt = y[t];
            F[t] = 0.5 - 0.5 * yt * yt * exp(-ht) - (lnrv[t] - th.xi - ht) * iu + g;
            continue;
        }
        if (T == 1) {
            ar = (1.0 - phi * phi) * x;
        } else if (t == 0) {
            ar = x - phi * (h[1] - mu);
        } else if (t == T - 1) {
            ar = x - phi * (h[T - 2] - mu);
        } else {
            ar = (1.0 + phi * phi) * x - phi * ((h[t - 1] - mu) + (h[t + 1] - mu));
        }
        const double yt = y[t];
        F[t] = 0.5 - 0.5 * yt * yt * exp(-ht) - (lnrv[t] - th.xi - ht) * iu + ar * ie;
    }
}

// Per-site action s_t summed per block; the last block adds the block sums in
// block order.
__global__ void __launch_bounds__(256) k_action(const double* __restrict__ h,
                                                const double* __restrict__ y,
                                                const double* __restrict__ lnrv, int64_t T,
                                                ThetaD th, double* __restrict__ partials,
                                                unsigned* __restrict__ counter,
                                                double* __restrict__ S_out)
{
    __shared__ double red[32];
    __shared__ int s_last;
    const double phi = th.phi, mu = th.mu, ie = 1.0 / th.se2, iu = 1.0 / th.su2;
    const double rs = th.rho * sqrt(th.se2), B = 1.0 / (th.se2 * (1.0 - th.rho * th.rho));
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double ht = h[t], yt = y[t];
        const double r = lnrv[t] - th.xi - ht;
        double s = 0.5 * ht + 0.5 * yt * yt * exp(-ht) + 0.5 * iu * r * r;
        const double x = ht - mu;
        if (t + 1 < T) {
            if (th.rho != 0.0) {
                const double d = lev_innovation(h, y, t, th, rs);
                s += 0.5 * B * d * d;
            } else {
                const double e = (h[t + 1] - mu) - phi * x;
                s += 0.5 * ie * e * e;
            }
        }
        if (t == 0) s += 0.5 * ie * (1.0 - phi * phi) * x * x;
        acc += s;
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
    const double S = block_sum(v, red);
    if (threadIdx.x == 0) {
        *S_out = S;
        *counter = 0u;
    }
}

// Momenta exactly as the trajectory kernels draw them: one Philox block per
// group of four sites, Box-Muller on 53-bit (FP64) or 23-bit (FP32) uniforms.
__global__ void k_draw_momenta(uint64_t seed, uint64_t series, uint64_t traj, int64_t T,
                               const float* __restrict__ minv, int bits, double* __restrict__ p)
{
    const int64_t nq = (T + 3) / 4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const u64x4 r = philox_block(seed, series, traj, STREAM_MOM, (uint64_t)q);
        double z[4];
        if (bits == 53) {
            box_muller(u01_53(r.w[0]), u01_53(r.w[1]), z[0], z[1]);
            box_muller(u01_53(r.w[2]), u01_53(r.w[3]), z[2], z[3]);
        } else {
            float f[4];
            box_muller_f(u01_23(r.w[0]), u01_23(r.w[1]), f[0], f[1]);
            box_muller_f(u01_23(r.w[2]), u01_23(r.w[3]), f[2], f[3]);
            for (int i = 0; i < 4; ++i) z[i] = f[i];
        }
        for (int i = 0; i < 4; ++i) {
            const int64_t t = 4 * q + i;
            if (t >= T) break;
            if (minv) {
                if (bits == 53) z[i] = z[i] / sqrt((double)minv[t]);
                else z[i] = (double)((float)z[i] / sqrtf(minv[t]));
            }
            p[t] = z[i];
        }
    }
}

int grid_stream(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int action_grid(int64_t T) { return grid_stream(T); }

cudaError_t launch_force(const double* h, const double* y, const double* lnrv, int64_t T,
                         ThetaD th, double* F, cudaStream_t st)
{
    k_force<<<grid_stream(T), 256, 0, st>>>(h, y, lnrv, T, th, F);
    return cudaGetLastError();
}

cudaError_t launch_action(const double* h, const double* y, const double* lnrv, int64_t T,
                          ThetaD th, double* partials, unsigned* counter, double* S_out,
                          cudaStream_t st)
{
    k_action<<<grid_stream(T), 256, 0, st>>>(h, y, lnrv, T, th, partials, counter, S_out);
    return cudaGetLastError();
}

cudaError_t launch_draw_momenta(uint64_t seed, uint64_t series, uint64_t traj, int64_t T,
                                const float* minv, int bits, double* p, cudaStream_t st)
{
    k_draw_momenta<<<grid_stream((T + 3) / 4), 256, 0, st>>>(seed, series, traj, T, minv, bits, p);
    return cudaGetLastError();
}

}  // namespace rsv
