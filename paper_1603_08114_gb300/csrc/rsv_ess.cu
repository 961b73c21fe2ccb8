// rsv_ess.cu -- effective sample size per site of a chain of snapshots.
//
// Geyer's initial monotone sequence estimator (C. J. Geyer, Statistical
// Science 7, 1992): normalised autocorrelations rho_k from the plain sums
// gamma_k = (1/n) sum_t (x_t - m)(x_{t+k} - m); pair sums
// Gamma_m = rho_{2m} + rho_{2m+1} taken while positive and made
// non-increasing; tau = -1 + 2 sum Gamma_m, floored at 1/log10(n) (so ESS
// <= n log10 n); ESS = n / tau; a constant column (zero variance) gets 0.
// One thread per site; the snapshot matrix is [n][T] FP32 (sample-major), so a
// warp reads 128 contiguous bytes per sample.
#include <cmath>

#include "rsv_ess.cuh"

namespace rsv {

namespace {

__global__ void __launch_bounds__(256) k_ess(const float* __restrict__ x, int64_t n, int64_t T,
                                             float* __restrict__ ess)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    // mean with compensation
    float s = 0.f, c = 0.f;
    for (int64_t k = 0; k < n; ++k) {
        const float v = x[k * T + t] - c;
        const float u = s + v;
        c = (u - s) - v;
        s = u;
    }
    const float m = s / (float)n;
    auto gamma = [&](int64_t lag) {
        float a = 0.f, ca = 0.f;
        for (int64_t k = 0; k + lag < n; ++k) {
            const float v = (x[k * T + t] - m) * (x[(k + lag) * T + t] - m) - ca;
            const float u = a + v;
            ca = (u - a) - v;
            a = u;
        }
        return a / (float)n;
    };
    const float g0 = gamma(0);
    if (!(g0 > 0.f)) {  // the chain never moved at this site
        ess[t] = 0.f;
        return;
    }
    float tau_sum = 0.f, prev = INFINITY;
    for (int64_t mm = 0; 2 * mm + 1 < n; ++mm) {
        const float G = (mm == 0 ? 1.0f : gamma(2 * mm) / g0) + gamma(2 * mm + 1) / g0;
        if (!(G > 0.f)) break;
        const float Gm = fminf(G, prev);
        tau_sum += Gm;
        prev = Gm;
    }
    float tau = -1.f + 2.f * tau_sum;
    const float nn = (float)(n > 10 ? n : 10);
    tau = fmaxf(tau, 1.f / log10f(nn));
    ess[t] = (float)n / tau;
}

}  // namespace

cudaError_t launch_ess(const float* x, int64_t n, int64_t T, float* ess, cudaStream_t st)
{
    const int64_t g = (T + 255) / 256;
    k_ess<<<(unsigned)g, 256, 0, st>>>(x, n, T, ess);
    return cudaGetLastError();
}

}  // namespace rsv
