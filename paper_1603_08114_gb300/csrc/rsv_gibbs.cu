// rsv_gibbs.cu -- the theta update between HMC trajectories, on the device.
//
// The paper updates theta with the code of its ref. [Takaishi4] and does not
// describe it (Sec. 2).  This is an exact Gibbs sweep under flat priors on
// phi in (-1,1), mu, xi and 1/sigma^2 priors on both variances, in the order
//   xi      ~ N(mean(lnRV - h), s_u^2 / T)
//   s_u^2   ~ IG(T/2, sum (lnRV - xi - h)^2 / 2)
//   mu      ~ N(m_mu, s_eta^2 / P),  from the quadratic form of eq. (3) and the
//             stationary law of h_1: P = (1-phi^2) + (T-1)(1-phi)^2
//   s_eta^2 ~ IG(T/2, Q/2),  Q = (1-phi^2) x_1^2 + sum (x_{t+1} - phi x_t)^2
//   phi     : independence Metropolis from N(sum x_t x_{t+1} / D, s_eta^2 / D)
//             truncated to (-1,1), D = sum_{t=2}^{T-1} x_t^2, accepted with
//             ratio sqrt(1-phi'^2) / sqrt(1-phi^2).
// One pass over the accepted state gathers sufficient statistics centred on the
// current theta (q = lnRV - xi - h, x = h - mu, e = x_{t+1} - phi x_t), so the
// sums carry no cancellation; the last block to finish combines them in block
// order and one thread takes the scalar draws from Philox stream 2.
#include <cmath>

#include "rsv_device.cuh"
#include "rsv_gibbs.cuh"

namespace rsv {

namespace {

constexpr int NSTAT = 8;  // sum q, sum q^2, X_a, X_b, XX_m, XY, sum e, sum e^2

// Sequential uniforms of Philox stream 2 for one trajectory (block 0, 1, ...).
struct Stream {
    uint64_t seed, series, traj, blk;
    u64x4 w;
    int pos;
    __device__ double u01()
    {
        if (pos == 4) {
            w = philox_block(seed, series, traj, STREAM_THETA, blk++);
            pos = 0;
        }
        return u01_53(w.w[pos++]);
    }
    // cosine branch of Box-Muller: one normal per two uniforms
    __device__ double normal()
    {
        const double u1 = u01(), u2 = u01();
        return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
    // Gamma(alpha, 1): Marsaglia & Tsang (ACM TOMS 26, 2000) for alpha >= 1;
    // alpha < 1 as Gamma(alpha + 1) u^(1/alpha).  NaN after 1000 rejections.
    __device__ double gamma(double alpha)
    {
        double scale = 1.0;
        if (alpha < 1.0) {
            const double g = gamma1(alpha + 1.0);
            const double u = u01();
            return g * pow(u, 1.0 / alpha);
        }
        return scale * gamma1(alpha);
    }
    __device__ double gamma1(double alpha)
    {
        const double d = alpha - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
        for (int it = 0; it < 1000; ++it) {
            const double z = normal();
            double v = 1.0 + c * z;
            if (v <= 0.0) continue;
            v = v * v * v;
            const double u = u01();
            if (log(u) < 0.5 * z * z + d - d * v + d * log(v)) return d * v;
        }
        return NAN;
    }
};

// Per-site contributions, FP64 state.
__device__ __forceinline__ void site_stats_d(const double* h, const double* lnrv, int64_t t,
                                            int64_t T, const ThetaD& th, double (&s)[NSTAT])
{
    const double ht = h[t];
    const double q = (lnrv[t] - th.xi) - ht;
    const double x = ht - th.mu;
    s[0] += q;
    s[1] += q * q;
    if (t + 1 < T) {
        const double xn = h[t + 1] - th.mu;
        const double e = xn - th.phi * x;
        s[2] += x;
        s[5] += x * xn;
        s[6] += e;
        s[7] += e * e;
    }
    if (t >= 1) s[3] += x;
    if (t >= 1 && t + 1 < T) s[4] += x * x;
}

// Per-site contributions, (hi, lo) FP32 state: double-float arithmetic.
__device__ __forceinline__ void site_stats_f(const float2* h, const float2* lr, int64_t t,
                                            int64_t T, ff xi, ff mu, ff phi, ff (&s)[NSTAT])
{
    const float2 hv = h[t];
    const ff ht = {hv.x, hv.y};
    const float2 lv = lr[t];
    const ff q = ff_sub(ff_sub(ff{lv.x, lv.y}, xi), ht);
    const ff x = ff_sub(ht, mu);
    ff_acc(s[0], q);
    ff_acc(s[1], ff_mul(q, q));
    if (t + 1 < T) {
        const float2 hn = h[t + 1];
        const ff xn = ff_sub(ff{hn.x, hn.y}, mu);
        const ff e = ff_sub(xn, ff_mul(phi, x));
        ff_acc(s[2], x);
        ff_acc(s[5], ff_mul(x, xn));
        ff_acc(s[6], e);
        ff_acc(s[7], ff_mul(e, e));
    }
    if (t >= 1) ff_acc(s[3], x);
    if (t >= 1 && t + 1 < T) ff_acc(s[4], ff_mul(x, x));
}

__device__ void gibbs_draws(const double (&S)[NSTAT], double x0, int64_t T, double* theta,
                            double* theta_out, uint64_t seed, uint64_t series, uint64_t traj,
                            int mask, int* phi_acc)
{
    ThetaD th = load_theta(theta);
    Stream st{seed, series, traj, 0, {}, 4};
    const double Td = (double)T;
    const double xi0 = th.xi, mu0 = th.mu, phi = th.phi;
    double xi = xi0, su2 = th.su2, mu = mu0, se2 = th.se2, ph = phi;
    // xi
    if (mask & 1) xi = xi0 + S[0] / Td + sqrt(su2 / Td) * st.normal();
    // s_u^2: sum (q - dxi)^2
    if (mask & 2) {
        const double dxi = xi - xi0;
        const double ss = S[1] - 2.0 * dxi * S[0] + Td * dxi * dxi;
        const double g = st.gamma(0.5 * Td);
        if (g > 0.0 && ss > 0.0) su2 = 0.5 * ss / g;  // degenerate state: keep
    }
    // mu
    if (mask & 4) {
        const double w0 = 1.0 - phi * phi, w1 = (1.0 - phi) * (1.0 - phi);
        const double den = w0 + (Td - 1.0) * w1;
        const double m = mu0 + (w0 * x0 + (1.0 - phi) * S[6]) / den;
        mu = m + st.normal() / sqrt(den / se2);
    }
    const double dmu = mu - mu0;
    // s_eta^2
    if (mask & 8) {
        const double a = x0 - dmu, om = 1.0 - phi;
        const double Q = (1.0 - phi * phi) * a * a + S[7] - 2.0 * om * dmu * S[6] +
                         (Td - 1.0) * om * om * dmu * dmu;
        const double g = st.gamma(0.5 * Td);
        if (g > 0.0 && Q > 0.0) se2 = 0.5 * Q / g;
    }
    // phi
    int acc = 0;
    if (mask & 16) {
        const double num = S[5] - dmu * (S[2] + S[3]) + (Td - 1.0) * dmu * dmu;
        const double Xm = S[2] - x0;  // sum_{t=1}^{T-2} x_t
        const double D = S[4] - 2.0 * dmu * Xm + (Td - 2.0) * dmu * dmu;
        if (T >= 3 && D > 0.0) {
            const double m = num / D, sd = sqrt(se2 / D);
            double prop = NAN;
            for (int it = 0; it < 1000; ++it) {
                const double c = m + sd * st.normal();
                if (c > -1.0 && c < 1.0) {
                    prop = c;
                    break;
                }
            }
            const double u = st.u01();
            if (prop == prop) {
                const double lr = 0.5 * log(1.0 - prop * prop) - 0.5 * log(1.0 - phi * phi);
                if (log(u) < lr) {
                    ph = prop;
                    acc = 1;
                }
            }
        }
    }
    theta[0] = ph;
    theta[1] = mu;
    theta[2] = xi;
    theta[3] = se2;
    theta[4] = su2;
    if (theta_out)
        for (int i = 0; i < 5; ++i) theta_out[i] = theta[i];
    if (phi_acc) *phi_acc = acc;
}

// Block sum of NSTAT double-float values in a fixed order (butterfly in each
// warp, then warp 0 over the warps in order); the result is valid in thread 0.
__device__ __forceinline__ void block_sum_ff(ff (&s)[NSTAT], float2 (*red)[NSTAT])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) {
        const ff w = warp_sum_ff(s[i]);
        if (lane == 0) red[warp][i] = make_float2(w.hi, w.lo);
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NSTAT; ++i) {
            const float2 v = lane < nw ? red[lane][i] : make_float2(0.f, 0.f);
            s[i] = warp_sum_ff(ff{v.x, v.y});
        }
    }
    __syncthreads();
}

// Statistics pass + last-block draws.  `cur` selects the state buffer.  The
// mixed path keeps every per-site and cross-block sum in double-float (FP32
// arithmetic; the FP64 pipe of this GPU is slow) and converts the totals to
// FP64 once for the scalar draws.
template <bool MIXED>
__global__ void __launch_bounds__(256) k_gibbs(GibbsArgs A)
{
    __shared__ double red[32];
    __shared__ float2 redf[32][NSTAT];
    __shared__ ff s_c[3];
    __shared__ int s_last;
    const int* curp = A.cur;
    const int cur = curp ? *(volatile int*)curp : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (MIXED) {
        if (threadIdx.x == 0) {
            const ThetaD th = load_theta(A.theta);
            s_c[0] = ff_from_double(th.xi);
            s_c[1] = ff_from_double(th.mu);
            s_c[2] = ff_from_double(th.phi);
        }
        __syncthreads();
        const ff xi = s_c[0], mu = s_c[1], phi = s_c[2];
        const float2* h = cur ? A.h1f : A.h0f;
        ff s[NSTAT];
        for (int i = 0; i < NSTAT; ++i) s[i] = ff{0.f, 0.f};
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A.T; t += stride)
            site_stats_f(h, A.lr_f, t, A.T, xi, mu, phi, s);
        block_sum_ff(s, redf);
        float2* pf = reinterpret_cast<float2*>(A.partials);
        if (threadIdx.x == 0)
            for (int i = 0; i < NSTAT; ++i)
                pf[(int64_t)blockIdx.x * NSTAT + i] = make_float2(s[i].hi, s[i].lo);
    } else {
        const ThetaD th = load_theta(A.theta);
        double S[NSTAT];
        for (int i = 0; i < NSTAT; ++i) S[i] = 0.0;
        const double* h = cur ? A.h1d : A.h0d;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A.T; t += stride)
            site_stats_d(h, A.lnrv, t, A.T, th, S);
        for (int i = 0; i < NSTAT; ++i) {
            const double b = block_sum(S[i], red);
            if (threadIdx.x == 0) A.partials[(int64_t)blockIdx.x * NSTAT + i] = b;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[NSTAT];
    if (MIXED) {
        const float2* pf = reinterpret_cast<const float2*>(A.partials);
        ff s[NSTAT];
        for (int i = 0; i < NSTAT; ++i) {
            s[i] = ff{0.f, 0.f};
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
                const float2 v = __ldcg(pf + (int64_t)b * NSTAT + i);
                s[i] = ff_add(s[i], ff{v.x, v.y});
            }
        }
        block_sum_ff(s, redf);
        for (int i = 0; i < NSTAT; ++i) tot[i] = ff_to_double(s[i]);
    } else {
        for (int i = 0; i < NSTAT; ++i) {
            double v = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
                v += __ldcg(A.partials + (int64_t)b * NSTAT + i);
            tot[i] = block_sum(v, red);
        }
    }
    if (threadIdx.x == 0) {
        *A.counter = 0u;
        const ThetaD th = load_theta(A.theta);
        double x0;
        if (MIXED) {
            const float2 v = (cur ? A.h1f : A.h0f)[0];
            x0 = ((double)v.x + (double)v.y) - th.mu;
        } else {
            x0 = (cur ? A.h1d : A.h0d)[0] - th.mu;
        }
        gibbs_draws(tot, x0, A.T, A.theta, A.theta_out, A.seed, A.series, A.traj, A.mask,
                    A.phi_acc);
        if (A.theta_f) *A.theta_f = mixed_theta(load_theta(A.theta));
        __threadfence();
    }
}

}  // namespace

// About 4 sites per thread, up to 8 blocks of 256 per SM: the statistics pass
// is bound by load latency, so it wants many threads in flight.
int gibbs_grid(int64_t T)
{
    int64_t g = (T + 1023) / 1024;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_gibbs(const GibbsArgs& a, bool mixed, cudaStream_t st)
{
    const int g = gibbs_grid(a.T);
    if (mixed) k_gibbs<true><<<g, 256, 0, st>>>(a);
    else k_gibbs<false><<<g, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rsv
