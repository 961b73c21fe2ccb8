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
#include "rsv_gibbs_dev.cuh"

namespace rsv {

namespace {

// ---------------------------------------------------------------------------
// The draws with their variates precomputed in parallel.  The FP64 pipe of
// this GPU takes about 64 cycles per warp instruction whether one lane or 32
// are active, so a single thread walking the draws spends most of its time
// there.  Every random variate the sweep uses is a function of stream 2 alone
// (uniforms, their logs, Box-Muller normals, and the Marsaglia-Tsang
// candidates v = (1 + c z)^3 with their logs, c fixed by T), so all of them
// are computed for stream positions 0..NPRE-1 at once, one position per lane,
// with the transcendental steps spread over four warps (four FP64 units);
// so are the few quantities that need only the current theta.  One warp then
// walks the sweep consuming stream 2 in order (block k of Philox stream 2
// gives positions 4k..4k+3), with the same FP64 expressions, and evaluates
// directly past the precomputed positions.
// ---------------------------------------------------------------------------
constexpr int NPRE = 32;

struct PreDraws {
    double u[NPRE + 1], lu[NPRE], sq[NPRE], cs[NPRE], bm[NPRE], v[NPRE], v3[NPRE], lv3[NPRE];
    double gc, gd;                  // Marsaglia-Tsang c, d of the sweep's gamma shape
    double sxi, mmu, smu, lphi;     // sqrt(s_u^2/T); mean and precision root of mu; log(1-phi^2)
};

// Variates in stream order: u01 takes one position; normal() two, the cosine
// branch of Box-Muller sqrt(-2 ln u1) cospi(2 u2); gamma(alpha) by Marsaglia &
// Tsang (ACM TOMS 26, 2000) for alpha >= 1 (NaN after 1000 rejections), and
// as Gamma(alpha + 1) u^(1/alpha) for alpha < 1.
struct WalkStream {
    const PreDraws* P;
    uint64_t seed, series, traj;
    int pos;
    double alpha_pre;
    __device__ double direct_u(int i) const
    {
        const u64x4 w = philox_block(seed, series, traj, STREAM_THETA, (uint64_t)(i >> 2));
        return u01_53(w.w[i & 3]);
    }
    __device__ double uni(int i) const { return i <= NPRE ? P->u[i] : direct_u(i); }
    __device__ double loguni(int i) const { return i < NPRE ? P->lu[i] : log(uni(i)); }
    __device__ double normal_at(int i) const
    {
        return i < NPRE ? P->bm[i] : sqrt(-2.0 * loguni(i)) * cospi(2.0 * uni(i + 1));
    }
    __device__ double u01() { return uni(pos++); }
    __device__ double normal()
    {
        const double z = normal_at(pos);
        pos += 2;
        return z;
    }
    __device__ double gamma(double alpha)
    {
        if (alpha < 1.0) {
            const double g = gamma1(alpha + 1.0);
            const double u = u01();
            return g * pow(u, 1.0 / alpha);
        }
        return gamma1(alpha);
    }
    __device__ double gamma1(double alpha)
    {
        const bool pre = alpha == alpha_pre;
        const double d = pre ? P->gd : alpha - 1.0 / 3.0;
        const double c = pre ? P->gc : 1.0 / sqrt(9.0 * d);
        for (int it = 0; it < 1000; ++it) {
            const int i = pos;
            const bool hit = pre && i < NPRE;
            const double z = normal();
            double v = hit ? P->v[i] : 1.0 + c * z;
            if (v <= 0.0) continue;
            v = hit ? P->v3[i] : v * v * v;
            const double lu = loguni(pos++);
            const double lv = hit ? P->lv3[i] : log(v);
            if (lu < 0.5 * z * z + d - d * v + d * lv) return d * v;
        }
        return NAN;
    }
};

// Fill P (all threads of the block call it; result valid after it returns).
__device__ void predraw(PreDraws* P, const ThetaD& th, int64_t T, uint64_t seed, uint64_t series,
                        uint64_t traj)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double Td = (double)T;
    const double alpha = 0.5 * Td < 1.0 ? 0.5 * Td + 1.0 : 0.5 * Td;
    if (warp == 0) {
        const u64x4 w = philox_block(seed, series, traj, STREAM_THETA, (uint64_t)(lane >> 2));
        P->u[lane] = u01_53(w.w[lane & 3]);
    } else if (warp == 1 && lane == 0) {
        const u64x4 w = philox_block(seed, series, traj, STREAM_THETA, (uint64_t)(NPRE >> 2));
        P->u[NPRE] = u01_53(w.w[0]);
    } else if (warp == 2 && lane == 0) {
        P->gd = alpha - 1.0 / 3.0;
        P->gc = 1.0 / sqrt(9.0 * P->gd);
    } else if (warp == 3 && lane == 0) {
        P->sxi = sqrt(th.su2 / Td);
        P->lphi = log(1.0 - th.phi * th.phi);
    } else if (warp == 4 && lane == 0) {
        const double phi = th.phi;
        const double w0 = 1.0 - phi * phi, w1 = (1.0 - phi) * (1.0 - phi);
        const double den = w0 + (Td - 1.0) * w1;
        P->smu = sqrt(den / th.se2);
    }
    __syncthreads();
    if (warp == 0) {
        const double lu = log(P->u[lane]);
        P->lu[lane] = lu;
        P->sq[lane] = sqrt(-2.0 * lu);
    } else if (warp == 1) {
        P->cs[lane] = cospi(2.0 * P->u[lane + 1]);
    }
    __syncthreads();
    if (warp == 0) {
        const double z = P->sq[lane] * P->cs[lane];
        const double v = 1.0 + P->gc * z;
        P->bm[lane] = z;
        P->v[lane] = v;
        P->v3[lane] = v * v * v;
    }
    __syncthreads();
    if (warp == 0) {
        const double v3 = P->v3[lane];
        P->lv3[lane] = P->v[lane] > 0.0 ? log(v3) : 0.0;
    }
    __syncthreads();
}

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

// Per-site contributions, (hi, lo) FP32 state, in FP32: the sweep reads the
// totals in FP32, so per-site FP32 terms (relative error ~1e-7, unbiased)
// summed per thread in FP32 and across threads in double-float are enough.
// The centring values xi, mu, phi are the FP32 theta the sweep starts from.
// hv = h_t, lv = lnRV_t, hn = h_{t+1} (read only if t + 1 < T), as (hi, lo).
__device__ __forceinline__ void site_stats_f(float2 hv, float2 lv, float2 hn, int64_t t, int64_t T,
                                            float xi, float mu, float phi, float (&s)[NSTAT])
{
    const float q = ((lv.x - hv.x) - xi) + (lv.y - hv.y);
    const float x = (hv.x - mu) + hv.y;
    s[0] += q;
    s[1] = fmaf(q, q, s[1]);
    if (t + 1 < T) {
        const float xn = (hn.x - mu) + hn.y;
        const float e = fmaf(-phi, x, xn);
        s[2] += x;
        s[5] = fmaf(x, xn, s[5]);
        s[6] += e;
        s[7] = fmaf(e, e, s[7]);
    }
    if (t >= 1) s[3] += x;
    if (t >= 1 && t + 1 < T) s[4] = fmaf(x, x, s[4]);
}

// The sweep itself (called by every lane of one warp, uniformly).
__device__ void gibbs_draws(const double (&S)[NSTAT], double x0, int64_t T, const ThetaD& th,
                            double* theta, double* theta_out, const PreDraws* P, uint64_t seed,
                            uint64_t series, uint64_t traj, int mask, int* phi_acc)
{
    const double Td = (double)T;
    WalkStream st{P, seed, series, traj, 0, 0.5 * Td < 1.0 ? 0.5 * Td + 1.0 : 0.5 * Td};
    const double xi0 = th.xi, mu0 = th.mu, phi = th.phi;
    double xi = xi0, su2 = th.su2, mu = mu0, se2 = th.se2, ph = phi;
    // xi
    if (mask & 1) xi = xi0 + S[0] / Td + P->sxi * st.normal();
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
        mu = m + st.normal() / P->smu;
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
                const double lr = 0.5 * log(1.0 - prop * prop) - 0.5 * P->lphi;
                if (log(u) < lr) {
                    ph = prop;
                    acc = 1;
                }
            }
        }
    }
    if ((threadIdx.x & 31) == 0) {
        theta[0] = ph;
        theta[1] = mu;
        theta[2] = xi;
        theta[3] = se2;
        theta[4] = su2;
        if (theta_out)
            for (int i = 0; i < 5; ++i) theta_out[i] = theta[i];
        if (phi_acc) *phi_acc = acc;
    }
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

// FP64 path: statistics pass + last-block draws.  `cur` selects the state
// buffer.
__global__ void __launch_bounds__(256) k_gibbs(GibbsArgs A)
{
    __shared__ double red[32];
    __shared__ int s_last;
    const int* curp = A.cur;
    const int cur = curp ? *(volatile int*)curp : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    {
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
    // FP64 totals, the FP64 sweep with its variates precomputed
    __shared__ PreDraws s_pre;
    __shared__ double s_tot[NSTAT];
    const ThetaD th = load_theta(A.theta);
    for (int i = 0; i < NSTAT; ++i) {
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            v += __ldcg(A.partials + (int64_t)b * NSTAT + i);
        const double t = block_sum(v, red);
        if (threadIdx.x == 0) s_tot[i] = t;
    }
    predraw(&s_pre, th, A.T, A.seed, A.series, A.traj);  // ends with a barrier
    if (threadIdx.x < 32) {
        double tot[NSTAT];
        for (int i = 0; i < NSTAT; ++i) tot[i] = s_tot[i];
        const double x0 = (cur ? A.h1d : A.h0d)[0] - th.mu;
        gibbs_draws(tot, x0, A.T, th, A.theta, A.theta_out, &s_pre, A.seed, A.series, A.traj,
                    A.mask, A.phi_acc);
        if (threadIdx.x == 0) *A.counter = 0u;
    }
    __threadfence();
}

// theta rounded to FP32 (exact after the first mixed sweep): one conversion
// per lane, then shared across the warp.
__device__ __forceinline__ void theta_f32(const GibbsArgs& A, float (&th)[5])
{
    const int lane = threadIdx.x & 31;
    const float mine = lane < 5 ? (float)A.theta[lane] : 0.0f;
#pragma unroll
    for (int k = 0; k < 5; ++k) th[k] = __shfl_sync(0xffffffffu, mine, k);
}

// The FP32 sweep by one warp from the statistics tot (centred at th) and
// x0 = h_1 - mu; writes theta, its record and constants.
__device__ void sweep_f(const GibbsArgs& A, const float (&tot)[NSTAT], float x0, float (&th)[5])
{
    const int lane = threadIdx.x & 31;
    WarpDrawsF st;
    st.seed = A.seed;
    st.series = A.series;
    st.traj = A.traj;
    st.fill(A.T);
    int acc = 0;
    gibbs_draws_f(tot, x0, A.T, th, st, A.mask, &acc);
    if (lane < 5) {
        float v = th[0];
#pragma unroll
        for (int k = 1; k < 5; ++k)
            if (lane == k) v = th[k];
        A.theta[lane] = (double)v;
        if (A.theta_out) A.theta_out[lane] = (double)v;
    }
    if (lane == 0) {
        if (A.phi_acc) *A.phi_acc = acc;
        *A.theta_f = mixed_theta_f(th);
        if (A.counter) *A.counter = 0u;
    }
    __threadfence();
}

// Mixed path: the statistics in double-float (FP32 arithmetic; the FP64 pipe
// of this GPU is slow) from (hi, lo) state, centred on the constants of
// theta_f; the last block combines them, one warp per statistic, and warp 0
// takes the sweep in FP32 (variates in registers, no block barriers), writes
// theta (FP32-valued) and refreshes theta_f.
constexpr int kGibbsMixedBlock = 256;
__global__ void __launch_bounds__(kGibbsMixedBlock, 2) k_gibbs_mixed(GibbsArgs A)
{
    __shared__ float2 redf[kGibbsMixedBlock / 32][NSTAT];
    __shared__ float2 s_tot[NSTAT];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cur = A.cur ? *(volatile int*)A.cur : 0;
    const float2* h = cur ? A.h1f : A.h0f;
    const MixedTheta& m0 = *A.theta_f;
    const ff mu = m0.mu;
    // the FP32 theta of the sweep (the hi parts of the prepared constants)
    const float xi_f = ff_sub(m0.ximu, m0.mu).hi, mu_f = m0.mu.hi, phi_f = m0.phi_ff.hi;
    {
        float sf[NSTAT];
        for (int i = 0; i < NSTAT; ++i) sf[i] = 0.f;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        // U sites per thread per round, their loads issued before any of
        // their arithmetic (the pass is bound by load latency otherwise)
        constexpr int U = 4;
        for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < A.T;
             t0 += U * stride) {
            float2 hv[U], lv[U], hn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = t0 + u * stride;
                hv[u] = lv[u] = hn[u] = make_float2(0.f, 0.f);
                if (t < A.T) {
                    hv[u] = h[t];
                    lv[u] = A.lr_f[t];
                    if (t + 1 < A.T) hn[u] = h[t + 1];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = t0 + u * stride;
                if (t < A.T) {
                    // the chain's snapshot of h, taken on the way
                    if (A.snap_out) A.snap_out[t] = hv[u].x + hv[u].y;
                    site_stats_f(hv[u], lv[u], hn[u], t, A.T, xi_f, mu_f, phi_f, sf);
                }
            }
        }
        ff s[NSTAT];
        for (int i = 0; i < NSTAT; ++i) s[i] = ff{sf[i], 0.f};
        block_sum_ff(s, redf);
        float2* pf = reinterpret_cast<float2*>(A.partials);
        if (threadIdx.x == 0)
            for (int i = 0; i < NSTAT; ++i)
                pf[(int64_t)blockIdx.x * NSTAT + i] = make_float2(s[i].hi, s[i].lo);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // warp w sums statistic w over the blocks (NSTAT == warps per block)
    static_assert(NSTAT == kGibbsMixedBlock / 32, "one warp per statistic");
    {
        const float2* pf = reinterpret_cast<const float2*>(A.partials);
        ff acc = {0.f, 0.f};
        const int nb = (int)gridDim.x;
        // up to 16 partials per lane (the grid is at most 2 x 152 blocks,
        // 10 per lane), all loads issued before the sums
        constexpr int NB = 16;
        for (int b0 = lane; b0 < nb; b0 += 32 * NB) {
            float2 v[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int b = b0 + 32 * i;
                v[i] = b < nb ? __ldcg(pf + (int64_t)b * NSTAT + warp) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) acc = ff_add(acc, ff{v[i].x, v[i].y});
        }
        acc = warp_sum_ff(acc);
        if (lane == 0) s_tot[warp] = make_float2(acc.hi, acc.lo);
    }
    __syncthreads();
    if (warp != 0) return;
    float tot[NSTAT];
    for (int i = 0; i < NSTAT; ++i) tot[i] = s_tot[i].x + s_tot[i].y;
    float th[5];
    theta_f32(A, th);
    const float2 hv = h[0];
    const ff x0 = ff_sub(ff{hv.x, hv.y}, mu);
    sweep_f(A, tot, x0.hi + x0.lo, th);
}

// The same sweep with its sums from the statistics of the current state (no
// pass over the sites, see record_sums): one warp.
__global__ void __launch_bounds__(32) k_gibbs_stats(GibbsArgs A)
{
    const int cur = A.cur ? *(volatile int*)A.cur : 0;
    const StatsRec r = A.rstats[cur];
    float th[5];
    theta_f32(A, th);
    float tot[NSTAT], x0;
    record_sums(r, th, A.T, tot, x0);
    sweep_f(A, tot, x0, th);
}

}  // namespace

// FP64 path: about 4 sites per thread, up to 8 blocks of 256 per SM.  Mixed
// path: one wave of two blocks of 256 per SM (loads of four sites in flight).
int gibbs_grid(int64_t T)
{
    int64_t g = (T + 1023) / 1024;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}
static int gibbs_grid_mixed(int64_t T)
{
    int64_t g = (T + 2047) / 2048;
    if (g > 152 * 2) g = 152 * 2;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_gibbs(const GibbsArgs& a, bool mixed, cudaStream_t st)
{
    if (mixed && a.rstats) k_gibbs_stats<<<1, 32, 0, st>>>(a);
    else if (mixed) k_gibbs_mixed<<<gibbs_grid_mixed(a.T), kGibbsMixedBlock, 0, st>>>(a);
    else k_gibbs<<<gibbs_grid(a.T), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rsv
