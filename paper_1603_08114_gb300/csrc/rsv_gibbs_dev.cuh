// rsv_gibbs_dev.cuh -- device code of the mixed (FP32) theta sweep, shared by
// the theta kernels (rsv_gibbs.cu) and the persistent chain kernel
// (rsv_chain.cu).  See rsv_gibbs.cu for the conditionals (the paper does not
// describe its theta update).
#pragma once

#include <cmath>

#include "rsv_device.cuh"
#include "rsv_traj.cuh"

namespace rsv {
namespace {

constexpr int NSTAT = 8;  // sum q, sum q^2, X_a, X_b, XX_m, XY, sum e, sum e^2

// ---------------------------------------------------------------------------
// Mixed path: the same sweep in FP32.  Stream positions are consumed in the
// same order, with 23-bit uniforms (k + 1/2) 2^-23 of the same Philox words;
// theta is kept FP32-valued, so that the mixed trajectory kernel's constants
// follow from it in FP32 / double-float arithmetic.  A rounding of theta to
// FP32 after each draw moves it by ~1e-7 relative, far below its posterior
// spread.  Marsaglia & Tsang's acceptance value
//   r = z^2/2 + d (1 - v + ln v),  v = (1 + x)^3,  x = c z,  c^2 = 1/(9 d),
// is taken for |x| < 1/4 from its expansion: with ln v = 3 ln(1 + x) the
// terms of order x^2 cancel against z^2/2 exactly and
//   r = 3 d sum_{k>=4} (-1)^(k+1) x^k / k
// (in FP32 the direct form loses everything to cancellation when d ~ T/2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mt_accept_value(float z, float c, float d)
{
    const float x = c * z;
    if (fabsf(x) < 0.25f) {
        // Horner over k = 20 .. 4 of (-1)^(k+1) x^(k-4) / k
        float sacc = 0.0f;
#pragma unroll
        for (int k = 20; k >= 4; --k) sacc = fmaf(sacc, x, ((k & 1) ? 1.0f : -1.0f) / (float)k);
        const float x2 = x * x;
        return 3.0f * d * (x2 * x2) * sacc;
    }
    const float v = (1.0f + x) * (1.0f + x) * (1.0f + x);
    return 0.5f * z * z + d - d * v + d * (3.0f * log1pf(x));
}

__device__ __forceinline__ float u01_23_at(uint64_t seed, uint64_t series, uint64_t traj, int i)
{
    const u64x4 w = philox_block(seed, series, traj, STREAM_THETA, (uint64_t)(i >> 2));
    return u01_23(w.w[i & 3]);
}

// The variates of stream positions 0..31 in the registers of one warp (lane
// i holds position i) and the walk over them: a position the warp holds is
// read by a shuffle (the position is the same in every lane), any other is
// computed directly.
struct WarpDrawsF {
    uint64_t seed, series, traj;
    float u, lu, z, v, g;   // this lane's position: uniform, log, normal, candidate
    int acc;                // candidate at this position accepted
    float gc, gd;           // Marsaglia-Tsang c, d of the sweep's gamma shape
    float alpha_pre;
    int pos;
    __device__ void fill(int64_t T)
    {
        const int lane = threadIdx.x & 31;
        const float Tf = (float)T;
        alpha_pre = 0.5f * Tf < 1.0f ? 0.5f * Tf + 1.0f : 0.5f * Tf;
        gd = alpha_pre - 1.0f / 3.0f;
        gc = 1.0f / sqrtf(9.0f * gd);
        u = u01_23_at(seed, series, traj, lane);
        lu = logf(u);
        const float un = __shfl_down_sync(0xffffffffu, u, 1);  // position i+1 (lane 31: unused)
        z = sqrtf(-2.0f * lu) * cospif(2.0f * un);
        v = 1.0f + gc * z;
        g = gd * (v * v * v);
        const float lu2 = __shfl_down_sync(0xffffffffu, lu, 2);  // position i+2
        acc = (lane < 30 && v > 0.0f && lu2 < mt_accept_value(z, gc, gd)) ? 1 : 0;
        pos = 0;
    }
    __device__ float uni(int i) const
    {
        const float r = __shfl_sync(0xffffffffu, u, i & 31);
        return i < 32 ? r : u01_23_at(seed, series, traj, i);
    }
    __device__ float loguni(int i) const
    {
        const float r = __shfl_sync(0xffffffffu, lu, i & 31);
        return i < 32 ? r : logf(uni(i));
    }
    __device__ float normal()
    {
        const int i = pos;
        pos += 2;
        const float r = __shfl_sync(0xffffffffu, z, i & 31);
        return i < 31 ? r : sqrtf(-2.0f * loguni(i)) * cospif(2.0f * uni(i + 1));
    }
    __device__ float gamma(float alpha)
    {
        if (alpha < 1.0f) {
            const float gg = gamma1(alpha + 1.0f);
            const float uu = uni(pos++);
            return gg * powf(uu, 1.0f / alpha);
        }
        return gamma1(alpha);
    }
    __device__ float gamma1(float alpha)
    {
        const bool pre = alpha == alpha_pre;
        const float d = pre ? gd : alpha - 1.0f / 3.0f;
        const float c = pre ? gc : 1.0f / sqrtf(9.0f * d);
        for (int it = 0; it < 1000; ++it) {
            const int i = pos;
            if (pre && i < 30) {
                const float vi = __shfl_sync(0xffffffffu, v, i);
                const int ai = __shfl_sync(0xffffffffu, acc, i);
                const float gi = __shfl_sync(0xffffffffu, g, i);
                pos += vi > 0.0f ? 3 : 2;
                if (ai) return gi;
                continue;
            }
            const float zz = normal();
            const float vv = 1.0f + c * zz;
            if (vv <= 0.0f) continue;
            const float l = loguni(pos++);
            if (l < mt_accept_value(zz, c, d)) return d * vv * vv * vv;
        }
        return NAN;
    }
};

// One sweep in FP32 (every lane of one warp calls it uniformly); theta as
// floats in/out; x0 = h_1 - mu; S the statistics.
__device__ void gibbs_draws_f(const float (&S)[NSTAT], float x0, int64_t T, float (&th)[5],
                              WarpDrawsF& st, int mask, int* acc_out)
{
    const float Tf = (float)T;
    const float phi = th[0], mu0 = th[1], xi0 = th[2];
    float se2 = th[3], su2 = th[4];
    float xi = xi0, mu = mu0, ph = phi;
    if (mask & 1) xi = xi0 + S[0] / Tf + sqrtf(su2 / Tf) * st.normal();
    if (mask & 2) {
        const float dxi = xi - xi0;
        const float ss = S[1] - 2.0f * dxi * S[0] + Tf * dxi * dxi;
        const float g = st.gamma(0.5f * Tf);
        if (g > 0.0f && ss > 0.0f) su2 = 0.5f * ss / g;
    }
    if (mask & 4) {
        const float w0 = 1.0f - phi * phi, w1 = (1.0f - phi) * (1.0f - phi);
        const float den = w0 + (Tf - 1.0f) * w1;
        const float m = mu0 + (w0 * x0 + (1.0f - phi) * S[6]) / den;
        mu = m + st.normal() / sqrtf(den / se2);
    }
    const float dmu = mu - mu0;
    if (mask & 8) {
        const float a = x0 - dmu, om = 1.0f - phi;
        const float Q = (1.0f - phi * phi) * a * a + S[7] - 2.0f * om * dmu * S[6] +
                        (Tf - 1.0f) * om * om * dmu * dmu;
        const float g = st.gamma(0.5f * Tf);
        if (g > 0.0f && Q > 0.0f) se2 = 0.5f * Q / g;
    }
    int acc = 0;
    if (mask & 16) {
        const float num = S[5] - dmu * (S[2] + S[3]) + (Tf - 1.0f) * dmu * dmu;
        const float Xm = S[2] - x0;
        const float D = S[4] - 2.0f * dmu * Xm + (Tf - 2.0f) * dmu * dmu;
        if (T >= 3 && D > 0.0f) {
            const float m = num / D, sd = sqrtf(se2 / D);
            float prop = NAN;
            for (int it = 0; it < 1000; ++it) {
                const float c = m + sd * st.normal();
                if (c > -1.0f && c < 1.0f) {
                    prop = c;
                    break;
                }
            }
            const float lu = st.loguni(st.pos++);
            if (prop == prop) {
                const float lr = 0.5f * logf(1.0f - prop * prop) - 0.5f * logf(1.0f - phi * phi);
                if (lu < lr) {
                    ph = prop;
                    acc = 1;
                }
            }
        }
    }
    th[0] = ph;
    th[1] = mu;
    th[2] = xi;
    th[3] = se2;
    th[4] = su2;
    *acc_out = acc;
}


// The sums of the FP32 sweep from the statistics record r of the current
// state (no pass over the sites), and x0 = h_1 - mu.  The record's sums, centred at its mu_r,
// are moved to the sweep's FP32 theta (x = h - mu, q = lnRV - xi - h,
// e = x_{t+1} - phi x_t) in double-float:
//   x' = x_r + d (d = mu_r - mu):  Sx = sx + T d,  Sxx = sxx + 2 d sx + T d^2,
//     Sxn = sxn + d (2 sx - x_0 - x_{T-1}) + (T-1) d^2,  Sxl = sxl + d sl;
//   with c = xi + mu:  sum q = sl - T c - Sx,
//     sum q^2 = Sxx - 2 Sxl + 2 c Sx + sll - 2 c sl + T c^2;
//   X_a = Sx - x_{T-1},  X_b = Sx - x_0,  XX_m = Sxx - x_0^2 - x_{T-1}^2 (T > 1),
//   XY = Sxn,  sum e = X_b - phi X_a,
//   sum e^2 = (Sxx - x_0^2) - 2 phi Sxn + phi^2 (Sxx - x_{T-1}^2).
__device__ __forceinline__ void record_sums(const StatsRec& r, const float (&th)[5], int64_t T,
                                            float (&tot)[NSTAT], float& x0f)
{
    const float thf = (float)T;
    const ff Tf = {thf, (float)(T - (int64_t)thf)};
    const ff T1 = ff_add(Tf, ff{-1.f, 0.f});
    const StateStats& s = r.s;
    const ff d = ff_sub(r.mu, ff{th[1], 0.f});
    const ff d2 = ff_mul(d, d);
    const ff Sx = ff_add(s.sx, ff_mul(Tf, d));
    const ff Sxx = ff_add(ff_add(s.sxx, ff_mul(ff_mul_f(d, 2.f), s.sx)), ff_mul(Tf, d2));
    const ff Sxn = ff_add(ff_add(s.sxn, ff_mul(d, ff_sub(ff_mul_f(s.sx, 2.f), ff_add(s.x0, s.xT)))),
                          ff_mul(T1, d2));
    const ff Sxl = ff_add(s.sxl, ff_mul(d, r.sl));
    const ff x0 = ff_add(s.x0, d), xT = ff_add(s.xT, d);
    const ff c = two_sum(th[2], th[1]);
    const ff x0s = ff_mul(x0, x0), xTs = ff_mul(xT, xT);
    const ff phi = {th[0], 0.f};
    ff S[NSTAT];
    S[0] = ff_sub(ff_sub(r.sl, ff_mul(Tf, c)), Sx);
    S[1] = ff_add(ff_sub(Sxx, ff_mul_f(Sxl, 2.f)), ff_mul(ff_mul_f(c, 2.f), Sx));
    S[1] = ff_add(S[1], ff_sub(r.sll, ff_mul(ff_mul_f(c, 2.f), r.sl)));
    S[1] = ff_add(S[1], ff_mul(Tf, ff_mul(c, c)));
    S[2] = ff_sub(Sx, xT);
    S[3] = ff_sub(Sx, x0);
    S[4] = T > 1 ? ff_sub(ff_sub(Sxx, x0s), xTs) : ff{0.f, 0.f};
    S[5] = Sxn;
    S[6] = ff_sub(S[3], ff_mul(phi, S[2]));
    S[7] = ff_add(ff_sub(ff_sub(Sxx, x0s), ff_mul(ff_mul_f(phi, 2.f), Sxn)),
                  ff_mul(ff_mul(phi, phi), ff_sub(Sxx, xTs)));
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) tot[i] = S[i].hi + S[i].lo;
    x0f = x0.hi + x0.lo;
}

}  // namespace
}  // namespace rsv
