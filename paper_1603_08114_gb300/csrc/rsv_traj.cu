// rsv_traj.cu -- one HMC trajectory of the RSV model, tiled over the series.
//
// Method (arXiv:1603.08114, Sec. 3): leapfrog eqs. (6)-(8) repeated n_md times,
// dH = H(p', h') - H(p, h), Metropolis min{1, e^{-dH}}.
//
// GB300 design.  The paper launches three kernels per leapfrog step from the
// host (Sec. 5).  Here one block integrates a whole trajectory of its tile on
// chip: the tile's window, widened by K = n_md + 1 sites on each side, is held
// in registers (J sites per thread), neighbours are exchanged by warp shuffles
// and a small shared-memory edge buffer once per step, and no block ever waits
// for another.  Sites within n_md of a window edge go stale one site per step,
// so after n_md steps the owned sites (and the one right neighbour that dH
// needs) are exactly what an untiled integration gives.  Each block writes its
// part of dH; the last block to finish sums the parts in a fixed order and
// takes the Metropolis decision.
//
// State is kept in x = h - mu so that the force reads
//   dS/dh = ie * AR + iu * x + (1/2 - c' iu) - a' e^{-x},
//   AR_t = e_{t-1} - phi e_t,  e_t = x_{t+1} - phi x_t  (e_{T-1} = 0,
//   e_{-1} = (1 - phi^2) x_0), a' = y^2/2 e^{-mu}, c' = lnRV - xi - mu,
// which is the gradient of S written with the AR innovations e_t (the same
// stencil as eq. (7)'s (1+phi^2) x_t - phi (x_{t-1} + x_{t+1}) inside).
#include <cmath>
#include <cstdio>

#include "rsv_device.cuh"
#include "rsv_traj.cuh"

namespace rsv {

namespace {

constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the special-function unit (ex2.approx.ftz.f32: relative error about
// 2^-22; 2^-inf = +0).
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exchange the first and last value of each thread's slot run with its
// neighbours: left_last = last value of thread tid-1, right_first = first
// value of thread tid+1.  `edge` is one of two alternating buffers of 2*nw.
template <typename V>
__device__ __forceinline__ void exchange(V first, V last, V& left_last, V& right_first, V* edge,
                                         int nw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    left_last = __shfl_up_sync(0xffffffffu, last, 1);
    right_first = __shfl_down_sync(0xffffffffu, first, 1);
    if (lane == 0) edge[2 * warp] = first;
    if (lane == 31) edge[2 * warp + 1] = last;
    __syncthreads();
    if (lane == 0) left_last = warp > 0 ? edge[2 * (warp - 1) + 1] : first;
    if (lane == 31) right_first = warp + 1 < nw ? edge[2 * (warp + 1)] : last;
}

struct Window {
    int64_t lo, hi, wlo, whi;
    int n;
};
__device__ __forceinline__ Window window_of(int64_t T, int64_t tile, int K)
{
    Window w;
    w.lo = (int64_t)blockIdx.x * tile;
    w.hi = min(T, w.lo + tile);
    w.wlo = max(w.lo - (int64_t)K, (int64_t)0) & ~(int64_t)3;
    w.whi = min(T, w.hi + (int64_t)K);
    w.n = (int)(w.whi - w.wlo);
    return w;
}

// Innovations e_j = x_{j+1} - phi x_j of one thread's run (xR = first x of the
// next thread), with e forced to 0 at the window's last active slot `la`.
template <int J, typename V, bool EDGE>
__device__ __forceinline__ void innovations(const V (&x)[J], V xR, V phi, int la, V (&e)[J])
{
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const V nx = (j + 1 < J) ? x[j + 1] : xR;
        e[j] = fma(-phi, x[j], nx);
        if (EDGE && j == la) e[j] = V(0);
    }
}

// Finish of a trajectory: called by every block after it has written its
// partial dH; the last block to arrive sums all partials in block order,
// draws or reads ln u and takes the Metropolis decision.
__device__ void finish(const TrajArgs& A, double part, int cur, double* red)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        A.partials[blockIdx.x] = part;
        __threadfence();
        const unsigned prev = atomicAdd(A.counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(A.partials + i);
    const double dH = block_sum(v, red);
    if (threadIdx.x == 0) {
        *A.counter = 0u;
        double lu;
        if (A.log_u) {
            lu = *A.log_u;
        } else {
            const u64x4 w = philox_block(A.seed, A.series, A.traj, STREAM_MH, 0);
            lu = log(u01_53(w.w[0]));
        }
        const bool fin = isfinite(dH);
        const int acc = (fin && lu < -dH) ? 1 : 0;
        if (!fin) atomicOr(A.status, ST_NONFINITE);
        *A.dH_out = dH;
        *A.acc_out = acc;
        if (A.cur && acc) *(volatile int*)A.cur = cur ^ 1;
        if (A.fb_state && A.fallback_window > 0) {
            int na = A.fb_state[0] + acc, nt = A.fb_state[1] + 1;
            if (nt >= A.fallback_window) {
                if (A.mass_on && *A.mass_on && 10 * na < 6 * nt) *(int*)A.mass_on = 0;
                na = 0;
                nt = 0;
            }
            A.fb_state[0] = na;
            A.fb_state[1] = nt;
        }
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// FP64 path.  Shared memory (slot-major, index j*NT + tid): a'[W], kc[W],
// minv[W] (MASS), edge buffers [2][2*nw], reduction scratch [nw].
// ---------------------------------------------------------------------------
template <int J, bool MASS>
__global__ void __launch_bounds__(256, 1) k_traj_fp64(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NT = blockDim.x, W = NT * J, nw = NT >> 5, tid = threadIdx.x;
    double* s_a = reinterpret_cast<double*>(smem_raw);
    double* s_kc = s_a + W;
    double* s_mi = s_kc + W;
    double* s_edge = s_mi + (MASS ? W : 0);
    double* s_red = s_edge + 4 * nw;

    const ThetaD th = A.theta ? load_theta(A.theta) : A.th_inline;
    const double phi = th.phi, mu = th.mu;
    const double ie = 1.0 / th.se2, iu = 1.0 / th.su2;
    const double emu = exp(-mu);
    const double st0 = 1.0 - phi * phi;
    const Window w = window_of(A.T, A.tile, A.K);
    const int base = tid * J;
    const int la = w.n - 1 - base;
    const bool edge_thread = (la >= 0 && la < J);
    const int cur = A.cur ? *(volatile int*)A.cur : 0;
    const double* hin = cur ? A.h1d : A.h0d;
    double* hout = cur ? const_cast<double*>(A.h0d) : A.h1d;
    const bool mass_on = MASS && (A.mass_on == nullptr || *A.mass_on != 0);

    double x[J], p[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int i = base + j;
        const int64_t s = w.wlo + i;
        const bool act = i < w.n;
        const double hv = act ? hin[s] : mu;
        const double yv = act ? A.y[s] : 0.0;
        const double lr = act ? A.lnrv[s] : th.xi + mu;
        x[j] = hv - mu;
        s_a[j * NT + tid] = 0.5 * yv * yv * emu;
        s_kc[j * NT + tid] = 0.5 - ((lr - th.xi) - mu) * iu;
        if (MASS) s_mi[j * NT + tid] = (act && mass_on) ? (double)A.minv[s] : 1.0;
    }
    if (A.p_in) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = base + j;
            p[j] = i < w.n ? A.p_in[w.wlo + i] : 0.0;
        }
    } else {
#pragma unroll
        for (int q = 0; q < J / 4; ++q) {
            const int64_t s0 = w.wlo + base + 4 * q;
            const u64x4 r = philox_block(A.seed, A.series, A.traj, STREAM_MOM, (uint64_t)(s0 >> 2));
            box_muller(u01_53(r.w[0]), u01_53(r.w[1]), p[4 * q + 0], p[4 * q + 1]);
            box_muller(u01_53(r.w[2]), u01_53(r.w[3]), p[4 * q + 2], p[4 * q + 3]);
        }
        if (MASS) {
#pragma unroll
            for (int j = 0; j < J; ++j) p[j] = p[j] / sqrt(s_mi[j * NT + tid]);
        }
    }
    __syncthreads();

    // H(p, h) restricted to the owned sites of this thread (per-site action
    // s_t in x coordinates; the constant mu/2 per site cancels in dH).
    int par = 0;
    auto owned_energy = [&](double& acc) {
        double xL, xR, e[J];
        exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
        par ^= 1;
        if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
        else innovations<J, double, false>(x, xR, phi, la, e);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int64_t s = w.wlo + base + j;
            if (s >= w.lo && s < w.hi) {
                const double cp = (A.lnrv[s] - th.xi) - mu;
                const double r = cp - x[j];
                double v = 0.5 * x[j] + s_a[j * NT + tid] * exp(-x[j]) + 0.5 * iu * r * r
                         + 0.5 * ie * e[j] * e[j];
                if (s == 0) v += 0.5 * ie * st0 * x[j] * x[j];
                const double mi = MASS ? s_mi[j * NT + tid] : 1.0;
                v += 0.5 * mi * p[j] * p[j];
                acc += v;
            }
        }
    };
    double E0 = 0.0, E1 = 0.0;
    owned_energy(E0);

    const double dt = A.dtau, hd = 0.5 * A.dtau;
    for (int k = 0; k < A.n_md; ++k) {
        // eq. (6): h(tau + dtau/2) = h(tau) + dtau/2 p / m
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const double c = MASS ? hd * s_mi[j * NT + tid] : hd;
            x[j] = fma(c, p[j], x[j]);
        }
        double xL, xR, e[J];
        exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
        par ^= 1;
        if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
        else innovations<J, double, false>(x, xR, phi, la, e);
        // e_{-1}: left neighbour's innovation, or the stationary term at a window start
        double eprev = (tid == 0) ? st0 * x[0] : fma(-phi, xL, x[0]);
        // eq. (7): p(tau + dtau) = p(tau) - dtau dS/dh
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const double ar = fma(-phi, e[j], eprev);
            eprev = e[j];
            double f = fma(iu, x[j], s_kc[j * NT + tid]);
            f = fma(ie, ar, f);
            f = fma(-s_a[j * NT + tid], exp(-x[j]), f);
            p[j] = fma(-dt, f, p[j]);
        }
        // eq. (8): h(tau + dtau) = h(tau + dtau/2) + dtau/2 p / m
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const double c = MASS ? hd * s_mi[j * NT + tid] : hd;
            x[j] = fma(c, p[j], x[j]);
        }
    }

    owned_energy(E1);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int64_t s = w.wlo + base + j;
        if (s >= w.lo && s < w.hi) {
            hout[s] = x[j] + mu;
            if (A.p_out) A.p_out[s] = p[j];
        }
    }
    const double part = block_sum(E1 - E0, s_red);
    finish(A, part, cur, s_red);
}

// ---------------------------------------------------------------------------
// Mixed path: FP32 leapfrog on a compensated (hi, lo) state, dH in
// double-float per site with FP64 accumulation across threads.
// Shared memory (slot-major): x0 hi/lo, p0 hi/lo [W each], edge [2][2*nw]
// float2, reduction scratch [nw] double.
// ---------------------------------------------------------------------------
template <int J, bool MASS>
__global__ void __launch_bounds__(384, 1) k_traj_mixed(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NT = blockDim.x, W = NT * J, nw = NT >> 5, tid = threadIdx.x;
    double* s_red = reinterpret_cast<double*>(smem_raw);
    float2* s_edge = reinterpret_cast<float2*>(s_red + 32);
    float* s_x0h = reinterpret_cast<float*>(s_edge + 4 * 32);
    float* s_x0l = s_x0h + W;
    float* s_p0h = s_x0l + W;
    float* s_p0l = s_p0h + W;

    const ThetaD th = A.theta ? load_theta(A.theta) : A.th_inline;
    const float phif = (float)th.phi;
    const float ief = (float)(1.0 / th.se2), iuf = (float)(1.0 / th.su2);
    const float dt = (float)A.dtau;
    const ff mu_ff = ff_from_double(th.mu);
    const ff ximu_ff = ff_from_double(th.xi + th.mu);
    const float bshift = (float)(th.mu * 1.4426950408889634);
    const Window w = window_of(A.T, A.tile, A.K);
    const int base = tid * J;
    const int la = w.n - 1 - base;
    const bool edge_thread = (la >= 0 && la < J);
    const int cur = A.cur ? *(volatile int*)A.cur : 0;
    const float2* hin = cur ? A.h1f : A.h0f;
    float2* hout = cur ? const_cast<float2*>(A.h0f) : A.h1f;
    const bool mass_on = MASS && (A.mass_on == nullptr || *A.mass_on != 0);

    float xh[J], xl[J], ph[J], pl[J], bm[J], kf[J];
    float dtm[MASS ? J : 1];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int i = base + j;
        const int64_t s = w.wlo + i;
        const bool act = i < w.n;
        const float2 hv = act ? hin[s] : make_float2(mu_ff.hi, mu_ff.lo);
        // x = h - mu in double-float
        ff x = two_sum(hv.x, -mu_ff.hi);
        x.lo += hv.y - mu_ff.lo;
        x = fast_two_sum(x.hi, x.lo);
        xh[j] = x.hi;
        xl[j] = x.lo;
        const float b0 = act ? A.b0_f[s] : -INFINITY;
        bm[j] = b0 - bshift;  // log2(y^2/2 e^{-mu})
        const float2 lr = act ? A.lr_f[s] : make_float2(ximu_ff.hi, ximu_ff.lo);
        ff cp = two_sum(lr.x, -ximu_ff.hi);  // c' = lnRV - xi - mu
        cp.lo += lr.y - ximu_ff.lo;
        kf[j] = fmaf(-iuf, cp.hi + cp.lo, 0.5f);
        if (MASS) dtm[MASS ? j : 0] = (act && mass_on) ? A.minv[s] : 1.0f;
    }
    if (A.p_in) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = base + j;
            const double pv = i < w.n ? A.p_in[w.wlo + i] : 0.0;
            const ff pf = ff_from_double(pv);
            ph[j] = pf.hi;
            pl[j] = pf.lo;
        }
    } else {
#pragma unroll
        for (int q = 0; q < J / 4; ++q) {
            const int64_t s0 = w.wlo + base + 4 * q;
            const u64x4 r = philox_block(A.seed, A.series, A.traj, STREAM_MOM, (uint64_t)(s0 >> 2));
            box_muller_f(u01_23(r.w[0]), u01_23(r.w[1]), ph[4 * q + 0], ph[4 * q + 1]);
            box_muller_f(u01_23(r.w[2]), u01_23(r.w[3]), ph[4 * q + 2], ph[4 * q + 3]);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (MASS) ph[j] = ph[j] / sqrtf(dtm[MASS ? j : 0]);
            pl[j] = 0.0f;
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        s_x0h[j * NT + tid] = xh[j];
        s_x0l[j * NT + tid] = xl[j];
        s_p0h[j * NT + tid] = ph[j];
        s_p0l[j * NT + tid] = pl[j];
        if (MASS) dtm[MASS ? j : 0] *= dt;  // dtau / m_t
    }
    int par = 0;

    // Compensated update v += c*u of a (hi, lo) pair: lo carries what hi lost.
    auto cupd = [](float& hi, float& lo, float c, float u) {
        const float y = fmaf(c, u, lo);
        const float t = hi + y;
        lo = y - (t - hi);
        hi = t;
    };

    // Leapfrog with the two half steps of consecutive steps merged:
    // x += dt/2 p; n_md times { p -= dt F(x); x += (dt or dt/2 at the end) p }.
#pragma unroll
    for (int j = 0; j < J; ++j) cupd(xh[j], xl[j], MASS ? 0.5f * dtm[MASS ? j : 0] : 0.5f * dt, ph[j]);
    for (int k = 0; k < A.n_md; ++k) {
        float xL, xR, e[J];
        exchange(xh[0], xh[J - 1], xL, xR, reinterpret_cast<float*>(s_edge) + par * 2 * nw, nw);
        par ^= 1;
        if (edge_thread) innovations<J, float, true>(xh, xR, phif, la, e);
        else innovations<J, float, false>(xh, xR, phif, la, e);
        float eprev = (tid == 0) ? (1.0f - phif * phif) * xh[0] : fmaf(-phif, xL, xh[0]);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float ar = fmaf(-phif, e[j], eprev);
            eprev = e[j];
            float f = fmaf(iuf, xh[j], kf[j]);
            f = fmaf(ief, ar, f);
            f -= ex2_approx(fmaf(-kLog2e, xh[j], bm[j]));
            cupd(ph[j], pl[j], -dt, f);
        }
        const float hs = (k + 1 < A.n_md) ? 1.0f : 0.5f;
#pragma unroll
        for (int j = 0; j < J; ++j) cupd(xh[j], xl[j], MASS ? hs * dtm[MASS ? j : 0] : hs * dt, ph[j]);
    }

    // ---- dH: per-site differences in double-float -------------------------
    // K = sum (p'^2 - p^2)/m, L = sum (x' - x), R = sum (x'-c')^2 - (x-c')^2,
    // Q = sum e'^2 - e^2, E = sum a (e^{-h'} - e^{-h});
    // dH = K/2 + L/2 + R/(2 s_u^2) + Q/(2 s_eta^2) + E + stationary term.
    ff accK = {0.f, 0.f}, accL = {0.f, 0.f}, accR = {0.f, 0.f}, accQ = {0.f, 0.f},
       accE = {0.f, 0.f};
    double stat = 0.0;
    const ff phi_ff = ff_from_double(th.phi);
    {
        float xLh, xRh, xLl, xRl;
        exchange(xh[0], xh[J - 1], xLh, xRh, reinterpret_cast<float*>(s_edge) + par * 2 * nw, nw);
        par ^= 1;
        exchange(xl[0], xl[J - 1], xLl, xRl, reinterpret_cast<float*>(s_edge) + par * 2 * nw, nw);
        par ^= 1;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = base + j;
            const int64_t s = w.wlo + i;
            if (s < w.lo || s >= w.hi) continue;
            const ff x1 = {xh[j], xl[j]};
            const ff x0 = {s_x0h[j * NT + tid], s_x0l[j * NT + tid]};
            const ff d = ff_sub(x1, x0);
            ff_acc(accL, d);
            // kinetic
            ff q1 = two_prod(ph[j], ph[j]);
            q1.lo = fmaf(2.0f * ph[j], pl[j], q1.lo);
            const float p0h = s_p0h[j * NT + tid], p0l = s_p0l[j * NT + tid];
            ff q0 = two_prod(p0h, p0h);
            q0.lo = fmaf(2.0f * p0h, p0l, q0.lo);
            ff dk = ff_sub(q1, q0);
            if (MASS) dk = ff_mul_f(dk, dtm[MASS ? j : 0] / dt);
            ff_acc(accK, dk);
            // realized-volatility term: (x'-x)(x'+x-2c')
            const float2 lr = A.lr_f[s];
            ff cp = two_sum(lr.x, -ximu_ff.hi);
            cp.lo += lr.y - ximu_ff.lo;
            ff sgm = ff_add(x1, x0);
            sgm = ff_sub(sgm, ff{2.0f * cp.hi, 2.0f * cp.lo});
            ff_acc(accR, ff_mul(d, sgm));
            // AR term: e' and e of site s need site s+1
            if (s + 1 < A.T) {
                ff n1, n0;
                if (j + 1 < J) {
                    n1 = {xh[j + 1], xl[j + 1]};
                    n0 = {s_x0h[(j + 1) * NT + tid], s_x0l[(j + 1) * NT + tid]};
                } else {
                    n1 = {xRh, xRl};
                    n0 = {s_x0h[tid + 1], s_x0l[tid + 1]};
                }
                const ff e1 = ff_sub(n1, ff_mul(phi_ff, x1));
                const ff e0 = ff_sub(n0, ff_mul(phi_ff, x0));
                ff_acc(accQ, ff_mul(ff_sub(e1, e0), ff_add(e1, e0)));
            }
            if (s == 0) {
                const double a1 = ff_to_double(x1), a0 = ff_to_double(x0);
                stat = 0.5 * (1.0 - th.phi * th.phi) / th.se2 * (a1 * a1 - a0 * a0);
            }
            // return term: a e^{-h} (e^{-(h'-h)} - 1)
            const float h0f = x0.hi + mu_ff.hi;
            const float E0 = A.a_f[s] * expf(-h0f);
            const float re = E0 * expm1f(-d.hi);
            ff_acc(accE, ff{re, 0.0f});
        }
    }
    ff tot = ff_add(ff_add(ff_mul_f(accK, 0.5f), ff_mul_f(accL, 0.5f)), accE);
    tot = ff_add(tot, ff_mul(accR, ff_from_double(0.5 / th.su2)));
    tot = ff_add(tot, ff_mul(accQ, ff_from_double(0.5 / th.se2)));
    tot = warp_sum_ff(tot);
    double mine = (threadIdx.x & 31) == 0 ? ff_to_double(tot) : 0.0;
    mine += stat;

    // write the proposal (h as (hi, lo)) and p'
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int64_t s = w.wlo + base + j;
        if (s >= w.lo && s < w.hi) {
            ff h = two_sum(xh[j], mu_ff.hi);
            h.lo += xl[j] + mu_ff.lo;
            h = fast_two_sum(h.hi, h.lo);
            hout[s] = make_float2(h.hi, h.lo);
            if (A.p_out) A.p_out[s] = (double)ph[j] + (double)pl[j];
        }
    }
    const double part = block_sum(mine, s_red);
    finish(A, part, cur, s_red);
}

// ---------------------------------------------------------------------------
// Small element-wise kernels.
// ---------------------------------------------------------------------------
__global__ void k_commit_fp64(double* __restrict__ h, const double* __restrict__ hprop,
                              double* __restrict__ p, const double* __restrict__ pprop,
                              const int* __restrict__ acc, int64_t T)
{
    const bool a = h != nullptr && *acc != 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (a) h[t] = hprop[t];
        if (p) p[t] = pprop[t];
    }
}

__global__ void k_prep_mixed(const double* __restrict__ y, const double* __restrict__ lnrv,
                             float* __restrict__ a_f, float* __restrict__ b0_f,
                             float2* __restrict__ lr_f, int64_t T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double a = 0.5 * y[t] * y[t];
        a_f[t] = (float)a;
        b0_f[t] = a > 0.0 ? (float)log2(a) : -INFINITY;
        const ff l = ff_from_double(lnrv[t]);
        lr_f[t] = make_float2(l.hi, l.lo);
    }
}

__global__ void k_h_to_ff(const double* __restrict__ h, float2* __restrict__ hf, int64_t T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const ff v = ff_from_double(h[t]);
        hf[t] = make_float2(v.hi, v.lo);
    }
}

__global__ void k_ff_to_h(const float2* __restrict__ hf, double* __restrict__ h,
                          const int* __restrict__ acc, int64_t T)
{
    if (acc && *acc == 0) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = hf[t];
        h[t] = (double)v.x + (double)v.y;
    }
}

__global__ void k_ff_to_h_sel(const float2* __restrict__ b0, const float2* __restrict__ b1,
                              const int* __restrict__ cur, double* __restrict__ h, int64_t T)
{
    const float2* src = *cur ? b1 : b0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[t];
        h[t] = (double)v.x + (double)v.y;
    }
}

__global__ void k_d_sel(const double* __restrict__ b0, const double* __restrict__ b1,
                        const int* __restrict__ cur, double* __restrict__ h, int64_t T)
{
    if (*cur == 0 && b0 == h) return;
    const double* src = *cur ? b1 : b0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x)
        h[t] = src[t];
}

__global__ void k_snapshot(const double* __restrict__ b0, const double* __restrict__ b1,
                           const float2* __restrict__ f0, const float2* __restrict__ f1,
                           const int* __restrict__ cur, float* __restrict__ out, int64_t T)
{
    const int c = *cur;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (f0) {
            const float2 v = (c ? f1 : f0)[t];
            out[t] = v.x + v.y;
        } else {
            out[t] = (float)(c ? b1 : b0)[t];
        }
    }
}

int grid_for(int64_t T)
{
    int64_t g = (T + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// Per-block shared memory of the trajectory kernels.
size_t smem_bytes(bool mixed, bool mass, int nt, int j)
{
    const size_t W = (size_t)nt * (size_t)j, nw = (size_t)nt / 32;
    if (mixed) return 32 * sizeof(double) + 4 * 32 * sizeof(float2) + 4 * W * sizeof(float);
    return (2 + (mass ? 1 : 0)) * W * sizeof(double) + 4 * nw * sizeof(double) + nw * sizeof(double);
}

template <int J, bool MASS>
cudaError_t launch_fp64(const TrajArgs& a, const TileCfg& c, cudaStream_t st)
{
    auto k = k_traj_fp64<J, MASS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem);
    if (e != cudaSuccess) return e;
    k<<<c.grid, c.nt, c.smem, st>>>(a);
    return cudaGetLastError();
}
template <int J, bool MASS>
cudaError_t launch_mixed(const TrajArgs& a, const TileCfg& c, cudaStream_t st)
{
    auto k = k_traj_mixed<J, MASS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem);
    if (e != cudaSuccess) return e;
    k<<<c.grid, c.nt, c.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Sites-per-thread values compiled for each path.
static const int kJ_fp64[] = {4, 8, 16, 28};
static const int kJ_mixed[] = {4, 8, 16, 20};

TileCfg plan_tiles(int64_t T, int n_md, bool mixed, bool mass, int num_sms)
{
    const int64_t K = (int64_t)n_md + 1;
    const int ntmax = mixed ? 384 : 256;
    const size_t smem_cap = 227 * 1024;
    TileCfg best{0, 0, 0, 0, 0};
    double best_cost = 1e300;
    const int* js = mixed ? kJ_mixed : kJ_fp64;
    for (int ji = 0; ji < 4; ++ji) {
        const int j = js[ji];
        for (int nt = 32; nt <= ntmax; nt += 32) {
            const int64_t cap = (int64_t)nt * j;
            const int64_t tile = cap - 2 * K - 3;
            if (tile < 1) continue;
            const size_t sm = smem_bytes(mixed, mass, nt, j);
            if (sm > smem_cap) continue;
            // a single window covers short series completely
            int64_t t_eff = T <= cap ? T : tile;
            const int64_t grid = (T + t_eff - 1) / t_eff;
            if (grid > (int64_t)1 << 31) continue;
            // cost: waves of blocks (one block per SM) times the slots each computes
            const int64_t waves = (grid + num_sms - 1) / num_sms;
            double cost = (double)waves * (double)cap;
            // prefer fuller windows, then more threads
            cost *= 1.0 + 1e-3 * (double)(ntmax - nt) / ntmax;
            if (cost < best_cost) {
                best_cost = cost;
                best = TileCfg{nt, j, t_eff, (int)grid, sm};
            }
        }
    }
    return best;
}

TileCfg fixed_tiles(int64_t T, int n_md, bool mixed, bool mass, int nt, int j, int64_t tile)
{
    TileCfg bad{0, 0, 0, 0, 0};
    const int* js = mixed ? kJ_mixed : kJ_fp64;
    bool jok = false;
    for (int i = 0; i < 4; ++i) jok |= js[i] == j;
    if (!jok || nt < 32 || nt % 32 || nt > (mixed ? 384 : 256) || tile < 1) return bad;
    const int64_t cap = (int64_t)nt * j;
    if (tile + 2 * ((int64_t)n_md + 1) + 3 > cap) return bad;
    const size_t sm = smem_bytes(mixed, mass, nt, j);
    if (sm > 227 * 1024) return bad;
    const int64_t grid = (T + tile - 1) / tile;
    if (grid > ((int64_t)1 << 31) - 1) return bad;
    return TileCfg{nt, j, tile, (int)grid, sm};
}

cudaError_t launch_traj(const TrajArgs& a, const TileCfg& c, bool mixed, bool mass,
                        cudaStream_t st)
{
#define RSV_CASE(FN, JJ) \
    case JJ: return mass ? FN<JJ, true>(a, c, st) : FN<JJ, false>(a, c, st);
    if (mixed) {
        switch (c.j) {
            RSV_CASE(launch_mixed, 4)
            RSV_CASE(launch_mixed, 8)
            RSV_CASE(launch_mixed, 20)
            RSV_CASE(launch_mixed, 16)
            default: return cudaErrorInvalidValue;
        }
    }
    switch (c.j) {
        RSV_CASE(launch_fp64, 4)
        RSV_CASE(launch_fp64, 8)
        RSV_CASE(launch_fp64, 16)
        RSV_CASE(launch_fp64, 28)
        default: return cudaErrorInvalidValue;
    }
#undef RSV_CASE
}

cudaError_t launch_commit_fp64(double* h, const double* hprop, double* p, const double* pprop,
                               const int* acc, int64_t T, cudaStream_t st)
{
    k_commit_fp64<<<grid_for(T), 256, 0, st>>>(h, hprop, p, pprop, acc, T);
    return cudaGetLastError();
}
cudaError_t launch_prep_mixed(const double* y, const double* lnrv, float* a_f, float* b0_f,
                              float2* lr_f, int64_t T, cudaStream_t st)
{
    k_prep_mixed<<<grid_for(T), 256, 0, st>>>(y, lnrv, a_f, b0_f, lr_f, T);
    return cudaGetLastError();
}
cudaError_t launch_h_to_ff(const double* h, float2* hf, int64_t T, cudaStream_t st)
{
    k_h_to_ff<<<grid_for(T), 256, 0, st>>>(h, hf, T);
    return cudaGetLastError();
}
cudaError_t launch_ff_to_h(const float2* hf, double* h, const int* acc, int64_t T,
                           cudaStream_t st)
{
    k_ff_to_h<<<grid_for(T), 256, 0, st>>>(hf, h, acc, T);
    return cudaGetLastError();
}
cudaError_t launch_ff_to_h_sel(const float2* b0, const float2* b1, const int* cur, double* h,
                               int64_t T, cudaStream_t st)
{
    k_ff_to_h_sel<<<grid_for(T), 256, 0, st>>>(b0, b1, cur, h, T);
    return cudaGetLastError();
}
cudaError_t launch_d_sel(const double* b0, const double* b1, const int* cur, double* h,
                         int64_t T, cudaStream_t st)
{
    k_d_sel<<<grid_for(T), 256, 0, st>>>(b0, b1, cur, h, T);
    return cudaGetLastError();
}
cudaError_t launch_snapshot(const double* b0, const double* b1, const float2* f0,
                            const float2* f1, const int* cur, float* out, int64_t T,
                            cudaStream_t st)
{
    k_snapshot<<<grid_for(T), 256, 0, st>>>(b0, b1, f0, f1, cur, out, T);
    return cudaGetLastError();
}

}  // namespace rsv
