// rsv_traj.cu -- HMC trajectories of the RSV model for one or many series.
//
// Method (arXiv:1603.08114, Sec. 3): leapfrog eqs. (6)-(8) repeated n_md times,
// dH = H(p', h') - H(p, h), Metropolis test with probability min{1, e^{-dH}}.
//
// GB300 design.  The paper launches three kernels per leapfrog step from the
// host (Sec. 5).  Here a persistent block takes a bin of work and integrates a
// whole trajectory of it on chip: the bin's sites sit in registers (J
// consecutive sites per thread), neighbours are exchanged once per step by warp
// shuffles plus a small shared-memory edge buffer, and no block ever waits for
// another.  A bin holds either several whole series side by side, each on
// whole warps with its own theta (the batched case), or one tile of a series
// longer than a window: the tile's window is widened by K = n_md + 1 sites on
// each side, sites near a window edge go stale one site per step, and after
// n_md steps the owned sites (and the right neighbour dH needs) are exactly
// what an untiled integration gives.  A whole series takes its Metropolis
// decision inside the block and overwrites its state in place on accept; the
// tiles of a split series write a proposal, and the last tile to finish sums
// their partial sums in tile order, decides and flips the series' buffer.
// In the mixed path without leverage those partial sums are the kinetic
// difference and the end state's statistics (StateStats): the potential
// energy of both ends comes from statistics kept per series and buffer, so
// the start needs only the kinetic energy.
//
// State is kept in x = h - mu, so that
//   dS/dh = ie * AR + iu * x + (1/2 - c' iu) - a' e^{-x},
//   AR_t = e_{t-1} - phi e_t,  e_t = x_{t+1} - phi x_t  (e_{T-1} = 0,
//   e_{-1} = (1 - phi^2) x_0),  a' = y^2/2 e^{-mu},  c' = lnRV - xi - mu,
// the gradient of S written with the AR innovations e_t (equal to eq. (7)'s
// stencil (1+phi^2) x_t - phi (x_{t-1} + x_{t+1}) inside the series).  The
// FP64 kernel uses this innovation form; the mixed kernel the equivalent
// three-point form with ghost neighbours (see mixed_steps).
//
// LEV instantiations take the RSV model with leverage, corr(eps_t, eta_t) =
// rho (the RSV reference cited in Sec. 2): with eps_t = y_t e^{-h_t/2},
//   S holds d_t^2 / (2 s_eta^2 (1 - rho^2)),  d_t = e_t - rho s_eta eps_t,
//   dS/dh_t = ... + B [d_{t-1} + d_t (rho s_eta eps_t / 2 - phi)],
//   B = 1 / (s_eta^2 (1 - rho^2)),
// and the y-term (y^2/2) e^{-h} = eps^2 / 2; the stationary term of h_1 is
// unchanged.
#include <cmath>

#include "rsv_traj_dev.cuh"

namespace rsv {

namespace {

// ---------------------------------------------------------------------------
// FP64 path.  Dynamic shared memory (slot-major, index j*NT + tid):
// a'[W] (with leverage y e^{-mu/2} instead), kc[W], and 1/m [W] with a mass.
// ---------------------------------------------------------------------------
template <int J, bool MASS, bool LEV>
__global__ void __launch_bounds__(256, 1) k_traj_fp64(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_wseg[NWMAX], s_wacc[NWMAX], s_flag;
    __shared__ double s_wpart[NWMAX], s_red[32], s_edge[4 * NWMAX], s_split;
    __shared__ double s_e2[kExpTabN];  // 2^(j/64), the table of exp_tab
    const int NT = blockDim.x, W = NT * J, nw = NT >> 5, tid = threadIdx.x;
    if (tid < kExpTabN) s_e2[tid] = kExp2Tab[tid];  // read after load_bin's barriers
    double* s_a = reinterpret_cast<double*>(smem_raw);
    double* s_kc = s_a + W;
    double* s_mi = s_kc + W;
    const bool mass_on = MASS && (A.mass_on == nullptr || *A.mass_on != 0);

    for (int b = blockIdx.x; b < A.nbins; b += gridDim.x) {
        View v;
        load_bin(A, b, s_wseg, s_wacc, v);
        const int base = v.base * J;
        const int la = v.n - 1 - base;
        const bool edge_thread = (la >= 0 && la < J);
        const ThetaD th = v.th;
        const double phi = th.phi, mu = th.mu;
        const double ie = 1.0 / th.se2, iu = 1.0 / th.su2;
        const double emu = exp(-mu), emh = exp(-0.5 * mu);
        const double st0 = 1.0 - phi * phi;
        // leverage: rs = rho s_eta, B = 1/(s_eta^2 (1 - rho^2)); B e_{-1} is the
        // stationary row (1 - phi^2) x_0 / s_eta^2
        const double rho = LEV ? th.rho : 0.0;
        const double rs = rho * sqrt(th.se2), ib = LEV ? 1.0 / (th.se2 * (1.0 - rho * rho)) : ie;
        const double stB = LEV ? st0 * (1.0 - rho * rho) : st0;
        const int64_t off = v.si.off, wlo = v.g.wlo;
        double* hin = v.cur ? A.h1d : A.h0d;
        double* hout = v.g.split ? (v.cur ? A.h0d : A.h1d) : hin;

        double x[J], p[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = base + j;
            const int64_t s = off + wlo + i;
            const bool act = i < v.n;
            const double hv = act ? hin[s] : mu;
            const double yv = act ? A.y[s] : 0.0;
            const double lr = act ? A.lnrv[s] : th.xi + mu;
            x[j] = hv - mu;
            s_a[j * NT + tid] = LEV ? yv * emh : 0.5 * yv * yv * emu;
            s_kc[j * NT + tid] = 0.5 - ((lr - th.xi) - mu) * iu;
            if (MASS) s_mi[j * NT + tid] = (act && mass_on) ? (double)A.minv[s] : 1.0;
        }
        if (A.p_in) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int i = base + j;
                p[j] = i < v.n ? A.p_in[off + wlo + i] : 0.0;
            }
        } else {
#pragma unroll
            for (int q = 0; q < J / 4; ++q) {
                const int64_t s0 = wlo + base + 4 * q;
                const u64x4 r = philox_block(A.seed, (uint64_t)v.g.series, A.traj, STREAM_MOM,
                                             (uint64_t)(s0 >> 2));
                box_muller(u01_53(r.w[0]), u01_53(r.w[1]), p[4 * q + 0], p[4 * q + 1]);
                box_muller(u01_53(r.w[2]), u01_53(r.w[3]), p[4 * q + 2], p[4 * q + 3]);
            }
            if (MASS) {
#pragma unroll
                for (int j = 0; j < J; ++j) p[j] = p[j] / sqrt(s_mi[j * NT + tid]);
            }
        }
        __syncthreads();
        // leverage: y e^{-mu/2} of the left neighbour site (none at a window start)
        const double yL = (LEV && !v.first) ? s_a[(J - 1) * NT + tid - 1] : 0.0;

        // eps_j = y_j e^{-h_j/2} and d_j = e_j - rs eps_j of this thread's run
        // (leverage only)
        auto lev_terms = [&](const double (&xx)[J], double (&eps)[J], double (&e)[J]) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                eps[j] = s_a[j * NT + tid] * exp_tab(-0.5 * xx[j], s_e2);
                if (!(edge_thread && j == la)) e[j] = fma(-rs, eps[j], e[j]);
            }
        };

        // H restricted to this thread's owned sites (x coordinates; the
        // constant mu/2 per site cancels in dH).
        int par = 0;
        auto owned_energy = [&](double& acc) {
            double xL, xR, e[J], eps[J];
            exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
            par ^= 1;
            if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
            else innovations<J, double, false>(x, xR, phi, la, e);
            if (LEV) lev_terms(x, eps, e);
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int64_t s = wlo + base + j;
                if (v.sid >= 0 && s >= v.g.lo && s < v.g.hi) {
                    const double cp = (A.lnrv[off + s] - th.xi) - mu;
                    const double r = cp - x[j];
                    const double ey = LEV ? 0.5 * eps[j] * eps[j] : s_a[j * NT + tid] * exp_tab(-x[j], s_e2);
                    double val = 0.5 * x[j] + ey + 0.5 * iu * r * r + 0.5 * ib * e[j] * e[j];
                    if (s == 0) val += 0.5 * ie * st0 * x[j] * x[j];
                    const double mi = MASS ? s_mi[j * NT + tid] : 1.0;
                    val += 0.5 * mi * p[j] * p[j];
                    acc += val;
                }
            }
        };
        double E0 = 0.0, E1 = 0.0;
        owned_energy(E0);

        // Per step, drifts and kicks in the literal order of the scheme: the
        // leapfrog eqs. (6)-(8) (drift dtau/2, kick dtau, drift dtau/2) or a
        // minimum-norm integrator (Scheme: drift a_0 dtau, then {kick b_k
        // dtau; drift a_{k+1} dtau}).
        const double dt = A.dtau;
        const int nk = A.sch.nk;
        for (int k = 0; k < A.n_md; ++k) {
            for (int st = 0; st <= nk; ++st) {
                // eq. (6)/(8): h += c dtau p / m
                const double cd = A.sch.a[st] * dt;
#pragma unroll
                for (int j = 0; j < J; ++j)
                    x[j] = fma(MASS ? cd * s_mi[j * NT + tid] : cd, p[j], x[j]);
                if (st == nk) break;
                double xL, xR, e[J], eps[J];
                exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
                par ^= 1;
                if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
                else innovations<J, double, false>(x, xR, phi, la, e);
                // e_{-1}: left neighbour's innovation, or the stationary term at a window start
                double eprev = v.first ? stB * x[0] : fma(-phi, xL, x[0]);
                if (LEV) {
                    lev_terms(x, eps, e);
                    if (!v.first) eprev = fma(-rs, yL * exp_tab(-0.5 * xL, s_e2), eprev);
                }
                // eq. (7): p -= kick dS/dh
                const double kick = A.sch.b[st] * dt;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    double f = fma(iu, x[j], s_kc[j * NT + tid]);
                    if (LEV) {
                        // d_{j-1} + d_j (rs eps_j / 2 - phi), and eps^2 / 2
                        const double ar = fma(e[j], fma(0.5 * rs, eps[j], -phi), eprev);
                        f = fma(ib, ar, f);
                        f = fma(-0.5 * eps[j], eps[j], f);
                    } else {
                        const double ar = fma(-phi, e[j], eprev);
                        f = fma(ie, ar, f);
                        f = fma(-s_a[j * NT + tid], exp_tab(-x[j], s_e2), f);
                    }
                    eprev = e[j];
                    p[j] = fma(-kick, f, p[j]);
                }
            }
        }
        owned_energy(E1);

        const double part = warp_sum(E1 - E0);
        if ((tid & 31) == 0) s_wpart[tid >> 5] = part;
        __syncthreads();
        segment_decisions(A, v, s_wpart, s_wacc, &s_split);
        __syncthreads();
        const bool write_h = v.sid >= 0 && (v.g.split || s_wacc[v.g.warp0]);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int64_t s = wlo + base + j;
            if (v.sid >= 0 && s >= v.g.lo && s < v.g.hi) {
                if (write_h) hout[off + s] = x[j] + mu;
                if (A.p_out) A.p_out[off + s] = p[j];
            }
        }
        if (v.g.split) finish_split(A, v, s_split, s_red, &s_flag);
    }
}

// 2^(j/32), j = 0..31, as double-float pairs, written by the theta prep kernel
// (FP64, 32 lanes, once per call) and copied to shared memory by each block.
__device__ float2 g_exptab[32];

template <int J, bool MASS, bool LEV>
__global__ void __launch_bounds__(mixed_ntmax<J, MASS>(), 1) k_traj_mixed(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MixedSmem<LEV> S;
    if (threadIdx.x < 32) S.exptab[threadIdx.x] = g_exptab[threadIdx.x];
    for (int b = blockIdx.x; b < A.nbins; b += gridDim.x)
        traj_mixed_bin<J, MASS, LEV, false>(A, b, S, smem_raw, A.snap_prev);
}

// ---------------------------------------------------------------------------
// Element-wise kernels.
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
                             float* __restrict__ a_f, float2* __restrict__ lr_f, int64_t T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double a = 0.5 * y[t] * y[t];
        a_f[t] = copysignf((float)a, (float)y[t]);  // the sign of y for the leverage term
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

// Series of packed site t (binary search over the series offsets).
__device__ __forceinline__ int series_of(const SerInfo* ser, int n, int64_t t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ser[mid].off <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_finalize(const SerInfo* __restrict__ ser, int n, int64_t total,
                           const int* __restrict__ cur, const int* __restrict__ acc,
                           const double* __restrict__ h1d, const float2* __restrict__ h0f,
                           const float2* __restrict__ h1f, double* __restrict__ h)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = n > 1 ? series_of(ser, n, t) : 0;
        const int c = cur ? cur[s] : 0;
        if (h0f) {
            if (acc && acc[s] == 0) continue;
            const float2 v = (c ? h1f : h0f)[t];
            h[t] = (double)v.x + (double)v.y;
        } else if (c) {
            h[t] = h1d[t];
        }
    }
}

// The statistics (StateStats) of the state hf: one block per segment over its
// owned sites (a thread's sites in order, then a butterfly in each warp and
// the warps in order), written as kPartialWords double-floats per segment
// (sum lnRV, the statistics, sum lnRV^2); then one warp per series adds its
// tiles and files the record as buffer 0's.
constexpr int kStatsThreads = 512;
__global__ void __launch_bounds__(kStatsThreads) k_state_stats(
    const Seg* __restrict__ segs, const SerInfo* __restrict__ ser, const float2* __restrict__ hf,
    const float* __restrict__ a_f, const float2* __restrict__ lr_f,
    const MixedTheta* __restrict__ theta_f, double* __restrict__ scratch)
{
    __shared__ float2 s_tab[32];
    __shared__ float2 s_red[kStatsThreads / 32][kPartialWords];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 32) s_tab[tid] = g_exptab[tid];
    __syncthreads();
    const Seg g = segs[blockIdx.x];
    const SerInfo si = ser[g.series];
    const MixedTheta& mt = theta_f[g.series];
    StateStats st;
    stats_zero(st);
    ff sl = {0.f, 0.f}, sll = {0.f, 0.f};
    for (int64_t t = g.lo + tid; t < g.hi; t += kStatsThreads) {
        const int64_t s = si.off + t;
        const float2 hv = hf[s];
        ff x = two_sum(hv.x, -mt.mu.hi);  // x = h - mu as the trajectory kernel forms it
        x.lo += hv.y - mt.mu.lo;
        x = fast_two_sum(x.hi, x.lo);
        const bool has_next = t + 1 < si.T;
        ff xn = {0.f, 0.f};
        if (has_next) {
            const float2 hn = hf[s + 1];
            xn = two_sum(hn.x, -mt.mu.hi);
            xn.lo += hn.y - mt.mu.lo;
            xn = fast_two_sum(xn.hi, xn.lo);
        }
        const float2 lr = lr_f[s];
        stats_site(st, x, xn, has_next, ff{lr.x, lr.y}, fabsf(a_f[s]), mt, s_tab);
        ff_acc(sl, ff{lr.x, lr.y});
        ff_acc(sll, ff_mul(ff{lr.x, lr.y}, ff{lr.x, lr.y}));
        if (t == 0) st.x0 = x;
        if (t + 1 == si.T) st.xT = x;
    }
    // slot 0: sum lnRV; slots 1..7: the statistics; slot 8: sum lnRV^2
#pragma unroll
    for (int i = 0; i < kPartialWords; ++i) {
        const ff v = i == 0 ? sl : i <= kStatsFF ? stats_ff(st)[i - 1] : sll;
        const ff r = warp_sum_ff(ff_add(v, ff{0.f, 0.f}));
        if (lane == 0) s_red[warp][i] = make_float2(r.hi, r.lo);
    }
    __syncthreads();
    if (tid < kPartialWords) {
        ff r = {0.f, 0.f};
        for (int w = 0; w < kStatsThreads / 32; ++w)
            r = ff_add(r, ff{s_red[w][tid].x, s_red[w][tid].y});
        float2* out = reinterpret_cast<float2*>(scratch) + (int64_t)blockIdx.x * kPartialWords;
        out[tid] = make_float2(r.hi, r.lo);
    }
}
__global__ void k_stats_combine(const SerInfo* __restrict__ ser, int n,
                                const MixedTheta* __restrict__ theta_f,
                                const double* __restrict__ scratch, StatsRec* __restrict__ rstats)
{
    // one warp per series: lane l adds tiles l, l + 32, ... in order, then a
    // butterfly per value
    const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= n) return;
    const SerInfo si = ser[s];
    const float2* rec = reinterpret_cast<const float2*>(scratch);
    ff acc[kPartialWords];
#pragma unroll
    for (int k = 0; k < kPartialWords; ++k) acc[k] = ff{0.f, 0.f};
    for (int i = lane; i < si.nseg; i += 32) {
        const float2* w = rec + (int64_t)(si.seg0 + i) * kPartialWords;
        float2 v[kPartialWords];
#pragma unroll
        for (int k = 0; k < kPartialWords; ++k) v[k] = w[k];
#pragma unroll
        for (int k = 0; k < kPartialWords; ++k) acc[k] = ff_add(acc[k], ff{v[k].x, v[k].y});
    }
#pragma unroll
    for (int k = 0; k < kPartialWords; ++k) acc[k] = warp_sum_ff(acc[k]);
    if (lane == 0) {
        StatsRec r;
        r.sl = acc[0];
        r.sll = acc[1 + kStatsFF];
#pragma unroll
        for (int k = 0; k < kStatsFF; ++k) stats_ff(r.s)[k] = acc[1 + k];
        r.mu = theta_f[s].mu;
        r.ximu = theta_f[s].ximu;
        rstats[2 * (int64_t)s] = r;
    }
}

__global__ void k_snapshot(const SerInfo* __restrict__ ser, int n, int64_t total,
                           const int* __restrict__ cur, const double* __restrict__ h0d,
                           const double* __restrict__ h1d, const float2* __restrict__ h0f,
                           const float2* __restrict__ h1f, float* __restrict__ out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = n > 1 ? series_of(ser, n, t) : 0;
        const int c = cur ? cur[s] : 0;
        if (h0f) {
            const float2 v = (c ? h1f : h0f)[t];
            out[t] = v.x + v.y;
        } else {
            out[t] = (float)(c ? h1d : h0d)[t];
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

template <int J, bool MASS, bool LEV>
cudaError_t launch_fp64(const TrajArgs& a, const Plan& p, cudaStream_t st)
{
    auto k = k_traj_fp64<J, MASS, LEV>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    k<<<p.grid, p.nt, p.smem, st>>>(a);
    return cudaGetLastError();
}
template <int J, bool MASS, bool LEV>
cudaError_t launch_mixed(const TrajArgs& a, const Plan& p, cudaStream_t st)
{
    auto k = k_traj_mixed<J, MASS, LEV>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    k<<<p.grid, p.nt, p.smem, st>>>(a);
    return cudaGetLastError();
}

__global__ void k_theta_prep(const double* __restrict__ theta, ThetaD th_inline, int n,
                             double rho, MixedTheta* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const ff v = ff_from_double(exp2((double)threadIdx.x / 32.0));
        g_exptab[threadIdx.x] = make_float2(v.hi, v.lo);
    }
    if (i < n) {
        ThetaD th = theta ? load_theta(theta + 5 * (int64_t)i) : th_inline;
        th.rho = rho;
        // an FP32-valued theta (as the mixed theta update leaves it) gets the
        // update's own FP32 constants
        const float tf[5] = {(float)th.phi, (float)th.mu, (float)th.xi, (float)th.se2,
                             (float)th.su2};
        const bool f32 = rho == 0.0 && (double)tf[0] == th.phi && (double)tf[1] == th.mu &&
                         (double)tf[2] == th.xi && (double)tf[3] == th.se2 &&
                         (double)tf[4] == th.su2;
        out[i] = f32 ? mixed_theta_f(tf) : mixed_theta(th);
    }
}

}  // namespace

cudaError_t launch_theta_prep(const double* theta, ThetaD th_inline, int n, double rho,
                              MixedTheta* theta_f, cudaStream_t st)
{
    const int g = (n + 127) / 128;
    k_theta_prep<<<g < 1 ? 1 : g, 128, 0, st>>>(theta, th_inline, n, rho, theta_f);
    return cudaGetLastError();
}

int mixed_max_threads(int j, bool mass)
{
    switch (j) {
        case 4: return mass ? mixed_ntmax<4, true>() : mixed_ntmax<4, false>();
        case 8: return mixed_ntmax<8, false>();
        case 12: return mixed_ntmax<12, false>();
        case 16: return mixed_ntmax<16, false>();
        case 20: return mixed_ntmax<20, false>();
        default: return 0;
    }
}

int blocks_per_sm(bool mixed, bool mass, bool lev, int j, int nt, size_t smem)
{
    int n = 0;
    cudaError_t e = cudaSuccess;
#define RSV_OCC(KERN)                                                                     \
    do {                                                                                  \
        e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)smem);                                              \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, KERN, \
                                                                               nt, smem); \
    } while (0)
#define RSV_JM(JJ)                                                         \
    case JJ:                                                               \
        if (mass && lev) RSV_OCC((k_traj_mixed<JJ, true, true>));          \
        else if (mass) RSV_OCC((k_traj_mixed<JJ, true, false>));           \
        else if (lev) RSV_OCC((k_traj_mixed<JJ, false, true>));            \
        else RSV_OCC((k_traj_mixed<JJ, false, false>));                    \
        break;
#define RSV_JD(JJ)                                                         \
    case JJ:                                                               \
        if (mass && lev) RSV_OCC((k_traj_fp64<JJ, true, true>));           \
        else if (mass) RSV_OCC((k_traj_fp64<JJ, true, false>));            \
        else if (lev) RSV_OCC((k_traj_fp64<JJ, false, true>));             \
        else RSV_OCC((k_traj_fp64<JJ, false, false>));                     \
        break;
    if (mixed) {
        switch (j) { RSV_JM(4) RSV_JM(8) RSV_JM(12) RSV_JM(16) RSV_JM(20) default: return 0; }
    } else {
        switch (j) { RSV_JD(4) RSV_JD(8) RSV_JD(16) RSV_JD(28) default: return 0; }
    }
#undef RSV_JM
#undef RSV_JD
#undef RSV_OCC
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_traj(const TrajArgs& a, const Plan& p, cudaStream_t st)
{
#define RSV_CASE(FN, JJ)                                                        \
    case JJ:                                                                    \
        if (p.lev) return p.mass ? FN<JJ, true, true>(a, p, st) : FN<JJ, false, true>(a, p, st); \
        return p.mass ? FN<JJ, true, false>(a, p, st) : FN<JJ, false, false>(a, p, st);
    if (p.mixed) {
        switch (p.j) {
            RSV_CASE(launch_mixed, 4)
            RSV_CASE(launch_mixed, 8)
            RSV_CASE(launch_mixed, 12)
            RSV_CASE(launch_mixed, 16)
            RSV_CASE(launch_mixed, 20)
            default: return cudaErrorInvalidValue;
        }
    }
    switch (p.j) {
        RSV_CASE(launch_fp64, 4)
        RSV_CASE(launch_fp64, 8)
        RSV_CASE(launch_fp64, 16)
        RSV_CASE(launch_fp64, 28)
        default: return cudaErrorInvalidValue;
    }
#undef RSV_CASE
}

cudaError_t launch_state_stats(const Plan& p, const float2* hf, const float* a_f,
                               const float2* lr_f, const MixedTheta* theta_f, double* scratch,
                               StatsRec* rstats, cudaStream_t st)
{
    if (p.nsegs < 1 || p.nsegs > 0x7fffffff) return cudaErrorInvalidValue;
    k_state_stats<<<(unsigned)p.nsegs, kStatsThreads, 0, st>>>(p.d_segs, p.d_ser, hf, a_f, lr_f,
                                                               theta_f, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_stats_combine<<<(p.nseries + 7) / 8, 256, 0, st>>>(p.d_ser, p.nseries, theta_f, scratch,
                                                        rstats);
    return cudaGetLastError();
}
cudaError_t launch_commit_fp64(double* h, const double* hprop, double* p, const double* pprop,
                               const int* acc, int64_t T, cudaStream_t st)
{
    k_commit_fp64<<<grid_for(T), 256, 0, st>>>(h, hprop, p, pprop, acc, T);
    return cudaGetLastError();
}
cudaError_t launch_prep_mixed(const double* y, const double* lnrv, float* a_f, float2* lr_f,
                              int64_t T, cudaStream_t st)
{
    k_prep_mixed<<<grid_for(T), 256, 0, st>>>(y, lnrv, a_f, lr_f, T);
    return cudaGetLastError();
}
cudaError_t launch_h_to_ff(const double* h, float2* hf, int64_t T, cudaStream_t st)
{
    k_h_to_ff<<<grid_for(T), 256, 0, st>>>(h, hf, T);
    return cudaGetLastError();
}
cudaError_t launch_finalize(const Plan& p, const int* cur, const int* acc, const double* h1d,
                            const float2* h0f, const float2* h1f, double* h, cudaStream_t st)
{
    k_finalize<<<grid_for(p.total), 256, 0, st>>>(p.d_ser, p.nseries, p.total, cur, acc, h1d,
                                                   h0f, h1f, h);
    return cudaGetLastError();
}
cudaError_t launch_snapshot(const Plan& p, const int* cur, const double* h0d, const double* h1d,
                            const float2* h0f, const float2* h1f, float* out, cudaStream_t st)
{
    k_snapshot<<<grid_for(p.total), 256, 0, st>>>(p.d_ser, p.nseries, p.total, cur, h0d, h1d,
                                                   h0f, h1f, out);
    return cudaGetLastError();
}

}  // namespace rsv
