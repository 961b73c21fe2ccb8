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
// their partial dH in tile order, decides and flips the series' buffer.
//
// State is kept in x = h - mu, so that
//   dS/dh = ie * AR + iu * x + (1/2 - c' iu) - a' e^{-x},
//   AR_t = e_{t-1} - phi e_t,  e_t = x_{t+1} - phi x_t  (e_{T-1} = 0,
//   e_{-1} = (1 - phi^2) x_0),  a' = y^2/2 e^{-mu},  c' = lnRV - xi - mu,
// the gradient of S written with the AR innovations e_t (equal to eq. (7)'s
// stencil (1+phi^2) x_t - phi (x_{t-1} + x_{t+1}) inside the series).
#include <cmath>

#include "rsv_device.cuh"
#include "rsv_traj.cuh"

namespace rsv {

namespace {

constexpr int NWMAX = 16;  // warps per block at most
constexpr float kLog2e = 1.4426950408889634f;

// 2^x on the special-function unit (ex2.approx.ftz.f32, relative error about
// 2^-22; 2^-inf = +0).
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// left_last = last value of thread tid-1, right_first = first value of thread
// tid+1 (garbage across a segment boundary; callers never use it there).
// `edge` is one of two alternating buffers of 2*nw values.
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

// Innovations e_j = x_{j+1} - phi x_j of one thread's run (xR = first x of the
// next thread), with e = 0 at the segment's last active slot `la`.
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

// Per-thread view of the bin being processed.
struct View {
    int sid;     // segment id, -1 for an idle warp
    Seg g;
    SerInfo si;
    ThetaD th;
    int base;    // thread index inside the segment (slot run = base*J .. base*J+J-1)
    int n;       // active sites of the window
    bool first;  // first thread of the segment
    int cur;     // buffer holding the series' current state
};

__device__ __forceinline__ void load_bin(const TrajArgs& A, int b, int* s_wseg, int* s_wacc,
                                         View& v)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (tid < NWMAX) {
        s_wseg[tid] = -1;
        s_wacc[tid] = 0;
    }
    __syncthreads();
    const int f0 = A.bin_first[b], f1 = A.bin_first[b + 1];
    for (int i = f0 + tid; i < f1; i += blockDim.x) {
        const int id = A.bin_seg[i];
        const Seg g = A.segs[id];
        for (int w = g.warp0; w < g.warp0 + g.nwarp && w < NWMAX; ++w) s_wseg[w] = id;
    }
    __syncthreads();
    v.sid = s_wseg[warp];
    if (v.sid >= 0) {
        v.g = A.segs[v.sid];
        v.si = A.ser[v.g.series];
        v.th = A.theta ? load_theta(A.theta + 5 * (int64_t)v.g.series) : A.th_inline;
        v.cur = A.ser_cur ? *(volatile int*)(A.ser_cur + v.g.series) : 0;
    } else {
        // idle warp: an empty segment with harmless parameters
        v.g = Seg{0, 0, 0, 0, 0, warp, 1, 0};
        v.si = SerInfo{0, 1, 1, 0};
        v.th = ThetaD{0.5, 0.0, 0.0, 1.0, 1.0};
        v.cur = 0;
    }
    const int ts = (warp - v.g.warp0) * 32 + lane;  // thread index inside the segment
    v.n = (int)(v.g.whi - v.g.wlo);
    v.base = ts;  // the caller scales it by J
    v.first = (ts == 0);
}

// Metropolis decision of one series (Sec. 3): accept iff ln u < -dH; a
// non-finite dH rejects and raises ST_NONFINITE.
__device__ int decide(const TrajArgs& A, int series, double dH, int cur, bool flip)
{
    double lu;
    if (A.log_u) {
        lu = A.log_u[series];
    } else {
        const u64x4 w = philox_block(A.seed, (uint64_t)series, A.traj, STREAM_MH, 0);
        lu = log(u01_53(w.w[0]));
    }
    const bool fin = isfinite(dH);
    const int acc = (fin && lu < -dH) ? 1 : 0;
    if (!fin) atomicOr(A.status, ST_NONFINITE);
    if (A.dH_out) A.dH_out[series] = dH;
    if (A.acc_out) A.acc_out[series] = acc;
    if (flip && acc && A.ser_cur) *(volatile int*)(A.ser_cur + series) = cur ^ 1;
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
    return acc;
}

// The last tile of a split series to arrive sums the partials of all its
// tiles in tile order and decides.  Called by the whole block.
__device__ void finish_split(const TrajArgs& A, const View& v, double part, double* red,
                             int* s_flag)
{
    if (threadIdx.x == 0) {
        A.partials[v.sid] = part;
        __threadfence();
        const unsigned prev = atomicAdd(A.ser_cnt + v.g.series, 1u);
        *s_flag = (prev == (unsigned)v.si.nseg - 1u);
    }
    __syncthreads();
    const int last = *s_flag;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < v.si.nseg; i += blockDim.x) s += __ldcg(A.partials + v.si.seg0 + i);
    const double dH = block_sum(s, red);
    if (threadIdx.x == 0) {
        A.ser_cnt[v.g.series] = 0u;
        decide(A, v.g.series, dH, v.cur, true);
        __threadfence();
    }
}

// Sum the per-warp parts of each segment (in warp order) and decide whole
// series; split bins return their part in *split_part.
__device__ __forceinline__ void segment_decisions(const TrajArgs& A, const View& v,
                                                  const double* s_wpart, int* s_wacc,
                                                  double* split_part)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (v.sid >= 0 && warp == v.g.warp0 && lane == 0) {
        double d = 0.0;
        for (int w = v.g.warp0; w < v.g.warp0 + v.g.nwarp; ++w) d += s_wpart[w];
        if (!v.g.split) s_wacc[v.g.warp0] = decide(A, v.g.series, d, v.cur, false);
        else *split_part = d;
    }
}

// ---------------------------------------------------------------------------
// FP64 path.  Dynamic shared memory (slot-major, index j*NT + tid):
// a'[W], kc[W], and 1/m [W] with a mass.
// ---------------------------------------------------------------------------
template <int J, bool MASS>
__global__ void __launch_bounds__(256, 1) k_traj_fp64(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_wseg[NWMAX], s_wacc[NWMAX], s_flag;
    __shared__ double s_wpart[NWMAX], s_red[32], s_edge[4 * NWMAX], s_split;
    const int NT = blockDim.x, W = NT * J, nw = NT >> 5, tid = threadIdx.x;
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
        const double emu = exp(-mu);
        const double st0 = 1.0 - phi * phi;
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
            s_a[j * NT + tid] = 0.5 * yv * yv * emu;
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

        // H restricted to this thread's owned sites (x coordinates; the
        // constant mu/2 per site cancels in dH).
        int par = 0;
        auto owned_energy = [&](double& acc) {
            double xL, xR, e[J];
            exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
            par ^= 1;
            if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
            else innovations<J, double, false>(x, xR, phi, la, e);
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int64_t s = wlo + base + j;
                if (v.sid >= 0 && s >= v.g.lo && s < v.g.hi) {
                    const double cp = (A.lnrv[off + s] - th.xi) - mu;
                    const double r = cp - x[j];
                    double val = 0.5 * x[j] + s_a[j * NT + tid] * exp(-x[j]) + 0.5 * iu * r * r +
                                 0.5 * ie * e[j] * e[j];
                    if (s == 0) val += 0.5 * ie * st0 * x[j] * x[j];
                    const double mi = MASS ? s_mi[j * NT + tid] : 1.0;
                    val += 0.5 * mi * p[j] * p[j];
                    acc += val;
                }
            }
        };
        double E0 = 0.0, E1 = 0.0;
        owned_energy(E0);

        const double dt = A.dtau, hd = 0.5 * A.dtau;
        for (int k = 0; k < A.n_md; ++k) {
            // eq. (6): h(tau + dtau/2) = h(tau) + dtau/2 p / m
#pragma unroll
            for (int j = 0; j < J; ++j) x[j] = fma(MASS ? hd * s_mi[j * NT + tid] : hd, p[j], x[j]);
            double xL, xR, e[J];
            exchange(x[0], x[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
            par ^= 1;
            if (edge_thread) innovations<J, double, true>(x, xR, phi, la, e);
            else innovations<J, double, false>(x, xR, phi, la, e);
            // e_{-1}: left neighbour's innovation, or the stationary term at a window start
            double eprev = v.first ? st0 * x[0] : fma(-phi, xL, x[0]);
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
            for (int j = 0; j < J; ++j) x[j] = fma(MASS ? hd * s_mi[j * NT + tid] : hd, p[j], x[j]);
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

// ---------------------------------------------------------------------------
// Mixed path: FP32 leapfrog on compensated (hi, lo) FP32 pairs for both the
// position and the momentum (a random walk of their FP32 roundings over n_md
// steps would otherwise dominate dH at 2^22 sites); dH from double-float
// per-site differences, accumulated in FP64 across threads.
// Dynamic shared memory (slot-major): x0 hi/lo and p0 [W each] (p0 enters
// every trajectory with lo = 0: drawn in FP32, or rounded from p_in).
// ---------------------------------------------------------------------------
template <int J, bool MASS>
__global__ void __launch_bounds__(384, 1) k_traj_mixed(const TrajArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_wseg[NWMAX], s_wacc[NWMAX], s_flag;
    __shared__ double s_wpart[NWMAX], s_red[32], s_edge_d[4 * NWMAX], s_split;
    __shared__ float2 s_exptab[32];
    const int NT = blockDim.x, W = NT * J, nw = NT >> 5, tid = threadIdx.x;
    float* s_edge = reinterpret_cast<float*>(s_edge_d);
    ff_exp_table(s_exptab);
    float* s_x0h = reinterpret_cast<float*>(smem_raw);
    float* s_x0l = s_x0h + W;
    float* s_p0h = s_x0l + W;
    const bool mass_on = MASS && (A.mass_on == nullptr || *A.mass_on != 0);
    const float dt = (float)A.dtau;

    for (int b = blockIdx.x; b < A.nbins; b += gridDim.x) {
        View v;
        load_bin(A, b, s_wseg, s_wacc, v);
        const int base = v.base * J;
        const int la = v.n - 1 - base;
        const bool edge_thread = (la >= 0 && la < J);
        const ThetaD th = v.th;
        const float phif = (float)th.phi;
        const float ief = (float)(1.0 / th.se2), iuf = (float)(1.0 / th.su2);
        const ff mu_ff = ff_from_double(th.mu);
        const ff ximu_ff = ff_from_double(th.xi + th.mu);
        const float cmu = (float)(-th.mu * 1.4426950408889634);  // exponent of e^{-mu}
        const int64_t off = v.si.off, wlo = v.g.wlo;
        float2* hin = v.cur ? A.h1f : A.h0f;
        float2* hout = v.g.split ? (v.cur ? A.h0f : A.h1f) : hin;

        float xh[J], xl[J], ph[J], pl[J], af[J], kf[J];
        float dtm[MASS ? J : 1];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = base + j;
            const int64_t s = off + wlo + i;
            const bool act = i < v.n;
            const float2 hv = act ? hin[s] : make_float2(mu_ff.hi, mu_ff.lo);
            ff x = two_sum(hv.x, -mu_ff.hi);  // x = h - mu in double-float
            x.lo += hv.y - mu_ff.lo;
            x = fast_two_sum(x.hi, x.lo);
            xh[j] = x.hi;
            xl[j] = x.lo;
            af[j] = act ? A.a_f[s] : 0.0f;  // y^2/2
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
                const double pv = i < v.n ? A.p_in[off + wlo + i] : 0.0;
                ph[j] = (float)pv;
            }
        } else {
#pragma unroll
            for (int q = 0; q < J / 4; ++q) {
                const int64_t s0 = wlo + base + 4 * q;
                const u64x4 r = philox_block(A.seed, (uint64_t)v.g.series, A.traj, STREAM_MOM,
                                             (uint64_t)(s0 >> 2));
                box_muller_f(u01_23(r.w[0]), u01_23(r.w[1]), ph[4 * q + 0], ph[4 * q + 1]);
                box_muller_f(u01_23(r.w[2]), u01_23(r.w[3]), ph[4 * q + 2], ph[4 * q + 3]);
            }
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (MASS) ph[j] = ph[j] / sqrtf(dtm[MASS ? j : 0]);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            pl[j] = 0.0f;
            s_x0h[j * NT + tid] = xh[j];
            s_x0l[j * NT + tid] = xl[j];
            s_p0h[j * NT + tid] = ph[j];
            if (MASS) dtm[MASS ? j : 0] *= dt;  // dtau / m_t
        }
        int par = 0;

        // Compensated v += c*u on a (hi, lo) pair: lo carries what hi lost.
        auto cupd = [](float& hi, float& lo, float c, float u) {
            const float y = fmaf(c, u, lo);
            const float t = hi + y;
            lo = y - (t - hi);
            hi = t;
        };

        // Leapfrog with the two half steps of consecutive steps merged:
        // x += dt/2 p;  n_md times { p -= dt F(x); x += (dt, or dt/2 at the end) p }.
#pragma unroll
        for (int j = 0; j < J; ++j)
            cupd(xh[j], xl[j], MASS ? 0.5f * dtm[MASS ? j : 0] : 0.5f * dt, ph[j]);
        for (int k = 0; k < A.n_md; ++k) {
            float xL, xR, e[J];
            exchange(xh[0], xh[J - 1], xL, xR, s_edge + par * 2 * nw, nw);
            par ^= 1;
            if (edge_thread) innovations<J, float, true>(xh, xR, phif, la, e);
            else innovations<J, float, false>(xh, xR, phif, la, e);
            float eprev = v.first ? (1.0f - phif * phif) * xh[0] : fmaf(-phif, xL, xh[0]);
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const float ar = fmaf(-phif, e[j], eprev);
                eprev = e[j];
                float f = fmaf(iuf, xh[j], kf[j]);
                f = fmaf(ief, ar, f);
                // (y^2/2) e^{-h} = a 2^{-(x + mu) log2 e}: a small exponent argument
                f = fmaf(-af[j], ex2_approx(fmaf(-kLog2e, xh[j], cmu)), f);
                cupd(ph[j], pl[j], -dt, f);
            }
            const float hs = (k + 1 < A.n_md) ? 1.0f : 0.5f;
#pragma unroll
            for (int j = 0; j < J; ++j)
                cupd(xh[j], xl[j], MASS ? hs * dtm[MASS ? j : 0] : hs * dt, ph[j]);
        }

        // ---- dH from per-site differences in double-float ------------------
        // K = sum (p'^2 - p^2)/m, L = sum (x' - x), R = sum (x'-c')^2 - (x-c')^2,
        // Q = sum e'^2 - e^2, E = sum a (e^{-h'} - e^{-h});
        // dH = K/2 + L/2 + R/(2 s_u^2) + Q/(2 s_eta^2) + E + stationary term.
        ff accK = {0.f, 0.f}, accL = {0.f, 0.f}, accR = {0.f, 0.f}, accQ = {0.f, 0.f},
           accE = {0.f, 0.f};
        double stat = 0.0;
        const ff phi_ff = ff_from_double(th.phi);
        {
            float xLh, xRh, xLl, xRl;
            exchange(xh[0], xh[J - 1], xLh, xRh, s_edge + par * 2 * nw, nw);
            par ^= 1;
            exchange(xl[0], xl[J - 1], xLl, xRl, s_edge + par * 2 * nw, nw);
            par ^= 1;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int64_t s = wlo + base + j;
                if (v.sid < 0 || s < v.g.lo || s >= v.g.hi) continue;
                const ff x1 = {xh[j], xl[j]};
                const ff x0 = {s_x0h[j * NT + tid], s_x0l[j * NT + tid]};
                const ff d = ff_sub(x1, x0);
                ff_acc(accL, d);
                const float p0h = s_p0h[j * NT + tid];
                ff q1 = two_prod(ph[j], ph[j]);  // p'^2 = (hi + lo)^2 to ~2^-48
                q1.lo = fmaf(2.0f * ph[j], pl[j], q1.lo);
                ff dk = ff_sub(q1, two_prod(p0h, p0h));
                if (MASS) dk = ff_mul_f(dk, dtm[MASS ? j : 0] / dt);
                ff_acc(accK, dk);
                const float2 lr = A.lr_f[off + s];
                ff cp = two_sum(lr.x, -ximu_ff.hi);
                cp.lo += lr.y - ximu_ff.lo;
                ff sgm = ff_add(x1, x0);
                sgm = ff_sub(sgm, ff{2.0f * cp.hi, 2.0f * cp.lo});
                ff_acc(accR, ff_mul(d, sgm));
                if (s + 1 < v.si.T) {
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
                // a (e^{-h'} - e^{-h}) with both exponentials in double-float
                const ff E1 = ff_exp(ff_sub(ff{-mu_ff.hi, -mu_ff.lo}, x1), s_exptab);
                const ff E0 = ff_exp(ff_sub(ff{-mu_ff.hi, -mu_ff.lo}, x0), s_exptab);
                ff_acc(accE, ff_mul_f(ff_sub(E1, E0), af[j]));
            }
        }
        ff tot = ff_add(ff_add(ff_mul_f(accK, 0.5f), ff_mul_f(accL, 0.5f)), accE);
        tot = ff_add(tot, ff_mul(accR, ff_from_double(0.5 / th.su2)));
        tot = ff_add(tot, ff_mul(accQ, ff_from_double(0.5 / th.se2)));
        tot = warp_sum_ff(tot);
        double mine = (tid & 31) == 0 ? ff_to_double(tot) : 0.0;
        mine = warp_sum(mine + stat);
        if ((tid & 31) == 0) s_wpart[tid >> 5] = mine;
        __syncthreads();
        segment_decisions(A, v, s_wpart, s_wacc, &s_split);
        __syncthreads();
        const bool write_h = v.sid >= 0 && (v.g.split || s_wacc[v.g.warp0]);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int64_t s = wlo + base + j;
            if (v.sid >= 0 && s >= v.g.lo && s < v.g.hi) {
                if (write_h) {
                    ff hh = two_sum(xh[j], mu_ff.hi);
                    hh.lo += xl[j] + mu_ff.lo;
                    hh = fast_two_sum(hh.hi, hh.lo);
                    hout[off + s] = make_float2(hh.hi, hh.lo);
                }
                if (A.p_out) A.p_out[off + s] = (double)ph[j] + (double)pl[j];
            }
        }
        if (v.g.split) finish_split(A, v, s_split, s_red, &s_flag);
    }
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
        a_f[t] = (float)a;
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

template <int J, bool MASS>
cudaError_t launch_fp64(const TrajArgs& a, const Plan& p, cudaStream_t st)
{
    auto k = k_traj_fp64<J, MASS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    k<<<p.grid, p.nt, p.smem, st>>>(a);
    return cudaGetLastError();
}
template <int J, bool MASS>
cudaError_t launch_mixed(const TrajArgs& a, const Plan& p, cudaStream_t st)
{
    auto k = k_traj_mixed<J, MASS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    k<<<p.grid, p.nt, p.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int blocks_per_sm(bool mixed, bool mass, int j, int nt, size_t smem)
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
        if (mass) RSV_OCC((k_traj_mixed<JJ, true>));                       \
        else RSV_OCC((k_traj_mixed<JJ, false>));                           \
        break;
#define RSV_JD(JJ)                                                         \
    case JJ:                                                               \
        if (mass) RSV_OCC((k_traj_fp64<JJ, true>));                        \
        else RSV_OCC((k_traj_fp64<JJ, false>));                            \
        break;
    if (mixed) {
        switch (j) { RSV_JM(4) RSV_JM(8) RSV_JM(16) RSV_JM(20) default: return 0; }
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
#define RSV_CASE(FN, JJ) \
    case JJ: return p.mass ? FN<JJ, true>(a, p, st) : FN<JJ, false>(a, p, st);
    if (p.mixed) {
        switch (p.j) {
            RSV_CASE(launch_mixed, 4)
            RSV_CASE(launch_mixed, 8)
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
