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

#include "rsv_device.cuh"
#include "rsv_traj.cuh"

namespace rsv {

namespace {

constexpr int NWMAX = 32;  // warps per block at most
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
// Branch-free: every lane loads the two neighbouring warps' edge values (one
// address per warp and load, a broadcast) and selects.
template <typename V>
__device__ __forceinline__ void exchange(V first, V last, V& left_last, V& right_first, V* edge,
                                         int nw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V up = __shfl_up_sync(0xffffffffu, last, 1);
    const V dn = __shfl_down_sync(0xffffffffu, first, 1);
    if (lane == 0) edge[2 * warp] = first;
    if (lane == 31) edge[2 * warp + 1] = last;
    __syncthreads();
    const bool has_l = warp > 0, has_r = warp + 1 < nw;
    const V el = edge[2 * (has_l ? warp - 1 : warp) + 1];
    const V er = edge[2 * (has_r ? warp + 1 : warp)];
    left_last = lane == 0 ? (has_l ? el : first) : up;
    right_first = lane == 31 ? (has_r ? er : last) : dn;
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

// This warp's view, from the segment ids already placed in s_wseg (no
// barrier; a kernel may call it again after its step loop instead of keeping
// the view in registers through the loop).
__device__ __forceinline__ void view_of(const TrajArgs& A, const int* s_wseg, View& v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v.sid = s_wseg[warp];
    if (v.sid >= 0) {
        v.g = A.segs[v.sid];
        v.si = A.ser[v.g.series];
        v.th = A.theta ? load_theta(A.theta + 5 * (int64_t)v.g.series) : A.th_inline;
        v.th.rho = A.rho;
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

__device__ __forceinline__ void load_bin(const TrajArgs& A, int b, int* s_wseg, int* s_wacc,
                                         View& v)
{
    const int tid = threadIdx.x;
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
    view_of(A, s_wseg, v);
}

// Metropolis decision of one series (Sec. 3): accept iff ln u < -dH; a
// non-finite dH rejects and raises ST_NONFINITE.
// ln u of a drawn u is taken first in FP32 (logf of u rounded to FP32: off by
// at most 2^-24 + a few ulp of ln u, |ln u| < 37); only when that lies within
// 1e-6 (1 + |ln u|) of -dH, where the comparison could go either way, is it
// taken in FP64, so the decision is the FP64 comparison's at the cost of one
// FP64 logarithm in about a million trajectories.
__device__ int decide(const TrajArgs& A, int series, double dH, int cur, bool flip)
{
    const bool fin = isfinite(dH);
    int acc;
    if (A.log_u) {
        acc = (fin && A.log_u[series] < -dH) ? 1 : 0;
    } else {
        const u64x4 w = philox_block(A.seed, (uint64_t)series, A.traj, STREAM_MH, 0);
        const double u = u01_53(w.w[0]);
        const float lf = logf((float)u);
        const double gap = (double)lf + dH;  // ln u - (-dH), to within the margin
        if (!fin) acc = 0;
        else if (fabs(gap) > 1e-6 * (1.0 + fabs((double)lf))) acc = gap < 0.0 ? 1 : 0;
        else acc = log(u) < -dH ? 1 : 0;
    }
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

// The same two steps with the partial dH as double-float (mixed path): sums
// in FP32 arithmetic by one warp, one FP64 conversion for the decision.
__device__ void finish_split_ff(const TrajArgs& A, const View& v, float2 part, int* s_flag)
{
    float2* pf = reinterpret_cast<float2*>(A.partials);
    if (threadIdx.x == 0) {
        pf[v.sid] = part;
        __threadfence();
        const unsigned prev = atomicAdd(A.ser_cnt + v.g.series, 1u);
        *s_flag = (prev == (unsigned)v.si.nseg - 1u);
    }
    __syncthreads();
    const int last = *s_flag;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // lane l sums partials l, l + 32, ... in that order; the loads of eight
    // of them are issued together (one L2 round trip, not eight)
    ff s = {0.f, 0.f};
    for (int i0 = threadIdx.x; i0 < v.si.nseg; i0 += 32 * 8) {
        float2 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            w[u] = i0 + 32 * u < v.si.nseg ? __ldcg(pf + v.si.seg0 + i0 + 32 * u)
                                           : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + 32 * u < v.si.nseg) s = ff_add(s, ff{w[u].x, w[u].y});
    }
    s = warp_sum_ff(s);
    if (threadIdx.x == 0) {
        A.ser_cnt[v.g.series] = 0u;
        decide(A, v.g.series, ff_to_double(s), v.cur, true);
        __threadfence();
    }
}
__device__ __forceinline__ void segment_decisions_ff(const TrajArgs& A, const View& v,
                                                     const float2* s_wpf, int* s_wacc,
                                                     float2* split_part)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (v.sid >= 0 && warp == v.g.warp0 && lane == 0) {
        ff d = {0.f, 0.f};
        for (int w = v.g.warp0; w < v.g.warp0 + v.g.nwarp; ++w) d = ff_add(d, ff{s_wpf[w].x, s_wpf[w].y});
        if (!v.g.split) s_wacc[v.g.warp0] = decide(A, v.g.series, ff_to_double(d), v.cur, false);
        else *split_part = make_float2(d.hi, d.lo);
    }
}

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
                eps[j] = s_a[j * NT + tid] * exp(-0.5 * xx[j]);
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
                    const double ey = LEV ? 0.5 * eps[j] * eps[j] : s_a[j * NT + tid] * exp(-x[j]);
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
                    if (!v.first) eprev = fma(-rs, yL * exp(-0.5 * xL), eprev);
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
                        f = fma(-s_a[j * NT + tid], exp(-x[j]), f);
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

// ---------------------------------------------------------------------------
// Mixed path: FP32 leapfrog on compensated (hi, lo) FP32 pairs for both the
// position and the momentum (a random walk of their FP32 roundings over n_md
// steps would otherwise dominate dH at 2^22 sites); dH as the difference of
// the energies at both ends, each summed per thread in double-float, then
// across warps and tiles in double-float, with one FP64 conversion for the
// Metropolis test.
//
// Registers hold only the evolving state (x and p as (hi, lo), 4 J floats), so
// that a block can run up to 32 warps; the per-site constants of the force sit
// in shared memory and are read as float4.  Dynamic shared memory (slot-major:
// slot j of thread tid at [j][tid]; pairs (p, p + P), P = J/2):
//   s_ak  float4 [P][NT]  (-a_p, -a_{p+P}, k_p, k_{p+P}): a = y^2/2,
//                         k = 1/2 - c'/s_u^2
//   s_dm  float2 [P][NT]  -kick/m of the pair (with a mass only; the state
//                         then holds the velocity v = p/m)
//   s_v   float2 [P][NT]  the leverage weights v of the pair (leverage only)
//   s_xh, s_xl, s_ph  float [J][NS]  x (hi, lo) and p hi at the start of the
//                         trajectory and again at its end (p lo then over k);
//                         rows NS = mixed_row(NT, J) slots apart
// The arrays the leapfrog reads every step keep rows of NT slots: a warp's
// float4 (float2) row segment is then four (two) whole 128-byte lines; the
// rows of the start and end state, which only the load and write passes and
// the energies touch, are padded against bank conflicts instead.
// ---------------------------------------------------------------------------
// (with a mass and J = 4 at most 768 threads: its load pass needs more than
// the 64 registers a 1024-thread block leaves)
template <int J, bool MASS>
constexpr int mixed_ntmax()
{
    return J <= 4 ? (MASS ? 768 : 1024) : J <= 8 ? 768 : J <= 12 ? 640 : J <= 16 ? 512 : 384;
}

// 2^(j/32), j = 0..31, as double-float pairs, written by the theta prep kernel
// (FP64, 32 lanes, once per call) and copied to shared memory by each block.
__device__ float2 g_exptab[32];

// Per-block constants of the leapfrog of one segment.
struct MixedConst {
    float phi, c0, c1, cmu, dt;
    // integrator as substeps {kick; drift} (MixedScheme): kick sizes kq (a
    // mass's -kick/m holds kick = kq[0], scaled by kr), drift ratios (to
    // dtau) r, the last substep's r_last; nk substeps per step, n_sub in all
    float kick, kq[4], kr[4], r[4], r_last;
    int nk, n_sub;
    int la;        // slot of the series' last site in this thread (or out of [0, J))
    bool first;    // this thread holds the series' first site in slot 0
    // leverage: v of the left neighbour site (0 at a window start), and the
    // first-site correction cst (0 on other threads)
    float vL, cfirst;
};

// Packed FP32 pair arithmetic (FFMA2/FADD2: two independent FP32 lanes per
// instruction, each rounded exactly as its scalar counterpart).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a + (-1) b: one rounding, the same value as a scalar subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }

// Compensated v += c*u on (hi, lo) pairs (lo carries what hi lost), lane by lane.
__device__ __forceinline__ void cupd2(float2& hi, float2& lo, float2 c, float2 u)
{
    const float2 y = fma2(c, u, lo);
    const float2 t = add2(hi, y);
    lo = sub2(y, sub2(t, hi));
    hi = t;
}

// n_md leapfrog steps (eqs. (6)-(8)) with the two half steps of consecutive
// steps merged: x += dt/2 p;  n_md times { p -= dt F(x); x += (dt, or dt/2 at
// the end) p }.  The force of eq. (7) is taken in its three-point form
//   F_t = c0 x_t + c1 (x_{t-1} + x_{t+1}) + k_t - a_t e^{-h_t},
//   c0 = 1/s_u^2 + (1+phi^2)/s_eta^2,  c1 = -phi/s_eta^2,
// with a ghost neighbour phi x_t beyond either end of a series, which gives
// the end rows (x_0 - phi x_1)/s_eta^2, (x_{T-1} - phi x_{T-2})/s_eta^2 and,
// for T = 1, (1 - phi^2) x_0/s_eta^2.
// A thread's run of J sites is held as P = J/2 pairs (j, j + P): the two
// halves of the run advance side by side in the two lanes of packed FP32
// instructions.  Site by site the force and both updates are fused; the left
// neighbour's value from before the step is carried, the upper half's last
// site takes x_P from before the step.
// EDGE: some thread of the warp ends a series before its last slot; the ghost
// replaces the right neighbour there by a select.
// s_ak: float4 [P][NT] = (-a_p, -a_{p+P}, k_p, k_{p+P}); s_dm: float2 [P][NT]
// of -kick/m: with a diagonal mass the state carries the velocity v = p/m, so
// that the drift x += c dtau v is the same for every site and the mass enters
// the kick v -= kick F/m alone.
//
// LEV (leverage): with B in c0 and c1, the force gains
//   w_t (phi + (x_{t+1} - phi x_t)/2) - w_{t-1},  w_t = v_t e^{-h_t/2},
//   v_t = B rho s_eta y_t (0 at the series' last site, which has no d_t),
// the y-term weight a/(1-rho^2) at sites with a successor (the eps^2 part of
// d_t^2), and cst x_0 at the series' first site, where the stationary row
// (1-phi^2) x_0/s_eta^2 differs from the ghost's B (1-phi^2) x_0.
// e^{-h} is taken as (e^{-h/2})^2 from one ex2.  s_v: float2 [P][NT] of v.
template <int J, bool MASS, bool EDGE, bool LEV, bool KV>
__device__ __forceinline__ void mixed_steps(float2 (&X)[J / 2], float2 (&XL)[J / 2],
                                            float2 (&PH)[J / 2], float2 (&PL)[J / 2],
                                            const float4* __restrict__ s_ak,
                                            const float2* __restrict__ s_dm,
                                            const float2* __restrict__ s_v, float* s_edge,
                                            int& par, int nw, int n_md, const MixedConst& c)
{
    constexpr int P = J / 2;
    const int NT = blockDim.x, tid = threadIdx.x;
    const float2 c0 = f2(c.c0, c.c0), c1 = f2(c.c1, c.c1);
    const float2 nl2e = f2(-kLog2e, -kLog2e), cmu = f2(c.cmu, c.cmu);
    const float2 nl2h = f2(-0.5f * kLog2e, -0.5f * kLog2e), cmh = f2(0.5f * c.cmu, 0.5f * c.cmu);
    const float2 half = f2(0.5f, 0.5f), phi2 = f2(c.phi, c.phi), nphi2 = f2(-c.phi, -c.phi);
    const float2 zero = f2(0.0f, 0.0f);
    const float2 ndt = f2(-c.kick, -c.kick);
    // KV (kick sizes vary within a step): this substep's -kick, or with a
    // mass the ratio of its kick to the one -kick/m in s_dm holds
    float2 kc = MASS ? f2(1.0f, 1.0f) : ndt;
    // The edge exchange overlaps the interior pairs 1..P-2, which need no
    // neighbour from another thread: the edges are published (warp shuffles,
    // the warps' end values to shared memory), the interior pairs advance, and
    // only then the block barrier and pairs 0 and P-1.  Per site the same
    // operations in the same order as a pass in pair order.
    const int lane = tid & 31, warp = tid >> 5;
    // e^{-h/2} of a pair (leverage)
    auto e2_of = [&](float2 xq) -> float2 {
        const float2 t = fma2(nl2h, xq, cmh);
        return f2(ex2_approx(t.x), ex2_approx(t.y));
    };
    // one pair: force of eq. (7) in three-point form, then the kick and the
    // drift, compensated.  LEV: e2 = e^{-h/2} of the pair, prevw = w of its
    // left neighbours; returns the pair's w.
    auto advance = [&](int q, float2 prev, float2 nxt, float2 cx, float hs, float2 e2,
                       float2 prevw) -> float2 {
        const float4 ak = s_ak[q * NT + tid];
        const float2 xq = X[q];
        if (EDGE) {
            if (q == c.la) nxt.x = c.phi * xq.x;
            if (q + P == c.la) nxt.y = c.phi * xq.y;
        }
        float2 f = fma2(c0, xq, f2(ak.z, ak.w));
        f = fma2(c1, add2(prev, nxt), f);
        float2 w = zero;
        if (LEV) {
            f = fma2(f2(ak.x, ak.y), fma2(e2, e2, zero), f);
            w = fma2(s_v[q * NT + tid], e2, zero);
            const float2 g = fma2(half, fma2(nphi2, xq, nxt), phi2);
            f = sub2(fma2(w, g, f), prevw);
            if (q == 0) f.x = fmaf(c.cfirst, xq.x, f.x);
        } else {
            // (y^2/2) e^{-h} = a 2^{-(x + mu) log2 e}: a small exponent argument
            const float2 t = fma2(nl2e, xq, cmu);
            f = fma2(f2(ak.x, ak.y), f2(ex2_approx(t.x), ex2_approx(t.y)), f);
        }
        // with a mass the state holds the velocity v = p/m: the kick takes
        // the per-site -kick/m, the drift is the same for every site
        const float2 km = MASS ? (KV ? fma2(s_dm[q * NT + tid], kc, zero) : s_dm[q * NT + tid])
                               : (KV ? kc : ndt);
        cupd2(PH[q], PL[q], km, f);
        cupd2(X[q], XL[q], cx, PH[q]);
        return w;
    };
    for (int k = 0; k < c.n_sub; ++k) {
        float* edge = s_edge + par * 2 * nw;
        par ^= 1;
        const float first = X[0].x, last = X[P - 1].y;
        const float up = __shfl_up_sync(0xffffffffu, last, 1);
        const float dn = __shfl_down_sync(0xffffffffu, first, 1);
        if (lane == 0) edge[2 * warp] = first;
        if (lane == 31) edge[2 * warp + 1] = last;
        const float xP = X[0].y;  // x_P before the step
        const float2 x1 = X[1];   // pair 1 before the step (pair 0's right neighbours)
        const int ks = k & (c.nk - 1);  // nk = 1, 2 or 4
        float rk;
        if (KV) {
            rk = ks == 0 ? c.r[0] : ks == 1 ? c.r[1] : ks == 2 ? c.r[2] : c.r[3];
            if (MASS) {
                const float kr = ks == 0 ? c.kr[0] : ks == 1 ? c.kr[1] : ks == 2 ? c.kr[2] : c.kr[3];
                kc = f2(kr, kr);
            } else {
                const float kq = ks == 0 ? c.kq[0] : ks == 1 ? c.kq[1] : ks == 2 ? c.kq[2] : c.kq[3];
                kc = f2(-kq, -kq);
            }
        } else {
            rk = ks ? c.r[1] : c.r[0];
        }
        const float hs = (k + 1 < c.n_sub) ? rk : c.r_last;
        const float2 cx = f2(hs * c.dt, hs * c.dt);
        // leverage: e^{-h/2} of pairs 0 and P-1 before the step, and w of pair 0
        float2 e2_0 = zero, e2_last = zero, prevw = zero;
        if (LEV) {
            e2_0 = e2_of(X[0]);
            e2_last = e2_of(X[P - 1]);
            prevw = fma2(s_v[tid], e2_0, zero);
        }
        float2 prev = X[0];  // left neighbours of pair 1, before the step
#pragma unroll
        for (int q = 1; q + 1 < P; ++q) {
            const float2 xq = X[q];
            const float2 w = advance(q, prev, X[q + 1], cx, hs, LEV ? e2_of(xq) : zero, prevw);
            prev = xq;
            prevw = w;
        }
        __syncthreads();
        const bool has_l = warp > 0, has_r = warp + 1 < nw;
        const float el = edge[2 * (has_l ? warp - 1 : warp) + 1];
        const float er = edge[2 * (has_r ? warp + 1 : warp)];
        float xL = lane == 0 ? (has_l ? el : first) : up;
        float xR = lane == 31 ? (has_r ? er : last) : dn;
        if (c.first) xL = c.phi * X[0].x;
        if (!EDGE && c.la == J - 1) xR = c.phi * X[P - 1].y;
        // pair 0 (X[P-1] is still the state before the step), then P-1
        float2 prevw0 = zero;
        if (LEV) {
            const float2 vP = s_v[(P - 1) * NT + tid];
            prevw0 = f2(c.vL * ex2_approx(fmaf(-0.5f * kLog2e, xL, 0.5f * c.cmu)),
                        vP.x * e2_last.x);
        }
        advance(0, f2(xL, X[P - 1].x), x1, cx, hs, e2_0, prevw0);
        advance(P - 1, prev, f2(xP, xR), cx, hs, e2_last, prevw);
    }
}

// Energy of one owned site in double-float, without the site-independent
// constants (mu/2 per site, which cancel in dH): the parts accumulate
// separately and are weighted once per thread,
//   H = K/2 + L/2 + R/(2 s_u^2) + Q/(2 s_eta^2) + E  (+ the stationary term),
//   K = p^2/m, L = x, R = (x - c')^2, Q = (x_{t+1} - phi x_t)^2 (t < T-1),
//   E = (y^2/2) e^{-h}.
struct HParts {
    ff K, L, R, Q, E;
};
__device__ __forceinline__ void hparts_zero(HParts& a)
{
    a.K = a.L = a.R = a.Q = a.E = ff{0.f, 0.f};
}
__device__ __forceinline__ ff hparts_total(const HParts& a, const MixedTheta& mt)
{
    ff tot = ff_add(ff_mul_f(a.K, 0.5f), ff_mul_f(a.L, 0.5f));
    tot = ff_add(tot, a.E);
    tot = ff_add(tot, ff_mul(a.R, mt.hu));
    return ff_add(tot, ff_mul(a.Q, mt.he));
}
// x: h - mu; p: momentum (hi, lo); mi: 1/m; cp: c' = lnRV - xi - mu; a: y^2/2;
// xn: next site's x (used only if has_next).
// LEV: Q is d_t^2 = (x_{t+1} - phi x_t - rs_y e^{-h_t/2})^2, rs_y = rho s_eta y_t
// (weighted by B/2 in he).
// With a mass, p is the velocity v = p/m and mw the double-float mass m, so
// that K = m v^2 (see mass_weight).
// K of one site: p^2, or m v^2 with a mass (p the velocity, mw the mass).
template <bool MASS>
__device__ __forceinline__ ff kinetic(ff p, ff mw)
{
    ff p2 = two_prod(p.hi, p.hi);  // (hi + lo)^2 to ~2^-48
    p2.lo = fmaf(2.0f * p.hi, p.lo, p2.lo);
    return MASS ? ff_mul(p2, mw) : p2;
}
template <bool LEV, bool MASS>
__device__ __forceinline__ void hparts_site(HParts& acc, ff x, ff p, ff mw, ff cp, float a,
                                            ff xn, bool has_next, const MixedTheta& mt,
                                            const float2* tab, float rs_y = 0.0f)
{
    ff_acc(acc.K, kinetic<MASS>(p, mw));
    ff_acc(acc.L, x);
    const ff r = ff_sub(x, cp);
    ff_acc(acc.R, ff_mul(r, r));
    const ff nh = ff_sub(ff{-mt.mu.hi, -mt.mu.lo}, x);  // -h
    if (LEV) {
        const ff E2 = ff_exp(ff{0.5f * nh.hi, 0.5f * nh.lo}, tab);  // e^{-h/2}
        if (has_next) {
            const ff e = ff_sub(ff_sub(xn, ff_mul(mt.phi_ff, x)), ff_mul_f(E2, rs_y));
            ff_acc(acc.Q, ff_mul(e, e));
        }
        ff_acc(acc.E, ff_mul_f(ff_mul(E2, E2), a));
    } else {
        if (has_next) {
            const ff e = ff_sub(xn, ff_mul(mt.phi_ff, x));
            ff_acc(acc.Q, ff_mul(e, e));
        }
        const ff E = ff_exp(nh, tab);
        ff_acc(acc.E, ff_mul_f(E, a));
    }
}

// The mass m' = -kick / km that the kick v -= km F (km = -kick/m in FP32)
// integrates, in double-float: an approximate reciprocal (rcp.approx, ~2^-23)
// and one correction with the exact residual, so that K = m' v^2 is the
// kinetic energy of exactly the dynamics the kick applies (~2^-46).
__device__ __forceinline__ ff mass_weight(float kick, float km)
{
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(km));
    const float q = -kick * t;
    const float r = fmaf(-q, km, -kick);  // -kick - q km, exact
    return fast_two_sum(q, r * t);
}

// The stationary term (1 - phi^2) x_1^2 / (2 s_eta^2) of S, into Q (weighted
// by 1/(2 s_eta^2)), in double-float: FP64 here would cost every warp that
// predicates it.  With leverage Q is weighted by B/2 and the factor is
// (1 - phi^2)(1 - rho^2).
template <bool LEV>
__device__ __forceinline__ void stationary_part(HParts& acc, ff x1, const MixedTheta& mt)
{
    const ff om = LEV ? mt.st : ff_sub(ff{1.0f, 0.0f}, ff_mul(mt.phi_ff, mt.phi_ff));
    ff_acc(acc.Q, ff_mul(om, ff_mul(x1, x1)));
}

// ---- statistics of a state (model without leverage; see StateStats) ----
constexpr int kStatsFF = 7;
static_assert(sizeof(StateStats) == kStatsFF * sizeof(ff), "StateStats is kStatsFF double-floats");
static_assert(kRecWords == 1 + kStatsFF && kPartialWords == 2 + kStatsFF,
              "record layouts: (dk, statistics) and (sum lnRV, statistics, sum lnRV^2)");
__device__ __forceinline__ ff* stats_ff(StateStats& s) { return reinterpret_cast<ff*>(&s); }
__device__ __forceinline__ void stats_zero(StateStats& s)
{
#pragma unroll
    for (int i = 0; i < kStatsFF; ++i) stats_ff(s)[i] = ff{0.f, 0.f};
}
// One owned site: x = h - mu, xn = x_{t+1} (read only if has_next), lr =
// lnRV, a = y^2/2 (x0 and xT are set by the caller).
__device__ __forceinline__ void stats_site(StateStats& s, ff x, ff xn, bool has_next, ff lr,
                                           float a, const MixedTheta& mt, const float2* tab)
{
    ff_acc(s.sx, x);
    ff_acc(s.sxx, ff_mul(x, x));
    if (has_next) ff_acc(s.sxn, ff_mul(x, xn));
    ff_acc(s.sxl, ff_mul(x, lr));
    const ff nh = ff_sub(ff{-mt.mu.hi, -mt.mu.lo}, x);  // -h
    ff_acc(s.e, ff_mul_f(ff_exp(nh, tab), a));
}

// dH of a trajectory of a series of length T (model without leverage) from
//   dk = sum m v'^2 - sum m v^2 (twice the kinetic difference),
//   s1 = the end state's statistics, centred at the current theta mt,
//   r0 = the start state's record, centred wherever it was taken.
// The energy of eqs. (1)-(3) without its site-independent constants is
//   H = K/2 + sum x / 2 + R / (2 s_u^2) + Q / (2 s_eta^2) + sum (y^2/2) e^{-h},
//   R = sum (x - c')^2 = sxx - 2 sxl + 2 (xi + mu) sx + (terms of the data alone),
//   Q = sum_{t<T-1} (x_{t+1} - phi x_t)^2 + (1 - phi^2) x_0^2
//     = (1 + phi^2) sxx - phi^2 (x_0^2 + x_{T-1}^2) - 2 phi sxn;
// the start's sums are moved to the current centre (x' = x + dmu) and the
// differences taken before they are weighted.  Double-float throughout, one
// FP64 conversion at the end.
__device__ double stats_dH(ff dk, const StateStats& s1, const StatsRec& r0, const MixedTheta& mt,
                           int64_t T)
{
    const StateStats& s0 = r0.s;
    const float th = (float)T;
    const ff Tf = {th, (float)(T - (int64_t)th)};
    const ff T1 = ff_add(Tf, ff{-1.f, 0.f});
    const ff dmu = ff_sub(r0.mu, mt.mu);
    const ff dmu2 = ff_mul(dmu, dmu);
    const ff sx0 = ff_add(s0.sx, ff_mul(Tf, dmu));
    const ff sxx0 = ff_add(ff_add(s0.sxx, ff_mul(ff_mul_f(dmu, 2.f), s0.sx)), ff_mul(Tf, dmu2));
    const ff sxn0 = ff_add(
        ff_add(s0.sxn, ff_mul(dmu, ff_sub(ff_mul_f(s0.sx, 2.f), ff_add(s0.x0, s0.xT)))),
        ff_mul(T1, dmu2));
    const ff sxl0 = ff_add(s0.sxl, ff_mul(dmu, r0.sl));
    const ff x00 = ff_add(s0.x0, dmu), xT0 = ff_add(s0.xT, dmu);
    const ff dsx = ff_sub(s1.sx, sx0), dsxx = ff_sub(s1.sxx, sxx0), dsxn = ff_sub(s1.sxn, sxn0);
    const ff dsxl = ff_sub(s1.sxl, sxl0);
    const ff dx0 = ff_mul(ff_sub(s1.x0, x00), ff_add(s1.x0, x00));  // x_0'^2 - x_0^2
    const ff dxT = ff_mul(ff_sub(s1.xT, xT0), ff_add(s1.xT, xT0));
    const ff dr = ff_add(ff_sub(dsxx, ff_mul_f(dsxl, 2.f)), ff_mul(ff_mul_f(mt.ximu, 2.f), dsx));
    const ff p2 = ff_mul(mt.phi_ff, mt.phi_ff);
    ff dq = ff_mul(ff_add(ff{1.f, 0.f}, p2), dsxx);
    dq = ff_sub(dq, ff_mul(p2, ff_add(dx0, dxT)));
    dq = ff_sub(dq, ff_mul(ff_mul_f(mt.phi_ff, 2.f), dsxn));
    ff dh = ff_mul_f(ff_add(dk, dsx), 0.5f);
    dh = ff_add(dh, ff_mul(mt.hu, dr));
    dh = ff_add(dh, ff_mul(mt.he, dq));
    dh = ff_add(dh, ff_sub(s1.e, s0.e));
    return ff_to_double(dh);
}

// The decisions with the statistics (model without leverage).  s_wrec[w]:
// warp w's (dk, statistics of its owned sites) as kRecWords double-floats.
// A whole series sums its warps in warp order, decides and, on accept, files
// its new state's statistics in place of the old; a tile of a split series
// hands its sums to finish_split_stats in *split_rec.
__device__ __forceinline__ void rec_from(const float2* w, ff& dk, StateStats& st)
{
    dk = ff{w[0].x, w[0].y};
#pragma unroll
    for (int i = 0; i < kStatsFF; ++i) stats_ff(st)[i] = ff{w[1 + i].x, w[1 + i].y};
}
__device__ __forceinline__ void segment_decisions_stats(const TrajArgs& A, const View& v,
                                                        const float2 (*s_wrec)[kRecWords],
                                                        int* s_wacc, float2* split_rec,
                                                        const MixedTheta& mt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (v.sid < 0 || warp != v.g.warp0) return;
    // lane i < kRecWords sums value i over the segment's warps in warp order
    ff di = {0.f, 0.f};
    if (lane < kRecWords)
        for (int w = v.g.warp0; w < v.g.warp0 + v.g.nwarp; ++w)
            di = ff_add(di, ff{s_wrec[w][lane].x, s_wrec[w][lane].y});
    if (v.g.split) {
        if (lane < kRecWords) split_rec[lane] = make_float2(di.hi, di.lo);
        return;
    }
    ff d[kRecWords];
#pragma unroll
    for (int i = 0; i < kRecWords; ++i)
        d[i] = ff{__shfl_sync(0xffffffffu, di.hi, i), __shfl_sync(0xffffffffu, di.lo, i)};
    if (lane == 0) {
        StatsRec* rec = A.rstats + 2 * (int64_t)v.g.series + v.cur;
        StatsRec r1;
        r1.mu = mt.mu;
        r1.ximu = mt.ximu;
        r1.sl = rec->sl;
        r1.sll = rec->sll;
#pragma unroll
        for (int i = 0; i < kStatsFF; ++i) stats_ff(r1.s)[i] = d[1 + i];
        const double dH = stats_dH(d[0], r1.s, *rec, mt, v.si.T);
        const int acc = decide(A, v.g.series, dH, v.cur, false);
        s_wacc[v.g.warp0] = acc;
        if (acc) *rec = r1;  // the state is overwritten in place
    }
}
// The last tile of a split series to arrive sums every tile's sums in tile
// order (warp f takes value f, lane l tiles l, l + 32, ...), decides, flips
// the series' buffer on accept and files the proposal's statistics with it.
__device__ void finish_split_stats(const TrajArgs& A, const View& v, const float2* split_rec,
                                   int* s_flag, float2* s_red, const MixedTheta& mt)
{
    float2* pf = reinterpret_cast<float2*>(A.partials);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid < kRecWords) {
        pf[(int64_t)v.sid * kPartialWords + tid] = split_rec[tid];
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(A.ser_cnt + v.g.series, 1u);
        *s_flag = (prev == (unsigned)v.si.nseg - 1u);
    }
    __syncthreads();
    if (!*s_flag) return;
    __threadfence();
    const int nseg = v.si.nseg;
    for (int f = warp; f < kRecWords; f += nw) {
        ff sum = {0.f, 0.f};
        for (int i0 = lane; i0 < nseg; i0 += 32 * 8) {
            float2 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                w[u] = i0 + 32 * u < nseg
                           ? __ldcg(pf + (int64_t)(v.si.seg0 + i0 + 32 * u) * kPartialWords + f)
                           : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + 32 * u < nseg) sum = ff_add(sum, ff{w[u].x, w[u].y});
        }
        sum = warp_sum_ff(sum);
        if (lane == 0) s_red[f] = make_float2(sum.hi, sum.lo);
    }
    __syncthreads();
    if (tid == 0) {
        ff dk;
        StatsRec r1;
        StatsRec* rec = A.rstats + 2 * (int64_t)v.g.series;
        rec_from(s_red, dk, r1.s);
        r1.mu = mt.mu;
        r1.ximu = mt.ximu;
        r1.sl = rec[v.cur].sl;
        r1.sll = rec[v.cur].sll;
        const double dH = stats_dH(dk, r1.s, rec[v.cur], mt, v.si.T);
        A.ser_cnt[v.g.series] = 0u;
        if (decide(A, v.g.series, dH, v.cur, true)) rec[v.cur ^ 1] = r1;
        __threadfence();
    }
}

// Per-site work outside the leapfrog goes through shared memory: each warp
// loads its sites' inputs and writes their new state with consecutive lanes
// (coalesced), filing each site to or from its owner thread's slots; momenta
// and both ends of dH run in rolled loops over the thread's own slots (fully
// unrolled over J slots they are thousands of instructions per thread, more
// than the instruction caches hold).
template <int J, bool MASS, bool LEV>
__global__ void __launch_bounds__(mixed_ntmax<J, MASS>(), 1) k_traj_mixed(const TrajArgs A)
{
    static_assert(J % 4 == 0, "J must be a multiple of 4");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_wseg[NWMAX], s_wacc[NWMAX], s_flag;
    __shared__ double s_edge_d[4 * NWMAX];
    __shared__ float2 s_exptab[32];
    __shared__ MixedTheta s_mt[NWMAX];
    __shared__ float2 s_wpf[NWMAX], s_splitf;
    // without leverage: per-warp (dk, statistics) and a split tile's sums
    __shared__ float2 s_wrec[LEV ? 1 : NWMAX][kRecWords], s_splitrec[kRecWords];
    const int NT = blockDim.x, NS = mixed_row(NT, J), WS = NS * J, nw = NT >> 5;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    float* s_edge = reinterpret_cast<float*>(s_edge_d);
    if (tid < 32) s_exptab[tid] = g_exptab[tid];
    constexpr int P = J / 2;
    float4* s_ak = reinterpret_cast<float4*>(smem_raw);  // [P][NT] (-a, -a', k, k') of (p, p+P)
    float* s_ak1 = reinterpret_cast<float*>(smem_raw);
    float2* s_dm = reinterpret_cast<float2*>(s_ak + P * NT);  // [P][NT] -kick/m of (p, p+P)
    float* s_dm1 = reinterpret_cast<float*>(s_dm);
    float2* s_v = s_dm + (MASS ? P * NT : 0);  // [P][NT] leverage v of (p, p+P)
    float* s_v1 = reinterpret_cast<float*>(s_v);
    float* s_xh = reinterpret_cast<float*>(s_v + (LEV ? P * NT : 0));  // [J][NS]
    float* s_xl = s_xh + WS;
    float* s_ph = s_xl + WS;
    const bool mass_on = MASS && (A.mass_on == nullptr || *A.mass_on != 0);
    const float dt = (float)A.dtau;
    // slot j is lane j / P of pair j % P
    // slot j of thread t
    auto na_t = [&](int j, int t) -> float& { return s_ak1[((j % P) * NT + t) * 4 + j / P]; };
    auto k_t = [&](int j, int t) -> float& { return s_ak1[((j % P) * NT + t) * 4 + 2 + j / P]; };
    auto dm_t = [&](int j, int t) -> float& { return s_dm1[((j % P) * NT + t) * 2 + j / P]; };
    auto v_t = [&](int j, int t) -> float& { return s_v1[((j % P) * NT + t) * 2 + j / P]; };
    auto na_at = [&](int j) -> float& { return na_t(j, tid); };
    auto k_at = [&](int j) -> float& { return k_t(j, tid); };
    auto dm_at = [&](int j) -> float& { return dm_t(j, tid); };
    auto v_at = [&](int j) -> float& { return v_t(j, tid); };

    for (int b = blockIdx.x; b < A.nbins; b += gridDim.x) {
        float2 X[P], XL[P], PH[P], PL[P];
        MixedConst mc;
        ff h0;             // this thread's owned-site H at the start
        {
            View v;
            load_bin(A, b, s_wseg, s_wacc, v);
            const int base = v.base * J;
            reinterpret_cast<float*>(&s_mt[warp])[lane] =
                reinterpret_cast<const float*>(A.theta_f + v.g.series)[lane];
            __syncwarp();
            const MixedTheta& mt = s_mt[warp];
            mc.phi = mt.phi;
            mc.c0 = mt.c0;
            mc.c1 = mt.c1;
            mc.cmu = mt.cmu;
            mc.dt = dt;
            // substeps {kick; drift} of the scheme after its first drift (the
            // end drifts of consecutive steps merged): leapfrog {kick dtau;
            // drift dtau (last dtau/2)} after dtau/2; second-order minimum-norm
            // {kick dtau/2; drift (1-2 lambda) dtau or 2 lambda dtau} after
            // lambda dtau; fourth-order four kicks and drifts per step
            const MixedScheme& ms = A.msch;
            mc.kick = ms.kick;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                mc.kq[i] = ms.kq[i];
                mc.kr[i] = ms.kr[i];
                mc.r[i] = ms.r[i];
            }
            mc.r_last = ms.r_last;
            mc.nk = ms.nk;
            mc.n_sub = ms.nk * A.n_md;
            mc.la = v.n - 1 - base;
            mc.first = v.first;
            const int64_t off = v.si.off, wlo = v.g.wlo;
            const float2* hin = v.cur ? A.h1f : A.h0f;
            // pass 1a: momenta (standard normals, or the caller's p) -> s_ph;
            // the two sources in separate loops, so that neither is predicated
            // through the other (the FP64 -> FP32 conversions of p_in run on
            // the FP64 pipe)
            if (A.p_in) {
#pragma unroll 1
                for (int j = 0; j < J; ++j) {
                    const int ii = base + j;
                    s_ph[j * NS + tid] = ii < v.n ? (float)A.p_in[off + wlo + ii] : 0.0f;
                }
            } else {
#pragma unroll 2
                for (int q = 0; q < J / 4; ++q) {
                    const int64_t s0 = wlo + base + 4 * q;
                    const u64x4 r = philox_block(A.seed, (uint64_t)v.g.series, A.traj, STREAM_MOM,
                                                 (uint64_t)(s0 >> 2));
                    float z[4];
                    box_muller_f(u01_23(r.w[0]), u01_23(r.w[1]), z[0], z[1]);
                    box_muller_f(u01_23(r.w[2]), u01_23(r.w[3]), z[2], z[3]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) s_ph[(4 * q + i) * NS + tid] = z[i];
                }
            }
            // the previous trajectory's snapshot, which is this one's start
            // state, in a loop of its own: a global store between the load
            // pass's loads would keep them from being issued together
            if (A.snap_prev) {
                const int wb = (warp - v.g.warp0) * 32 * J;
                for (int kk = lane; kk < 32 * J; kk += 32) {
                    const int64_t sg = wlo + wb + kk;
                    if (v.sid >= 0 && sg >= v.g.lo && sg < v.g.hi) {
                        const float2 hv = hin[off + sg];
                        A.snap_prev[off + sg] = hv.x + hv.y;
                    }
                }
            }
            // pass 1b: site constants, x, mass -> shared memory, and H at the
            // start of the sites the lane loads.  The warp loads its 32 J
            // consecutive sites with consecutive lanes (coalesced) and files
            // each into its owner's slots; the warp's threads share one
            // segment.  H is formed from the values as filed (the end of the
            // trajectory reads the same ones back), and summed per warp with
            // the end's H, so which lane takes which site does not matter.
            __syncwarp();  // the owners' momenta of pass 1a are in s_ph
            HParts acc;
            hparts_zero(acc);
            {
                const int wb = (warp - v.g.warp0) * 32 * J;
#pragma unroll 2
                for (int kk = lane; kk < 32 * J; kk += 32) {
                    const int ol = kk / J, j = kk - ol * J;
                    const int to = (warp << 5) + ol;  // the owner thread
                    const int ii = wb + kk;
                    const int64_t s = off + wlo + ii;
                    const bool act = ii < v.n;
                    const float2 hv = act ? hin[s] : make_float2(mt.mu.hi, mt.mu.lo);
                    ff x = two_sum(hv.x, -mt.mu.hi);  // x = h - mu in double-float
                    x.lo += hv.y - mt.mu.lo;
                    x = fast_two_sum(x.hi, x.lo);
                    const float as = act ? A.a_f[s] : 0.0f;  // y^2/2 with the sign of y
                    const float a = fabsf(as);
                    const float2 lr = act ? A.lr_f[s] : make_float2(mt.ximu.hi, mt.ximu.lo);
                    ff cp = two_sum(lr.x, -mt.ximu.hi);  // c' = lnRV - xi - mu
                    cp.lo += lr.y - mt.ximu.lo;
                    float na = -a, vv = 0.0f;
                    if (LEV) {
                        const bool has_next = act && wlo + ii + 1 < v.si.T;
                        na = has_next ? -a * mt.ia : -a;
                        vv = has_next ? mt.rsb * copysignf(sqrtf(2.0f * a), as) : 0.0f;
                        v_t(j, to) = vv;
                    }
                    na_t(j, to) = na;
                    k_t(j, to) = fmaf(-mt.iu, cp.hi + cp.lo, 0.5f);
                    float kmv = -mc.kick;
                    float p0 = s_ph[j * NS + to];
                    if (MASS) {
                        const float mi = (act && mass_on) ? A.minv[s] : 1.0f;
                        kmv = -mc.kick * mi;
                        dm_t(j, to) = kmv;
                        // the velocity v = p/m: p ~ N(0, m_t) is the drawn normal
                        // times sqrt(m_t), so v is the normal times sqrt(1/m_t); a
                        // given p is divided by the mass the kick integrates
                        if (A.p_in)
                            p0 = act ? (float)(A.p_in[s] * ((double)kmv / -(double)mc.kick))
                                     : 0.0f;
                        else
                            p0 = p0 * sqrtf(mi);
                        s_ph[j * NS + to] = p0;
                    }
                    s_xh[j * NS + to] = x.hi;
                    s_xl[j * NS + to] = x.lo;
                    // H at the start of this site if the segment owns it; without
                    // leverage only K: the potential part comes from the state's
                    // stored statistics (stats_dH)
                    const int64_t sg = wlo + ii;
                    if (v.sid >= 0 && sg >= v.g.lo && sg < v.g.hi) {
                        const ff mw = MASS ? mass_weight(mc.kick, kmv) : ff{1.f, 0.f};
                        if (LEV) {
                            const bool has_next = sg + 1 < v.si.T;
                            ff xn = {0.f, 0.f};
                            if (has_next) {  // inside the window: owned sites are not its last
                                const float2 hn = hin[s + 1];
                                xn = two_sum(hn.x, -mt.mu.hi);
                                xn.lo += hn.y - mt.mu.lo;
                                xn = fast_two_sum(xn.hi, xn.lo);
                            }
                            const float ah = has_next ? -na * mt.omr : -na;
                            hparts_site<LEV, MASS>(acc, x, ff{p0, 0.f}, mw, cp, ah, xn, has_next,
                                                   mt, s_exptab, vv * mt.ibf);
                            if (sg == 0) stationary_part<LEV>(acc, x, mt);
                        } else {
                            ff_acc(acc.K, kinetic<MASS>(ff{p0, 0.f}, mw));
                        }
                    }
                }
            }
            __syncthreads();
            mc.vL = (LEV && !v.first) ? s_v1[((P - 1) * NT + tid - 1) * 2 + 1] : 0.0f;
            mc.cfirst = (LEV && v.first) ? mt.cst : 0.0f;
            h0 = LEV ? hparts_total(acc, mt) : ff_add(acc.K, ff{0.f, 0.f});
            // registers <- shared memory, then the first half step of eq. (6)
#pragma unroll
            for (int q = 0; q < P; ++q) {
                X[q] = f2(s_xh[q * NS + tid], s_xh[(q + P) * NS + tid]);
                XL[q] = f2(s_xl[q * NS + tid], s_xl[(q + P) * NS + tid]);
                PH[q] = f2(s_ph[q * NS + tid], s_ph[(q + P) * NS + tid]);
                PL[q] = f2(0.0f, 0.0f);
            }
            const float r0 = A.msch.r_first;  // first drift
#pragma unroll
            for (int q = 0; q < P; ++q) cupd2(X[q], XL[q], f2(r0 * dt, r0 * dt), PH[q]);
        }

        int par = 0;
        const bool mid_end = mc.la >= 0 && mc.la < J - 1;
        if (__any_sync(0xffffffffu, mid_end)) {
            if (A.msch.kv)
                mixed_steps<J, MASS, true, LEV, true>(X, XL, PH, PL, s_ak, s_dm, s_v, s_edge, par,
                                                      nw, A.n_md, mc);
            else
                mixed_steps<J, MASS, true, LEV, false>(X, XL, PH, PL, s_ak, s_dm, s_v, s_edge,
                                                       par, nw, A.n_md, mc);
        } else {
            if (A.msch.kv)
                mixed_steps<J, MASS, false, LEV, true>(X, XL, PH, PL, s_ak, s_dm, s_v, s_edge,
                                                       par, nw, A.n_md, mc);
            else
                mixed_steps<J, MASS, false, LEV, false>(X, XL, PH, PL, s_ak, s_dm, s_v, s_edge,
                                                        par, nw, A.n_md, mc);
        }

        // ---- the end of the trajectory: state -> shared memory (x over the
        // start's slots, p lo over k, which the leapfrog no longer needs) ----
        __syncthreads();  // every warp is done reading k and the start state
#pragma unroll
        for (int q = 0; q < P; ++q) {
            s_xh[q * NS + tid] = X[q].x;
            s_xh[(q + P) * NS + tid] = X[q].y;
            s_xl[q * NS + tid] = XL[q].x;
            s_xl[(q + P) * NS + tid] = XL[q].y;
            s_ph[q * NS + tid] = PH[q].x;
            s_ph[(q + P) * NS + tid] = PH[q].y;
            k_at(q) = PL[q].x;
            k_at(q + P) = PL[q].y;
        }
        __syncthreads();
        View v;
        view_of(A, s_wseg, v);
        const int base = v.base * J;
        const MixedTheta& mt = s_mt[warp];
        const int64_t off = v.si.off, wlo = v.g.wlo;
        HParts acc;
        hparts_zero(acc);
        StateStats st;
        stats_zero(st);
#pragma unroll 1
        for (int j = 0; j < J; ++j) {
            const int64_t sg = wlo + base + j;
            if (v.sid < 0 || sg < v.g.lo || sg >= v.g.hi) continue;
            const ff x = {s_xh[j * NS + tid], s_xl[j * NS + tid]};
            const int nidx = j + 1 < J ? (j + 1) * NS + tid : tid + 1;
            const ff xn = {s_xh[nidx], s_xl[nidx]};
            const float2 lr = A.lr_f[off + sg];
            const ff mw = MASS ? mass_weight(mc.kick, dm_at(j)) : ff{1.f, 0.f};
            const bool has_next = sg + 1 < v.si.T;
            const ff pv = {s_ph[j * NS + tid], k_at(j)};
            if (LEV) {
                ff cp = two_sum(lr.x, -mt.ximu.hi);
                cp.lo += lr.y - mt.ximu.lo;
                const float a = has_next ? -na_at(j) * mt.omr : -na_at(j);
                hparts_site<LEV, MASS>(acc, x, pv, mw, cp, a, xn, has_next, mt, s_exptab,
                                       v_at(j) * mt.ibf);
            } else {
                ff_acc(acc.K, kinetic<MASS>(pv, mw));
                stats_site(st, x, xn, has_next, ff{lr.x, lr.y}, -na_at(j), mt, s_exptab);
            }
        }
        if (!LEV && v.sid >= 0) {  // the series' first and last sites, where owned
            const int64_t s0 = wlo + base;
            if (s0 == 0 && v.g.lo == 0) st.x0 = ff{s_xh[tid], s_xl[tid]};
            const int64_t jl = v.si.T - 1 - s0;
            if (jl >= 0 && jl < J && v.si.T - 1 >= v.g.lo && v.si.T - 1 < v.g.hi)
                st.xT = ff{s_xh[(int)jl * NS + tid], s_xl[(int)jl * NS + tid]};
        }
        if (LEV) {
            if (v.sid >= 0 && wlo + base == 0 && v.g.lo == 0)
                stationary_part<LEV>(acc, ff{s_xh[tid], s_xl[tid]}, mt);
            ff dh = ff_sub(hparts_total(acc, mt), h0);
            dh = warp_sum_ff(dh);
            if (lane == 0) s_wpf[warp] = make_float2(dh.hi, dh.lo);
        } else {
            // (dk, statistics) of the warp's owned sites, each summed in a
            // fixed order
            ff r = warp_sum_ff(ff_sub(ff_add(acc.K, ff{0.f, 0.f}), h0));
            if (lane == 0) s_wrec[warp][0] = make_float2(r.hi, r.lo);
#pragma unroll
            for (int i = 0; i < kStatsFF; ++i) {
                r = warp_sum_ff(ff_add(stats_ff(st)[i], ff{0.f, 0.f}));
                if (lane == 0) s_wrec[warp][1 + i] = make_float2(r.hi, r.lo);
            }
        }
        __syncthreads();
        if (LEV) segment_decisions_ff(A, v, s_wpf, s_wacc, &s_splitf);
        else segment_decisions_stats(A, v, s_wrec, s_wacc, s_splitrec, mt);
        __syncthreads();
        const bool write_h = v.sid >= 0 && (v.g.split || s_wacc[v.g.warp0]);
        float2* hout = v.g.split ? (v.cur ? A.h0f : A.h1f) : (v.cur ? A.h1f : A.h0f);
        if (write_h) {
            // the warp writes its 32 J consecutive sites with consecutive lanes
            // (coalesced), reading each site from its owner's slot; write_h is
            // the same for the whole warp (a segment is whole warps)
            const int64_t wbase = wlo + (int64_t)(warp - v.g.warp0) * 32 * J;
#pragma unroll 1
            for (int k = lane; k < 32 * J; k += 32) {
                const int ol = k / J, j = k - ol * J;
                const int64_t sg = wbase + k;
                if (sg >= v.g.lo && sg < v.g.hi) {
                    const int idx = j * NS + warp * 32 + ol;
                    ff hh = two_sum(s_xh[idx], mt.mu.hi);
                    hh.lo += s_xl[idx] + mt.mu.lo;
                    hh = fast_two_sum(hh.hi, hh.lo);
                    hout[off + sg] = make_float2(hh.hi, hh.lo);
                }
            }
        }
        if (A.p_out) {  // a loop of its own: its FP64 conversions are never predicated
#pragma unroll 1
            for (int j = 0; j < J; ++j) {
                const int64_t sg = wlo + base + j;
                if (v.sid >= 0 && sg >= v.g.lo && sg < v.g.hi)
                    A.p_out[off + sg] = ((double)s_ph[j * NS + tid] + (double)k_at(j)) *
                                        (MASS ? -(double)mc.kick / (double)dm_at(j) : 1.0);
            }
        }
        if (v.g.split) {
            if (LEV) finish_split_ff(A, v, s_splitf, &s_flag);
            else finish_split_stats(A, v, s_splitrec, &s_flag, s_wrec[0], s_mt[v.g.warp0]);
        }
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
