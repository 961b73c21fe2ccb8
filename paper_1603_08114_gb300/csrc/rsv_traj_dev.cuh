// rsv_traj_dev.cuh -- device code of the trajectory kernels, shared by the
// per-trajectory kernels (rsv_traj.cu) and the persistent chain kernel
// (rsv_chain.cu).  See rsv_traj.cu for the method and the GB300 design.
#pragma once

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
// barrier).  TH: also theta of the series in FP64 (the mixed kernels keep
// theta's constants in shared memory and skip those loads).
template <bool TH = true>
__device__ __forceinline__ void view_of(const TrajArgs& A, const int* s_wseg, View& v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v.sid = s_wseg[warp];
    if (v.sid >= 0) {
        v.g = A.segs[v.sid];
        v.si = A.ser[v.g.series];
        if (TH) {
            v.th = A.theta ? load_theta(A.theta + 5 * (int64_t)v.g.series) : A.th_inline;
            v.th.rho = A.rho;
        }
        v.cur = A.ser_cur ? *(volatile int*)(A.ser_cur + v.g.series) : 0;
    } else {
        // idle warp: an empty segment with harmless parameters
        v.g = Seg{0, 0, 0, 0, 0, warp, 1, 0};
        v.si = SerInfo{0, 1, 1, 0};
        if (TH) v.th = ThetaD{0.5, 0.0, 0.0, 1.0, 1.0};
        v.cur = 0;
    }
    const int ts = (warp - v.g.warp0) * 32 + lane;  // thread index inside the segment
    v.n = (int)(v.g.whi - v.g.wlo);
    v.base = ts;  // the caller scales it by J
    v.first = (ts == 0);
}

// The segments of bin b into s_wseg (one id per warp, -1 for an idle warp) and
// this warp's view.  With wg/wsi/wcur given, the warp also files its segment,
// series and current-buffer selector there (view_filed reads them back without
// global loads).
template <bool TH = true>
__device__ __forceinline__ void load_bin(const TrajArgs& A, int b, int* s_wseg, int* s_wacc,
                                         View& v, Seg* wg = nullptr, SerInfo* wsi = nullptr,
                                         int* wcur = nullptr)
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
    view_of<TH>(A, s_wseg, v);
    if (wg && (tid & 31) == 0) {
        const int warp = tid >> 5;
        wg[warp] = v.g;
        wsi[warp] = v.si;
        wcur[warp] = v.cur;
    }
}

// The view load_bin filed for this warp (theta not included).
__device__ __forceinline__ void view_filed(const int* s_wseg, const Seg* wg, const SerInfo* wsi,
                                           const int* wcur, View& v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v.sid = s_wseg[warp];
    v.g = wg[warp];
    v.si = wsi[warp];
    v.cur = wcur[warp];
    const int ts = (warp - v.g.warp0) * 32 + lane;
    v.n = (int)(v.g.whi - v.g.wlo);
    v.base = ts;
    v.first = (ts == 0);
}

// Metropolis decision of one series (Sec. 3): accept iff ln u < -dH; a
// non-finite dH rejects and raises ST_NONFINITE.
// ln u of a drawn u is taken first in FP32 (logf of u rounded to FP32: off by
// at most 2^-24 + a few ulp of ln u, |ln u| < 37); only when that lies within
// 1e-6 (1 + |ln u|) of -dH, where the comparison could go either way, is it
// taken in FP64, so the decision is the FP64 comparison's at the cost of one
// FP64 logarithm in about a million trajectories.
// The drawn uniform of trajectory traj's Metropolis test.
__device__ __forceinline__ double metropolis_u(uint64_t seed, int series, uint64_t traj)
{
    const u64x4 w = philox_block(seed, (uint64_t)series, traj, STREAM_MH, 0);
    return u01_53(w.w[0]);
}
__device__ int metropolis_accept_u(double u, double dH)
{
    if (!isfinite(dH)) return 0;
    const float lf = logf((float)u);
    const double gap = (double)lf + dH;  // ln u - (-dH), to within the margin
    if (fabs(gap) > 1e-6 * (1.0 + fabs((double)lf))) return gap < 0.0 ? 1 : 0;
    return log(u) < -dH ? 1 : 0;
}
__device__ int metropolis_accept(const double* log_u, uint64_t seed, int series, uint64_t traj,
                                 double dH)
{
    if (log_u) return (isfinite(dH) && log_u[series] < -dH) ? 1 : 0;
    return metropolis_accept_u(metropolis_u(seed, series, traj), dH);
}
__device__ int decide(const TrajArgs& A, int series, double dH, int cur, bool flip)
{
    const bool fin = isfinite(dH);
    const int acc = metropolis_accept(A.log_u, A.seed, series, A.traj, dH);
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
//   s_ak  float4 [P][NTP]  (-a_p, -a_{p+P}, k_p, k_{p+P}): a = y^2/2,
//                         k = 1/2 - c'/s_u^2
//   s_dm  float2 [P][NTP]  -kick/m of the pair (with a mass only; the state
//                         then holds the velocity v = p/m)
//   s_v   float2 [P][NTP]  the leverage weights v of the pair (leverage only)
//   s_xh, s_xl, s_ph  float [J][NS]  x (hi, lo) and p hi at the start of the
//                         trajectory and again at its end (p lo then over k);
//                         rows NS = mixed_row(NT, J) slots apart
// The arrays the leapfrog reads every step keep rows of NTP = NT slots: a
// warp's float4 (float2) row segment is then four (two) whole 128-byte lines;
// the rows of the start and end state, which only the load and write passes
// and the energies touch, are padded against bank conflicts instead.
// ---------------------------------------------------------------------------
// (with a mass and J = 4 at most 768 threads: its load pass needs more than
// the 64 registers a 1024-thread block leaves)
template <int J, bool MASS>
constexpr int mixed_ntmax()
{
    return J <= 4 ? (MASS ? 768 : 1024) : J <= 8 ? 768 : J <= 12 ? 640 : J <= 16 ? 512 : 384;
}

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

// ---- double-float arithmetic on pairs of lanes (FADD2/FMUL2/FFMA2) --------
// An ff2 holds two independent double-floats, (hi.x, lo.x) and (hi.y, lo.y);
// every operation is the scalar ff operation of rsv_device.cuh lane by lane,
// with the same roundings, at half the instruction count.
struct ff2 {
    float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ ff2 ff2_zero() { return ff2{f2(0.f, 0.f), f2(0.f, 0.f)}; }
__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return ff2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    return ff2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ ff2 two_prod2(float2 a, float2 b)
{
    const float2 p = mul2(a, b);
    return ff2{p, fma2(a, b, neg2(p))};
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b)
{
    ff2 s = two_sum2(a.hi, b.hi);
    s.lo = add2(s.lo, add2(a.lo, b.lo));
    return fast_two_sum2(s.hi, s.lo);
}
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2{neg2(b.hi), neg2(b.lo)}); }
__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b)
{
    ff2 p = two_prod2(a.hi, b.hi);
    p.lo = fma2(a.hi, b.lo, fma2(a.lo, b.hi, p.lo));
    return fast_two_sum2(p.hi, p.lo);
}
__device__ __forceinline__ ff2 ff2_mul_f(ff2 a, float2 b)
{
    ff2 p = two_prod2(a.hi, b);
    p.lo = fma2(a.lo, b, p.lo);
    return fast_two_sum2(p.hi, p.lo);
}
// acc += v (the small part renormalised only when read, as ff_acc)
__device__ __forceinline__ void ff2_acc(ff2& acc, ff2 v)
{
    const ff2 s = two_sum2(acc.hi, v.hi);
    acc.hi = s.hi;
    acc.lo = add2(acc.lo, add2(s.lo, v.lo));
}
// the two lanes' sum, lane x first
__device__ __forceinline__ ff ff2_fold(ff2 a)
{
    return ff_add(ff_add(ff{a.hi.x, a.lo.x}, ff{0.f, 0.f}), ff{a.hi.y, a.lo.y});
}
// ff_exp lane by lane: the reduction by ln2/32 and the polynomial on the
// pair, the table look-up and the power-of-two scale per lane
__device__ __forceinline__ ff2 ff2_exp(ff2 t, const float2* tab)
{
    const float2 C_hi = f2(0x1.62e43p-6f, 0x1.62e43p-6f), C_lo = f2(-0x1.05c61p-34f, -0x1.05c61p-34f);
    const float2 sh = f2(0x1.8p23f, 0x1.8p23f);
    const float2 kr = fma2(t.hi, f2(46.166241308446828f, 46.166241308446828f), sh);
    const int k0 = __float_as_int(kr.x) - 0x4B400000, k1 = __float_as_int(kr.y) - 0x4B400000;
    const float2 kf = sub2(kr, sh);
    ff2 kc = two_prod2(kf, C_hi);
    kc.lo = fma2(kf, C_lo, kc.lo);
    const ff2 r = ff2_sub(t, kc);
    const float2 x = r.hi;
    const float2 poly =
        fma2(x, fma2(x, fma2(x, f2(1.0f / 120.0f, 1.0f / 120.0f), f2(1.0f / 24.0f, 1.0f / 24.0f)),
                     f2(1.0f / 6.0f, 1.0f / 6.0f)),
             f2(0.5f, 0.5f));
    const float2 q = mul2(mul2(x, x), poly);
    ff2 sm = two_sum2(x, q);
    sm.lo = add2(sm.lo, r.lo);
    ff2 e = two_sum2(f2(1.0f, 1.0f), sm.hi);
    e.lo = add2(e.lo, sm.lo);
    e = fast_two_sum2(e.hi, e.lo);
    const float2 t0 = tab[k0 & 31], t1 = tab[k1 & 31];
    const ff2 res = ff2_mul(ff2{f2(t0.x, t1.x), f2(t0.y, t1.y)}, e);
    const float2 sc = f2(__int_as_float(((k0 >> 5) + 127) << 23), __int_as_float(((k1 >> 5) + 127) << 23));
    return ff2{mul2(res.hi, sc), mul2(res.lo, sc)};
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
// s_ak: float4 [P][NTP] = (-a_p, -a_{p+P}, k_p, k_{p+P}); s_dm: float2 [P][NTP]
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
// e^{-h} is taken as (e^{-h/2})^2 from one ex2.  s_v: float2 [P][NTP] of v.
template <int J, bool MASS, bool EDGE, bool LEV, bool KV>
__device__ __forceinline__ void mixed_steps(float2 (&X)[J / 2], float2 (&XL)[J / 2],
                                            float2 (&PH)[J / 2], float2 (&PL)[J / 2],
                                            const float4* __restrict__ s_ak,
                                            const float2* __restrict__ s_dm,
                                            const float2* __restrict__ s_v, float* s_edge,
                                            int& par, int nw, int n_md, const MixedConst& c)
{
    constexpr int P = J / 2;
    const int NTP = mixed_ntp(blockDim.x), tid = threadIdx.x;
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
        const float4 ak = s_ak[q * NTP + tid];
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
            w = fma2(s_v[q * NTP + tid], e2, zero);
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
        const float2 km = MASS ? (KV ? fma2(s_dm[q * NTP + tid], kc, zero) : s_dm[q * NTP + tid])
                               : (KV ? kc : ndt);
        cupd2(PH[q], PL[q], km, f);
        cupd2(X[q], XL[q], cx, PH[q]);
        return w;
    };
    // unrolled, so that the compiler alternates the registers of the state's
    // old and new values between substeps instead of copying them back
    // (measured: ~80 fewer ALU instructions per SMSP and step, -3 % per step)
#pragma unroll(J >= 16 ? 2 : 4)
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
            const float2 vP = s_v[(P - 1) * NTP + tid];
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
    const float q = __fmul_rn(-kick, t);
    const float r = __fmaf_rn(-q, km, -kick);  // -kick - q km, exact
    return fast_two_sum(q, __fmul_rn(r, t));
}

// mass_weight lane by lane
__device__ __forceinline__ ff2 mass_weight2(float2 kick, float2 km)
{
    float t0, t1;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t0) : "f"(km.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t1) : "f"(km.y));
    const float2 t = f2(t0, t1);
    const float2 q = mul2(neg2(kick), t);
    const float2 r = fma2(neg2(q), km, neg2(kick));
    return fast_two_sum2(q, mul2(r, t));
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
// The shared memory of the mixed trajectory body besides its dynamic part.
template <bool LEV>
struct MixedSmem {
    int wseg[NWMAX], wacc[NWMAX], flag;
    // each warp's segment, series and current-buffer selector (load_bin)
    Seg wg[NWMAX];
    SerInfo wsi[NWMAX];
    int wcur[NWMAX];
    double edge_d[4 * NWMAX];
    float2 exptab[32];
    MixedTheta mt[NWMAX];
    float2 wpf[NWMAX], splitf;
    // without leverage: per-warp (dk, statistics) and a split tile's sums
    float2 wrec[LEV ? 1 : NWMAX][kRecWords], splitrec[kRecWords];
    // persistent chain: the buffer holding the current state, the mass flag,
    // where this trajectory's records go
    int cur, mass_on;
    double* partials;
};

// State loads: a persistent chain reads states other blocks wrote during the
// launch, so they bypass L1 (cached in L2 only).
template <bool PERSIST>
__device__ __forceinline__ float2 ld_state(const float2* p)
{
    return PERSIST ? __ldcg(p) : *p;
}

// Persistent chain: the block's record (twice the kinetic difference and the
// end state's statistics, each summed over the segment's warps in warp order)
// into partials[sid], kPartialWords double-floats per segment.
__device__ __forceinline__ void persist_record(double* partials, const View& v,
                                               const float2 (*s_wrec)[kRecWords])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (v.sid < 0 || warp != v.g.warp0 || lane >= kRecWords) return;
    ff di = {0.f, 0.f};
    for (int w = v.g.warp0; w < v.g.warp0 + v.g.nwarp; ++w)
        di = ff_add(di, ff{s_wrec[w][lane].x, s_wrec[w][lane].y});
    reinterpret_cast<float2*>(partials)[(int64_t)v.sid * kPartialWords + lane] =
        make_float2(di.hi, di.lo);
}

// One bin of a mixed trajectory (the whole block).  PERSIST: a bin of the
// persistent chain kernel (rsv_chain.cu): theta's constants already in
// s_mt, the momenta already in s_ph, the current buffer in S.cur, state
// loads through L2, and no decision (the block's record goes to partials,
// the end state to the other buffer).
template <int J, bool MASS, bool LEV, bool PERSIST>
__device__ __forceinline__ void traj_mixed_bin(const TrajArgs& A, int b, MixedSmem<LEV>& S,
                                               unsigned char* smem_raw, float* snap_prev)
{
    static_assert(J % 4 == 0, "J must be a multiple of 4");
    static_assert(!(PERSIST && LEV), "the persistent chain is for the model without leverage");
    int* s_wseg = S.wseg;
    int* s_wacc = S.wacc;
    int& s_flag = S.flag;
    float2* s_exptab = S.exptab;
    MixedTheta* s_mt = S.mt;
    float2* s_wpf = S.wpf;
    float2& s_splitf = S.splitf;
    auto s_wrec = S.wrec;
    float2* s_splitrec = S.splitrec;
    const int NT = blockDim.x, NTP = mixed_ntp(NT), NS = mixed_row(NT, J), WS = NS * J,
              nw = NT >> 5;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    float* s_edge = reinterpret_cast<float*>(S.edge_d);
    constexpr int P = J / 2;
    float4* s_ak = reinterpret_cast<float4*>(smem_raw);  // [P][NTP] (-a, -a', k, k') of (p, p+P)
    float* s_ak1 = reinterpret_cast<float*>(smem_raw);
    float2* s_dm = reinterpret_cast<float2*>(s_ak + P * NTP);  // [P][NTP] -kick/m of (p, p+P)
    float* s_dm1 = reinterpret_cast<float*>(s_dm);
    float2* s_v = s_dm + (MASS ? P * NTP : 0);  // [P][NTP] leverage v of (p, p+P)
    float* s_v1 = reinterpret_cast<float*>(s_v);
    float* s_xh = reinterpret_cast<float*>(s_v + (LEV ? P * NTP : 0));  // [J][NS]
    float* s_xl = s_xh + WS;
    float* s_ph = s_xl + WS;
    const bool mass_on =
        MASS && (PERSIST ? S.mass_on != 0 : (A.mass_on == nullptr || *A.mass_on != 0));
    const float dt = (float)A.dtau;
    // slot j is lane j / P of pair j % P
    // slot j of thread t
    auto na_t = [&](int j, int t) -> float& { return s_ak1[((j % P) * NTP + t) * 4 + j / P]; };
    auto k_t = [&](int j, int t) -> float& { return s_ak1[((j % P) * NTP + t) * 4 + 2 + j / P]; };
    auto dm_t = [&](int j, int t) -> float& { return s_dm1[((j % P) * NTP + t) * 2 + j / P]; };
    auto v_t = [&](int j, int t) -> float& { return s_v1[((j % P) * NTP + t) * 2 + j / P]; };
    auto na_at = [&](int j) -> float& { return na_t(j, tid); };
    auto k_at = [&](int j) -> float& { return k_t(j, tid); };
    auto dm_at = [&](int j) -> float& { return dm_t(j, tid); };
    auto v_at = [&](int j) -> float& { return v_t(j, tid); };

    float2 X[P], XL[P], PH[P], PL[P];
    MixedConst mc;
    ff h0;             // this thread's owned-site H at the start
    {
        View v;
        // a persistent chain filed its block's view once, before its first
        // trajectory
        if (PERSIST) view_filed(s_wseg, S.wg, S.wsi, S.wcur, v);
        else load_bin<false>(A, b, s_wseg, s_wacc, v, S.wg, S.wsi, S.wcur);
        if (PERSIST) v.cur = S.cur;
        const int base = v.base * J;
        if (!PERSIST)  // a persistent chain keeps the constants of its theta in s_mt
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
        if (PERSIST) {
            // a persistent chain has drawn the momenta into s_ph already
        } else if (A.p_in) {
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
        // (all of the lane's loads first: one L2 round trip, not one per site)
        if (snap_prev) {
            const int wb = (warp - v.g.warp0) * 32 * J;
            float2 hv[J];
#pragma unroll
            for (int it = 0; it < J; ++it) {
                const int64_t sg = wlo + wb + lane + 32 * it;
                const bool own = v.sid >= 0 && sg >= v.g.lo && sg < v.g.hi;
                hv[it] = own ? ld_state<PERSIST>(hin + off + sg) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int it = 0; it < J; ++it) {
                const int64_t sg = wlo + wb + lane + 32 * it;
                if (v.sid >= 0 && sg >= v.g.lo && sg < v.g.hi) snap_prev[off + sg] = hv[it].x + hv[it].y;
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
                const float2 hv = act ? ld_state<PERSIST>(hin + s) : make_float2(mt.mu.hi, mt.mu.lo);
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
        mc.vL = (LEV && !v.first) ? s_v1[((P - 1) * NTP + tid - 1) * 2 + 1] : 0.0f;
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
        // (k, k') of the pair, one 8-byte store
        *reinterpret_cast<float2*>(&k_at(q)) = PL[q];
    }
    __syncthreads();
    View v;
    view_filed(s_wseg, S.wg, S.wsi, S.wcur, v);
    if (PERSIST) v.cur = S.cur;
    const int base = v.base * J;
    const MixedTheta& mt = s_mt[warp];
    const int64_t off = v.si.off, wlo = v.g.wlo;
    HParts acc;
    hparts_zero(acc);
    StateStats st;
    stats_zero(st);
    if constexpr (LEV) {
        // four sites per iteration: each site's double-float sums are a long
        // dependent chain, and interleaved chains keep the pipes busier
#pragma unroll 4
        for (int j = 0; j < J; ++j) {
            const int64_t sg = wlo + base + j;
            if (v.sid < 0 || sg < v.g.lo || sg >= v.g.hi) continue;
            const float2 lr = A.lr_f[off + sg];
            const ff x = {s_xh[j * NS + tid], s_xl[j * NS + tid]};
            const int nidx = j + 1 < J ? (j + 1) * NS + tid : tid + 1;
            const ff xn = {s_xh[nidx], s_xl[nidx]};
            const ff mw = MASS ? mass_weight(mc.kick, dm_at(j)) : ff{1.f, 0.f};
            const bool has_next = sg + 1 < v.si.T;
            const ff pv = {s_ph[j * NS + tid], k_at(j)};
            ff cp = two_sum(lr.x, -mt.ximu.hi);
            cp.lo += lr.y - mt.ximu.lo;
            const float a = has_next ? -na_at(j) * mt.omr : -na_at(j);
            hparts_site<LEV, MASS>(acc, x, pv, mw, cp, a, xn, has_next, mt, s_exptab,
                                   v_at(j) * mt.ibf);
        }
    } else {
        // K and the statistics of the pair (q, q + P) at once, in the two
        // lanes of packed instructions (each lane the scalar site formulas of
        // kinetic and stats_site); a slot the segment does not own enters as
        // zeros, which add nothing
        ff2 K2 = ff2_zero(), sx2 = ff2_zero(), sxx2 = ff2_zero(), sxn2 = ff2_zero(),
            sxl2 = ff2_zero(), se2 = ff2_zero();
        const float2 kick2 = f2(mc.kick, mc.kick);
        const ff2 nmu = {f2(-mt.mu.hi, -mt.mu.hi), f2(-mt.mu.lo, -mt.mu.lo)};
#pragma unroll 2
        for (int q = 0; q < P; ++q) {
            const int j0 = q, j1 = q + P;
            const int64_t g0 = wlo + base + j0, g1 = wlo + base + j1;
            const bool o0 = v.sid >= 0 && g0 >= v.g.lo && g0 < v.g.hi;
            const bool o1 = v.sid >= 0 && g1 >= v.g.lo && g1 < v.g.hi;
            const bool n0 = o0 && g0 + 1 < v.si.T, n1 = o1 && g1 + 1 < v.si.T;
            const float2 lr0 = o0 ? A.lr_f[off + g0] : f2(0.f, 0.f);
            const float2 lr1 = o1 ? A.lr_f[off + g1] : f2(0.f, 0.f);
            const int i0 = j0 * NS + tid, i1 = j1 * NS + tid;
            const int m0 = (j0 + 1) * NS + tid, m1 = j1 + 1 < J ? (j1 + 1) * NS + tid : tid + 1;
            const float4 akv = s_ak[q * NTP + tid];  // (-a, -a', p lo, p lo')
            const ff2 x = {f2(o0 ? s_xh[i0] : 0.f, o1 ? s_xh[i1] : 0.f),
                           f2(o0 ? s_xl[i0] : 0.f, o1 ? s_xl[i1] : 0.f)};
            const ff2 xn = {f2(n0 ? s_xh[m0] : 0.f, n1 ? s_xh[m1] : 0.f),
                            f2(n0 ? s_xl[m0] : 0.f, n1 ? s_xl[m1] : 0.f)};
            const ff2 pv = {f2(o0 ? s_ph[i0] : 0.f, o1 ? s_ph[i1] : 0.f),
                            f2(o0 ? akv.z : 0.f, o1 ? akv.w : 0.f)};
            const float2 a = f2(o0 ? -akv.x : 0.f, o1 ? -akv.y : 0.f);
            // K: p^2 (with a mass m v^2, m from the kick as mass_weight)
            ff2 p2 = two_prod2(pv.hi, pv.hi);
            p2.lo = fma2(mul2(f2(2.0f, 2.0f), pv.hi), pv.lo, p2.lo);
            if (MASS) p2 = ff2_mul(p2, mass_weight2(kick2, s_dm[q * NTP + tid]));
            ff2_acc(K2, p2);
            // the statistics (stats_site)
            ff2_acc(sx2, x);
            ff2_acc(sxx2, ff2_mul(x, x));
            ff2_acc(sxn2, ff2_mul(x, xn));
            ff2_acc(sxl2, ff2_mul(x, ff2{f2(lr0.x, lr1.x), f2(lr0.y, lr1.y)}));
            ff2_acc(se2, ff2_mul_f(ff2_exp(ff2_sub(nmu, x), s_exptab), a));
        }
        acc.K = ff2_fold(K2);
        st.sx = ff2_fold(sx2);
        st.sxx = ff2_fold(sxx2);
        st.sxn = ff2_fold(sxn2);
        st.sxl = ff2_fold(sxl2);
        st.e = ff2_fold(se2);
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
    if (PERSIST) persist_record(S.partials, v, s_wrec);
    else if (LEV) segment_decisions_ff(A, v, s_wpf, s_wacc, &s_splitf);
    else segment_decisions_stats(A, v, s_wrec, s_wacc, s_splitrec, mt);
    __syncthreads();
    // a persistent chain writes every trajectory's end state as a proposal
    // into the other buffer and decides after its grid barrier
    const bool write_h = v.sid >= 0 && (PERSIST || v.g.split || s_wacc[v.g.warp0]);
    float2* hout = (PERSIST || v.g.split) ? (v.cur ? A.h0f : A.h1f) : (v.cur ? A.h1f : A.h0f);
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
    if (!PERSIST && v.g.split) {
        if (LEV) finish_split_ff(A, v, s_splitf, &s_flag);
        else finish_split_stats(A, v, s_splitrec, &s_flag, s_wrec[0], s_mt[v.g.warp0]);
    }
}

}  // namespace
}  // namespace rsv
