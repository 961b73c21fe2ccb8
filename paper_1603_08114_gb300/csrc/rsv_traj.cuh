// rsv_traj.cuh -- the trajectory kernels and their work plan (host side).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {

// A molecular-dynamics integrator as a symmetric composition: per step
// drift a[0] dtau, then nk times {kick b[k] dtau; drift a[k+1] dtau}
// (h += c dtau p/m, p -= c dtau dS/dh).  integrator 0: the leapfrog of
// eqs. (6)-(8) (a = 1/2, 1/2; b = 1); 1: the second-order minimum-norm scheme
// of Omelyan, Mryglod and Folk (a = lambda, 1 - 2 lambda, lambda; b = 1/2,
// 1/2); 2: their fourth-order minimum-norm scheme without force gradients
// (a = xi, chi, 1 - 2 (chi + xi), chi, xi; b = (1 - 2 l)/2, l, l, (1 - 2 l)/2).
struct Scheme {
    int nk;          // force evaluations (kicks) per step
    double a[5];     // drifts
    double b[4];     // kicks
};
inline Scheme make_scheme(int integrator, double lambda)
{
    Scheme s{};
    if (integrator == 2) {
        const double xi = 0.1786178958448091, l = -0.2123418310626054,
                     chi = -0.06626458266981849;
        s.nk = 4;
        s.a[0] = xi; s.a[1] = chi; s.a[2] = 1.0 - 2.0 * (chi + xi); s.a[3] = chi; s.a[4] = xi;
        s.b[0] = 0.5 * (1.0 - 2.0 * l); s.b[1] = l; s.b[2] = l; s.b[3] = 0.5 * (1.0 - 2.0 * l);
    } else if (integrator == 1) {
        s.nk = 2;
        s.a[0] = lambda; s.a[1] = 1.0 - 2.0 * lambda; s.a[2] = lambda;
        s.b[0] = 0.5; s.b[1] = 0.5;
    } else {
        s.nk = 1;
        s.a[0] = 0.5; s.a[1] = 0.5;
        s.b[0] = 1.0;
    }
    return s;
}

// The mixed kernel's FP32 form of a Scheme (prepared on the host): the two
// end drifts of consecutive steps merged, the trajectory is a first drift
// r_first dtau and n_md nk substeps {kick; drift}: substep k kicks by
// kq[k % nk] (kick = kq[0]; kr = kq / kick) and drifts by r[k % nk] dtau, the
// last one by r_last dtau.  kv: the kick sizes differ within a step.
struct MixedScheme {
    float dt, kick, kq[4], kr[4], r[4], r_last, r_first;
    int nk;
    bool kv;
};
inline MixedScheme make_mixed_scheme(int integrator, double lambda, double dtau)
{
    MixedScheme m{};
    const Scheme s = make_scheme(integrator, lambda);
    m.dt = (float)dtau;
    m.nk = s.nk;
    if (integrator == 1) {  // the same FP32 values as 2 kicks of dt/2
        const float lam = (float)lambda;
        m.kq[0] = m.kq[1] = 0.5f * m.dt;
        m.r[0] = 1.0f - 2.0f * lam;
        m.r[1] = 2.0f * lam;
        m.r_last = m.r_first = lam;
    } else if (integrator == 2) {
        for (int k = 0; k < 4; ++k) {
            m.kq[k] = (float)s.b[k] * m.dt;
            m.r[k] = k + 1 < s.nk ? (float)s.a[k + 1] : (float)(s.a[s.nk] + s.a[0]);
        }
        m.r_last = (float)s.a[s.nk];
        m.r_first = (float)s.a[0];
    } else {
        m.kq[0] = m.dt;
        m.r[0] = 1.0f;
        m.r_last = m.r_first = 0.5f;
    }
    m.kick = m.kq[0];
    for (int k = 0; k < 4; ++k) m.kr[k] = k < s.nk ? m.kq[k] / m.kick : 1.0f;
    m.kv = integrator == 2;
    return m;
}

// One contiguous run of one series inside one bin (a block's register window).
// A bin holds either several whole series side by side (each on whole warps),
// or one tile of a series too long for a window.  A tile integrates the window
// [wlo, whi) = its owned sites [lo, hi) widened by K = n_md + 1 sites on both
// sides (wlo rounded down to a multiple of 4), so that its owned sites and the
// right neighbour that dH needs are exact after n_md steps with no exchange
// between tiles.  Indices are series-local.
struct Seg {
    int64_t lo, hi;    // owned sites
    int64_t wlo, whi;  // integrated window
    int series;
    int warp0, nwarp;  // placement in the bin
    int split;         // 1: one tile of a series spread over several bins
};

struct SerInfo {
    int64_t off;  // first index of the series in the packed arrays
    int64_t T;
    int nseg;     // tiles of a split series (1 for a whole series)
    int seg0;     // segment id of its first tile (tiles have consecutive ids)
};

// Kernel configuration and the device copy of a plan.
struct Plan {
    int nt = 0, j = 0;          // threads per block, sites per thread
    int nbins = 0, grid = 0;
    size_t smem = 0;
    int64_t nsegs = 0;          // partials are indexed by segment id
    int nseries = 0;
    int nsplit = 0;             // series spread over several bins
    int64_t total = 0;          // packed length
    // device arrays (owned by the plan)
    Seg* d_segs = nullptr;
    int* d_bin_first = nullptr;  // [nbins + 1]
    int* d_bin_seg = nullptr;    // segment ids, bin-major
    SerInfo* d_ser = nullptr;
    int n_md = 0;
    int integrator = 0;         // 0 leapfrog, 1 and 2 minimum-norm (2 and 4 forces per step)
    double lambda = 0.0;        // of the second-order minimum-norm integrator
    bool mixed = false, mass = false;
    bool lev = false;           // RSV model with leverage (rho != 0)
};

// theta-derived constants of one series in FP32 / double-float for the mixed
// path, 32 floats per series.  The FP64 pipe of this GPU runs at 1/64 of the
// FP32 rate and every FP64 instruction occupies it for the whole warp, even
// with one lane active, so these are derived once per series (mixed_theta, by
// a small kernel or the theta update) instead of inside the trajectory kernel.
//
// With leverage (rho != 0) B = 1/(s_eta^2 (1 - rho^2)) takes the place of
// 1/s_eta^2 in c0, c1 and he, and the force and dH need the extra constants
// below; with rho = 0 they reduce to the plain model's values.
struct MixedTheta {
    // leapfrog: phi, c0 = 1/s_u^2 + (1+phi^2) B, 1/s_u^2, 1/s_eta^2,
    // -mu log2 e; c1 = -phi B (the force's stencil weights)
    float phi, c0, iu, ie, cmu;
    ff mu, ximu, phi_ff, hu, he;  // dH: mu, xi + mu, phi, 1/(2 s_u^2), B/2
    float c1;
    // leverage: cst = -(1-phi^2) rho^2 B (first-site correction of the ghost
    // row), ia = 1/(1-rho^2) (y-term weight of sites with a successor), omr =
    // 1 - rho^2, rsb = B rho s_eta (per-site v = rsb y), ibf = 1/B,
    // st = (1-phi^2)(1-rho^2) (stationary term in units of B/2)
    float cst, ia, omr, rsb, ibf;
    ff st;
    float pad[9];
};
static_assert(sizeof(MixedTheta) == 128, "MixedTheta is 32 floats");
__device__ __forceinline__ MixedTheta mixed_theta(const ThetaD& th)
{
    MixedTheta m;
    const double omr = 1.0 - th.rho * th.rho;
    const double B = 1.0 / (th.se2 * omr);
    m.phi = (float)th.phi;
    m.c0 = (float)(1.0 / th.su2 + (1.0 + th.phi * th.phi) / (th.se2 * omr));
    m.c1 = (float)(-th.phi / (th.se2 * omr));
    m.iu = (float)(1.0 / th.su2);
    m.ie = (float)(1.0 / th.se2);
    m.cmu = (float)(-th.mu * 1.4426950408889634);  // exponent of e^{-mu}
    m.mu = ff_from_double(th.mu);
    m.ximu = ff_from_double(th.xi + th.mu);
    m.phi_ff = ff_from_double(th.phi);
    m.hu = ff_from_double(0.5 / th.su2);
    m.he = ff_from_double(0.5 / (th.se2 * omr));
    m.cst = (float)(-(1.0 - th.phi * th.phi) * th.rho * th.rho * B);
    m.ia = (float)(1.0 / omr);
    m.omr = (float)omr;
    m.rsb = (float)(B * th.rho * sqrt(th.se2));
    m.ibf = (float)(th.se2 * omr);
    m.st = ff_from_double((1.0 - th.phi * th.phi) * omr);
    for (int i = 0; i < 9; ++i) m.pad[i] = 0.f;
    return m;
}

// MixedTheta of an FP32-valued theta (rho = 0) in FP32 / double-float
// arithmetic: the constants the mixed theta update derives from the theta it
// draws, and the theta prep kernel from a theta whose components are all
// FP32 values, so that the same theta gives the same constants either way.
__device__ __forceinline__ MixedTheta mixed_theta_f(const float (&t)[5])
{
    const float phi = t[0], mu = t[1], xi = t[2], se2 = t[3], su2 = t[4];
    MixedTheta m;
    m.phi = phi;
    m.iu = 1.0f / su2;
    m.ie = 1.0f / se2;
    m.c0 = m.iu + (1.0f + phi * phi) * m.ie;
    m.c1 = -phi * m.ie;
    m.cmu = -mu * 1.4426950408889634f;
    m.mu = ff{mu, 0.0f};
    m.ximu = two_sum(xi, mu);
    m.phi_ff = ff{phi, 0.0f};
    // 1/(2 s^2) in double-float: quotient and its exact FMA residual
    const float hu = 0.5f / su2, he = 0.5f / se2;
    m.hu = ff{hu, fmaf(-hu, su2, 0.5f) / su2};
    m.he = ff{he, fmaf(-he, se2, 0.5f) / se2};
    // the leverage constants at rho = 0 (the theta update is for eqs. (1)-(3))
    m.cst = 0.0f;
    m.ia = 1.0f;
    m.omr = 1.0f;
    m.rsb = 0.0f;
    m.ibf = se2;
    m.st = ff_sub(ff{1.0f, 0.0f}, two_prod(phi, phi));
    for (int i = 0; i < 9; ++i) m.pad[i] = 0.f;
    return m;
}

// Statistics of a state that its energy under eqs. (1)-(3) needs (mixed path,
// model without leverage), centred at the mu they were taken at: with
// x = h - mu,
//   sx = sum x,  sxx = sum x^2,  sxn = sum_{t<T-1} x_t x_{t+1},
//   sxl = sum x lnRV,  e = sum (y^2/2) e^{-h},  x0 = x_0,  xT = x_{T-1},
// in double-float, over the sites a tile owns (x0 and xT from the tiles that
// own those sites, 0 in the others), so that the tiles of a series add up.
// Only the centre depends on theta: under another mu' the sums follow in
// closed form from x' = x + mu - mu' (with sl = sum lnRV of the series), and
// the measurement term sum (x - c')^2, c' = lnRV - xi - mu, from sxx, sxl, sx
// and data constants, so the energy of a stored state under a new theta needs
// no pass over its sites.
struct StateStats {
    ff sx, sxx, sxn, sxl, e, x0, xT;
};
// The statistics of one series' state with their centre mu (and xi + mu of
// the same theta), and the data sums sl = sum lnRV, sll = sum lnRV^2 over the
// series (which the theta update needs).
struct StatsRec {
    ff mu, ximu, sl, sll;
    StateStats s;
};
// double-float values per segment in TrajArgs::partials: a tile of a split
// series reports its kinetic-energy difference and its end state's
// statistics (kRecWords); the statistics kernel writes sl, the statistics and
// sll (kPartialWords)
constexpr int kRecWords = 8;
constexpr int kPartialWords = 9;

struct TrajArgs {
    const Seg* segs;
    const int* bin_first;
    const int* bin_seg;
    int nbins;
    const SerInfo* ser;
    // theta: device [nseries][5], or NULL to use th_inline for every series
    const double* theta;
    ThetaD th_inline;
    int* ser_cur;        // buffer selector per series (NULL: all 0)
    unsigned* ser_cnt;   // arrival counters of split series (zero between launches)
    double* partials;    // per segment id
    double* dH_out;      // per series
    int* acc_out;        // per series
    const double* log_u; // per series, or NULL (drawn from Philox)
    // state: FP64 double buffer (FP64 path) or (hi, lo) FP32 double buffer (mixed)
    double* h0d;
    double* h1d;
    float2* h0f;
    float2* h1f;
    const double* p_in;  // optional initial momenta (FP64, packed)
    double* p_out;       // optional p' (FP64, packed), must not alias p_in
    const double* y;     // FP64 path
    const double* lnrv;
    const float* a_f;    // mixed path: y^2/2 with the sign of y, and lnRV as (hi, lo)
    const float2* lr_f;
    const MixedTheta* theta_f;  // mixed path: per-series constants (launch_theta_prep)
    // mixed path without leverage: [nseries][2] statistics of the state in
    // each buffer (the one ser_cur selects must hold the current state's)
    StatsRec* rstats;
    // mixed path, optional: the state the trajectory starts from as FP32
    // (h hi + lo), written for the owned sites on the way in (the snapshot of
    // the previous trajectory)
    float* snap_prev;
    double rho;          // leverage corr(eps_t, eta_t) of every series (0: eqs. (1)-(3))
    const float* minv;   // optional inverse mass (FP32, packed)
    const int* mass_on;  // optional flag; 0 = use m = 1
    int n_md;
    int integrator;      // 0 leapfrog (eqs. (6)-(8)), 1 and 2 minimum-norm (see Scheme)
    double lambda;       // of the second-order minimum-norm integrator
    Scheme sch;          // make_scheme(integrator, lambda)
    MixedScheme msch;    // make_mixed_scheme(integrator, lambda, dtau)
    double dtau;
    uint64_t seed, traj;
    int* status;
    int* fb_state;       // [2] mass fallback window counters (single series)
    int fallback_window;
};

// Build a plan for the series with the given offsets (host, [n+1]).
// sched_nt / sched_j / sched_tile > 0 fix the tiling, 0 chooses it.
// Returns false (reason in *why) if no tiling fits.
// integrator / lambda: see Plan; the halo is n_md * (forces per step) + 1.
// chain: the plan of a series run as one persistent chain (its own block-shape
// preference).
bool make_plan(const int64_t* offsets, int n, int n_md, int integrator, double lambda, bool mixed,
               bool mass, bool lev, int num_sms, int sched_nt, int sched_j, int64_t sched_tile,
               Plan& plan, const char** why, bool chain = false);
void free_plan(Plan& plan);

cudaError_t launch_traj(const TrajArgs& a, const Plan& p, cudaStream_t st);
// theta_f[s] = mixed_theta(theta of series s, leverage rho) for n series
// (theta: device [n][5], or NULL for th_inline); also fills the device table
// of 2^(j/32).
cudaError_t launch_theta_prep(const double* theta, ThetaD th_inline, int n, double rho,
                              MixedTheta* theta_f, cudaStream_t st);
// Row stride (in floats) of the mixed kernel's state rows [j][.]: nt threads
// plus a pad of ceil(32 / j).  A warp files and reads its 32 j consecutive
// sites with consecutive lanes, so one instruction touches j slots of each of
// about 32 / j owner threads; with rows a multiple of 32 words apart those
// all fall in the owners' few banks (j-way conflicts), with the pad the slots
// of one owner land in different banks (2- to 3-way at most).
__host__ __device__ constexpr int mixed_row_pad(int j) { return (32 + j - 1) / j; }
__host__ __device__ constexpr int mixed_row(int nt, int j) { return nt + mixed_row_pad(j); }
// Row stride (in pair slots) of the mixed kernel's pair arrays (site
// constants, -kick/m, leverage v): the block, so that a warp's float4 row
// segment, which the leapfrog reads every step, is four whole 128-byte lines
// (rows one slot longer, against the load pass's store conflicts, made the
// leapfrog ~10 % slower).
__host__ __device__ constexpr int mixed_ntp(int nt) { return nt; }
// Largest block (threads) of the mixed kernel with `j` sites per thread, with
// or without a mass (0 if j is not instantiated).
int mixed_max_threads(int j, bool mass);
// Resident blocks per SM of a trajectory kernel configuration (0 if invalid).
int blocks_per_sm(bool mixed, bool mass, bool lev, int j, int nt, size_t smem);

// rstats[s][0] = the statistics of series s in the (hi, lo) state hf, for
// every series of a mixed plan (scratch: kPartialWords doubles per segment).
cudaError_t launch_state_stats(const Plan& p, const float2* hf, const float* a_f,
                               const float2* lr_f, const MixedTheta* theta_f, double* scratch,
                               StatsRec* rstats, cudaStream_t st);

cudaError_t launch_commit_fp64(double* h, const double* hprop, double* p, const double* pprop,
                               const int* acc, int64_t T, cudaStream_t st);
cudaError_t launch_prep_mixed(const double* y, const double* lnrv, float* a_f, float2* lr_f,
                              int64_t T, cudaStream_t st);
cudaError_t launch_h_to_ff(const double* h, float2* hf, int64_t T, cudaStream_t st);
// Write the current state of every series into h (packed FP64): FP64 path
// from h1d where cur[s] = 1 (h0d is h itself); mixed path from the (hi, lo)
// buffer cur[s], restricted to series with acc[s] = 1 when acc != NULL.
cudaError_t launch_finalize(const Plan& p, const int* cur, const int* acc, const double* h1d,
                            const float2* h0f, const float2* h1f, double* h, cudaStream_t st);
cudaError_t launch_snapshot(const Plan& p, const int* cur, const double* h0d, const double* h1d,
                            const float2* h0f, const float2* h1f, float* out, cudaStream_t st);

}  // namespace rsv
