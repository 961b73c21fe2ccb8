// rsv_api_hmc.cu -- entry points of the HMC update: one trajectory, chains and
// batches of independent series (declared in include/rsv.h).
//
// All three run the same persistent trajectory kernel of rsv_traj.cu on a plan
// (rsv_plan.cu); this file checks arguments, keeps the workspace and orders the
// launches on the caller's stream.
#include <cmath>
#include <cstring>

#include "rsv.h"
#include "rsv_api_common.cuh"
#include "rsv_chain.cuh"
#include "rsv_ctx.cuh"
#include "rsv_gibbs.cuh"
#include "rsv_traj.cuh"

using namespace rsv;

namespace rsv {
namespace {

// Launch a trajectory kernel, bracketed by CUDA events when timing is on.
cudaError_t timed_traj(rsv_ctx* c, const TrajArgs& a, const Plan& p, cudaStream_t s)
{
    const bool rec = c->timing && !capture_active();
    if (rec) {
        if (c->ev_used + 2 > c->ev.size()) {
            for (int i = 0; i < 2; ++i) {
                cudaEvent_t e;
                cudaError_t r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
                c->ev.push_back(e);
            }
        }
        cudaEventRecord(c->ev[c->ev_used], s);
    }
    cudaError_t e = launch_traj(a, p, s);
    if (rec) {
        cudaEventRecord(c->ev[c->ev_used + 1], s);
        c->ev_used += 2;
    }
    c->launches += 1;
    c->traj_launches += 1;
    return e;
}

// Single-series plan from the context cache.  chain: the plan of an
// rsv_hmc_chain call that can run as one persistent launch (its own block
// shape preference).
rsv_status single_plan(rsv_ctx* c, int64_t T, int n_md, bool mixed, bool mass, const Plan** out,
                       bool chain = false)
{
    for (auto& e : c->plans) {
        if (e.T == T && e.n_md == n_md && e.mixed == mixed && e.mass == mass &&
            e.lev == (c->rho != 0.0) && e.integrator == c->integrator && e.lambda == c->lambda &&
            e.nt == c->sched_nt && e.j == c->sched_j && e.tile == c->sched_tile &&
            e.chain == chain) {
            *out = &e.plan;
            return RSV_OK;
        }
    }
    if (capture_active())
        return fail(RSV_EINVAL, "a new plan is needed during stream capture; run the call once "
                                "before capturing");
    if (c->plans.size() >= 8) {
        free_plan(c->plans.front().plan);
        c->plans.erase(c->plans.begin());
    }
    const int64_t off[2] = {0, T};
    const bool lev = c->rho != 0.0;
    rsv_ctx::Cached e{T,   n_md, c->integrator, c->lambda,  mixed,         mass, lev,
                      c->sched_nt, c->sched_j, c->sched_tile, chain, Plan()};
    const char* why = "";
    if (!make_plan(off, 1, n_md, c->integrator, c->lambda, mixed, mass, lev, c->num_sms,
                   c->sched_nt, c->sched_j, c->sched_tile, e.plan, &why, chain))
        return fail(RSV_EINVAL, "%s", why);
    c->plans.push_back(e);
    *out = &c->plans.back().plan;
    return RSV_OK;
}

// Workspace for a plan: partials per segment, per-series selectors, counters
// and scratch outputs, state buffers.
rsv_status ensure_plan_ws(rsv_ctx* c, const Plan& p, bool mixed, bool need_p)
{
    rsv_status st;
    const size_t N = (size_t)p.total, n = (size_t)p.nseries;
    if ((st = ctx_ensure_partials(c, p.nsegs)) != RSV_OK) return st;
    if ((st = c->ser_cur.ensure(n * sizeof(int))) != RSV_OK) return st;
    if ((st = c->ser_cnt.ensure(n * sizeof(unsigned))) != RSV_OK) return st;
    if ((st = c->ser_dh.ensure(n * sizeof(double))) != RSV_OK) return st;
    if ((st = c->ser_acc.ensure(n * sizeof(int))) != RSV_OK) return st;
    if (need_p && (st = c->dbuf1.ensure(N * 8)) != RSV_OK) return st;
    if (mixed) {
        if ((st = c->fbuf0.ensure(N * 8)) != RSV_OK) return st;
        if ((st = c->fbuf1.ensure(N * 8)) != RSV_OK) return st;
        if ((st = c->a_f.ensure(N * 4)) != RSV_OK) return st;
        if ((st = c->lr_f.ensure(N * 8)) != RSV_OK) return st;
        if ((st = c->theta_f.ensure(n * sizeof(MixedTheta))) != RSV_OK) return st;
        if ((st = c->rstats.ensure(n * 2 * sizeof(StatsRec))) != RSV_OK) return st;
    } else {
        if ((st = c->dbuf0.ensure(N * 8)) != RSV_OK) return st;
    }
    return RSV_OK;
}

struct RunOpts {
    double* h;
    double* p;  // explicit momenta (n_traj = 1) or NULL
    const double* y;
    const double* lnrv;
    const double* theta;  // device [n][5] or NULL -> th_inline
    ThetaD th_inline;
    const float* minv;
    double dtau;
    uint64_t seed, traj0;
    int64_t n_traj;
    const double* log_u;
    double* dH_out;  // [n_traj][n] or NULL
    int* acc_out;
    // chain extras (single series)
    int update_theta;
    double* theta_out;
    float* snaps;
    int64_t thin;
    int fallback_window;
    int* mass_used_out;
    bool commit_only_accepted;  // mixed: write back only accepted series
    bool chain;                 // rsv_hmc_chain (may run as one persistent launch)
};

// Trajectories per persistent launch at most: the grid barrier's counter
// reaches trajectories x blocks (< 2^32).
constexpr int64_t kChainMaxTraj = int64_t(1) << 24;

// The whole chain in one persistent cooperative launch (rsv_chain.cu), if the
// plan supports it and its blocks fit on the GPU at once; *done tells.
rsv_status run_persistent(rsv_ctx* c, const Plan& P, const RunOpts& o, const TrajArgs& a,
                          cudaStream_t s, bool* done)
{
    *done = false;
    rsv_status st;
    if ((st = ctx_ensure_partials(c, 2 * P.nsegs)) != RSV_OK) return st;
    int* ints = c->ints.as<int>();
    cudaError_t e = cudaMemsetAsync(ints + kChainBarrier, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "barrier reset");
    ChainArgs ch;
    memset(&ch, 0, sizeof(ch));
    ch.A = a;
    ch.A.ser_cur = nullptr;   // the kernel keeps the current buffer itself
    ch.A.theta = nullptr;
    ch.A.dH_out = nullptr;
    ch.A.acc_out = nullptr;
    ch.A.fb_state = nullptr;
    ch.A.snap_prev = nullptr;
    ch.A.traj = o.traj0;
    ch.n_traj = o.n_traj;
    ch.traj0 = o.traj0;
    ch.update_theta = o.update_theta;
    ch.theta = const_cast<double*>(o.theta);
    ch.theta_out = o.theta_out;
    ch.snaps = o.snaps;
    ch.thin = o.thin > 0 ? o.thin : 1;
    ch.dH_out = o.dH_out;
    ch.acc_out = o.acc_out;
    ch.partials = c->partials.as<double>();
    ch.nsegs = P.nsegs;
    ch.bar = reinterpret_cast<unsigned*>(ints + kChainBarrier);
    ch.wait_limit = c->wait_limit;
    ch.fallback_window = o.minv ? o.fallback_window : 0;
    ch.mass_on_out = ints + kMassOn;
    ch.ser_cur_out = c->ser_cur.as<int>();
    const bool rec = c->timing && !capture_active();
    if (rec && c->ev_used + 2 > c->ev.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t ev;
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "event");
            c->ev.push_back(ev);
        }
    }
    if (rec) cudaEventRecord(c->ev[c->ev_used], s);
    bool launched = false;
    e = launch_chain(ch, P, c->num_sms, s, &launched);
    if (e != cudaSuccess) return cuda_fail(e, "persistent chain kernel");
    if (!launched) return RSV_OK;
    if (rec) {
        cudaEventRecord(c->ev[c->ev_used + 1], s);
        c->ev_used += 2;
    }
    c->launches += 1;
    c->traj_launches += o.n_traj;  // the timed launch covers n_traj trajectories
    *done = true;
    return RSV_OK;
}

rsv_status run(rsv_ctx* c, const Plan& P, const RunOpts& o, cudaStream_t s)
{
    const bool mixed = P.mixed, mass = P.mass;
    const size_t N = (size_t)P.total;
    rsv_status st;
    if ((st = ensure_plan_ws(c, P, mixed, o.p != nullptr)) != RSV_OK) return st;
    if (o.update_theta &&
        (st = c->gibbs.ensure((size_t)gibbs_grid(P.total) * 8 * sizeof(double))) != RSV_OK)
        return st;
    int* ints = c->ints.as<int>();
    cudaError_t e;
    const size_t n = (size_t)P.nseries;
    if ((e = cudaMemsetAsync(c->ser_cur.ptr, 0, n * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->ser_cnt.ptr, 0, n * sizeof(unsigned), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(ints + kFbState, 0, 2 * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(ints + kMassOn, 0, sizeof(int), s)) != cudaSuccess)
        return cuda_fail(e, "workspace reset");
    if (mass && (e = cudaMemsetAsync(ints + kMassOn, 0x01, 1, s)) != cudaSuccess)
        return cuda_fail(e, "workspace reset");

    TrajArgs a;
    memset(&a, 0, sizeof(a));
    a.segs = P.d_segs;
    a.bin_first = P.d_bin_first;
    a.bin_seg = P.d_bin_seg;
    a.nbins = P.nbins;
    a.ser = P.d_ser;
    a.theta = o.theta;
    a.th_inline = o.th_inline;
    a.ser_cur = c->ser_cur.as<int>();
    a.ser_cnt = c->ser_cnt.as<unsigned>();
    a.partials = c->partials.as<double>();
    a.log_u = o.log_u;
    a.p_in = o.p;
    a.p_out = o.p ? c->dbuf1.as<double>() : nullptr;
    a.y = o.y;
    a.lnrv = o.lnrv;
    a.minv = o.minv;
    a.mass_on = ints + kMassOn;
    a.n_md = P.n_md;
    a.integrator = P.integrator;
    a.lambda = P.lambda;
    a.sch = make_scheme(P.integrator, P.lambda);
    a.msch = make_mixed_scheme(P.integrator, P.lambda, o.dtau);
    a.rho = c->rho;
    a.dtau = o.dtau;
    a.seed = o.seed;
    a.status = ints + kStatus;
    a.fb_state = (o.fallback_window > 0 && P.nseries == 1) ? ints + kFbState : nullptr;
    a.fallback_window = o.fallback_window;
    if (mixed) {
        a.a_f = c->a_f.as<float>();
        a.lr_f = c->lr_f.as<float2>();
        a.h0f = c->fbuf0.as<float2>();
        a.h1f = c->fbuf1.as<float2>();
        a.theta_f = c->theta_f.as<MixedTheta>();
        if ((e = counted(c, launch_theta_prep, o.theta, o.th_inline, (int)n, c->rho,
                         c->theta_f.as<MixedTheta>(), s)) != cudaSuccess)
            return cuda_fail(e, "theta prep kernel");
        if ((e = counted(c, launch_prep_mixed, o.y, o.lnrv, c->a_f.as<float>(),
                         c->lr_f.as<float2>(), P.total, s)) != cudaSuccess)
            return cuda_fail(e, "prep kernel");
        if ((e = counted(c, launch_h_to_ff, (const double*)o.h, c->fbuf0.as<float2>(), P.total,
                         s)) != cudaSuccess)
            return cuda_fail(e, "state split kernel");
        // without leverage dH takes the start's potential energy from the
        // statistics of the state; the kernel keeps them for both buffers
        a.rstats = c->rstats.as<StatsRec>();
        if (!P.lev) {
            c->launches += 1;  // two kernels
            if ((e = counted(c, launch_state_stats, P, (const float2*)c->fbuf0.as<float2>(),
                             (const float*)c->a_f.as<float>(),
                             (const float2*)c->lr_f.as<float2>(),
                             (const MixedTheta*)c->theta_f.as<MixedTheta>(),
                             c->partials.as<double>(), c->rstats.as<StatsRec>(), s)) != cudaSuccess)
                return cuda_fail(e, "state statistics kernels");
        }
    } else {
        a.h0d = o.h;
        a.h1d = c->dbuf0.as<double>();
    }
    // a mixed chain of one series without leverage: the whole chain in one
    // persistent launch when it can be
    bool done = false;
    if (mixed && !P.lev && o.chain && c->persistent && !o.p && !o.log_u && o.n_traj > 0 &&
        o.n_traj <= kChainMaxTraj && chain_supported(P) && !capture_active()) {
        if ((st = run_persistent(c, P, o, a, s, &done)) != RSV_OK) return st;
    }
    // mixed path: a snapshot that is due is written by the next trajectory's
    // load pass (its start state is that state), the last one by its own kernel
    float* pending_snap = nullptr;
    for (int64_t i = 0; !done && i < o.n_traj; ++i) {
        a.traj = o.traj0 + (uint64_t)i;
        a.dH_out = o.dH_out ? o.dH_out + i * (int64_t)n : c->ser_dh.as<double>();
        a.acc_out = o.acc_out ? o.acc_out + i * (int64_t)n : c->ser_acc.as<int>();
        a.snap_prev = pending_snap;
        pending_snap = nullptr;
        if ((e = timed_traj(c, a, P, s)) != cudaSuccess) return cuda_fail(e, "trajectory kernel");
        const bool snap_due = o.snaps && (i + 1) % o.thin == 0;
        float* snap_dst = snap_due ? o.snaps + (size_t)((i + 1) / o.thin - 1) * N : nullptr;
        bool snap_done = false;
        if (o.update_theta) {
            GibbsArgs g;
            memset(&g, 0, sizeof(g));
            g.h0d = a.h0d;
            g.h1d = a.h1d;
            g.h0f = a.h0f;
            g.h1f = a.h1f;
            g.cur = a.ser_cur;
            g.lnrv = o.lnrv;
            g.lr_f = a.lr_f;
            g.T = P.total;
            g.theta = const_cast<double*>(o.theta);
            g.theta_out = o.theta_out ? o.theta_out + 5 * i : nullptr;
            g.seed = o.seed;
            g.series = 0;
            g.traj = a.traj;
            g.mask = 31;
            g.partials = c->gibbs.as<double>();
            g.counter = reinterpret_cast<unsigned*>(ints + kGibbsCounter);
            g.theta_f = mixed ? c->theta_f.as<MixedTheta>() : nullptr;
            // mixed, no leverage: the sweep's sums come from the state's
            // statistics, which the trajectory kernel keeps
            g.rstats = (mixed && !P.lev) ? c->rstats.as<StatsRec>() : nullptr;
            // otherwise the mixed sweep reads every site of the new state: it
            // writes this trajectory's snapshot on the way (single series: the
            // packed state is the series)
            if (mixed && !g.rstats && snap_due && P.nseries == 1) {
                g.snap_out = snap_dst;
                snap_done = true;
            }
            if ((e = counted(c, launch_gibbs, g, mixed, s)) != cudaSuccess)
                return cuda_fail(e, "theta kernel");
        } else if (o.theta_out) {
            if ((e = cudaMemcpyAsync(o.theta_out + 5 * i, o.theta, 5 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return cuda_fail(e, "theta record");
        }
        if (snap_due && !snap_done && mixed && i + 1 < o.n_traj) {
            pending_snap = snap_dst;
            snap_done = true;
        }
        if (snap_due && !snap_done) {
            if ((e = counted(c, launch_snapshot, P, (const int*)a.ser_cur, (const double*)a.h0d,
                             (const double*)a.h1d, (const float2*)a.h0f, (const float2*)a.h1f,
                             snap_dst, s)) != cudaSuccess)
                return cuda_fail(e, "snapshot kernel");
        }
    }
    // the current state of every series back into h
    const int* accp = (mixed && o.commit_only_accepted) ? a.acc_out : nullptr;
    if ((e = counted(c, launch_finalize, P, (const int*)a.ser_cur, accp, (const double*)a.h1d,
                     (const float2*)a.h0f, (const float2*)a.h1f, o.h, s)) != cudaSuccess)
        return cuda_fail(e, "state copy kernel");
    if (o.p && (e = counted(c, launch_commit_fp64, (double*)nullptr, (const double*)nullptr, o.p,
                            (const double*)c->dbuf1.as<double>(), (const int*)a.acc_out,
                            P.total, s)) != cudaSuccess)
        return cuda_fail(e, "momentum copy kernel");
    if (o.mass_used_out &&
        (e = cudaMemcpyAsync(o.mass_used_out, ints + kMassOn, sizeof(int),
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "mass flag copy");
    return RSV_OK;
}

rsv_status check_common(int n_md, double dtau, rsv_precision prec)
{
    if (n_md < 1 || n_md > (1 << 20)) return fail(RSV_EINVAL, "n_md out of range");
    if (!(dtau > 0.0) || !std::isfinite(dtau)) return fail(RSV_EINVAL, "dtau must be > 0");
    if (prec != RSV_FP64 && prec != RSV_MIXED) return fail(RSV_EINVAL, "bad precision");
    return RSV_OK;
}

}  // namespace
}  // namespace rsv

extern "C" {

rsv_status rsv_hmc_trajectory(rsv_ctx* c, double* h, double* p, const double* y,
                              const double* lnrv, int64_t T, rsv_theta theta, const float* minv,
                              int n_md, double dtau, rsv_precision prec, uint64_t seed,
                              uint64_t traj, const double* log_u, double* dH_out,
                              int32_t* accept_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!h || !y || !lnrv || !dH_out || !accept_out) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    if ((st = check_common(n_md, dtau, prec)) != RSV_OK) return st;
    const Plan* P = nullptr;
    if ((st = single_plan(c, T, n_md, prec == RSV_MIXED, minv != nullptr, &P)) != RSV_OK) return st;
    RunOpts o;
    memset(&o, 0, sizeof(o));
    o.h = h;
    o.p = p;
    o.y = y;
    o.lnrv = lnrv;
    o.theta = nullptr;
    o.th_inline = to_dev(theta);
    o.minv = minv;
    o.dtau = dtau;
    o.seed = seed;
    o.traj0 = traj;
    o.n_traj = 1;
    o.log_u = log_u;
    o.dH_out = dH_out;
    o.acc_out = accept_out;
    o.commit_only_accepted = true;
    return run(c, *P, o, (cudaStream_t)stream);
}

rsv_status rsv_hmc_chain(rsv_ctx* c, double* h, const double* y, const double* lnrv, int64_t T,
                         double* theta, const float* minv, int n_md, double dtau,
                         rsv_precision prec, uint64_t seed, uint64_t traj0, int64_t n_traj,
                         int update_theta, double* dH_out, int32_t* accept_out,
                         double* theta_out, float* snaps, int64_t thin, int fallback_window,
                         int32_t* mass_used_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!h || !y || !lnrv || !theta) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    if ((st = check_common(n_md, dtau, prec)) != RSV_OK) return st;
    if (n_traj < 0) return fail(RSV_EINVAL, "n_traj must be >= 0");
    if (snaps && thin < 1) return fail(RSV_EINVAL, "thin must be >= 1 with snapshots");
    if (fallback_window < 0) return fail(RSV_EINVAL, "fallback_window must be >= 0");
    if (update_theta && c->rho != 0.0)
        return fail(RSV_EINVAL, "the theta update is for the model without leverage (rho = 0)");
    const Plan* P = nullptr;
    const bool chain = prec == RSV_MIXED && c->rho == 0.0 && c->persistent;
    if ((st = single_plan(c, T, n_md, prec == RSV_MIXED, minv != nullptr, &P, chain)) != RSV_OK)
        return st;
    RunOpts o;
    memset(&o, 0, sizeof(o));
    o.h = h;
    o.y = y;
    o.lnrv = lnrv;
    o.theta = theta;
    o.minv = minv;
    o.dtau = dtau;
    o.seed = seed;
    o.traj0 = traj0;
    o.n_traj = n_traj;
    o.dH_out = dH_out;
    o.acc_out = accept_out;
    o.update_theta = update_theta;
    o.theta_out = theta_out;
    o.snaps = snaps;
    o.thin = thin;
    o.fallback_window = fallback_window;
    o.mass_used_out = mass_used_out;
    o.commit_only_accepted = false;
    o.chain = true;
    return run(c, *P, o, (cudaStream_t)stream);
}

rsv_status rsv_chain_schedule(rsv_ctx* c, int64_t T, int n_md, rsv_precision prec, int with_mass,
                              int* threads, int* sites_per_thread, int64_t* tile, int* persistent)
{
    rsv_status st = ctx_begin(c, nullptr);
    if (st != RSV_OK) return st;
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    if ((st = check_common(n_md, 1.0, prec)) != RSV_OK) return st;
    const bool chain = prec == RSV_MIXED && c->rho == 0.0 && c->persistent;
    const Plan* P = nullptr;
    if ((st = single_plan(c, T, n_md, prec == RSV_MIXED, with_mass != 0, &P, chain)) != RSV_OK)
        return st;
    bool fits = false;
    if (chain) {
        cudaError_t e = chain_fits(*P, c->num_sms, &fits);
        if (e != cudaSuccess) return cuda_fail(e, "chain occupancy");
    }
    if (threads) *threads = P->nt;
    if (sites_per_thread) *sites_per_thread = P->j;
    if (tile) {  // the owned sites of a tile (the series itself when it is not cut)
        const int64_t K = (int64_t)n_md * make_scheme(P->integrator, P->lambda).nk + 1;
        const int64_t t = c->sched_nt > 0 ? c->sched_tile : (int64_t)P->nt * P->j - 2 * K - 3;
        *tile = P->nbins > 1 ? t : T;
    }
    if (persistent) *persistent = fits ? 1 : 0;
    return RSV_OK;
}

rsv_status rsv_plan_create(rsv_ctx* c, const int64_t* offsets, int64_t n_series, int n_md,
                           rsv_precision prec, int with_mass, rsv_plan** out)
{
    rsv_status st = ctx_begin(c, nullptr);
    if (st != RSV_OK) return st;
    if (!offsets || !out) return fail(RSV_EINVAL, "null argument");
    *out = nullptr;
    if (n_series < 1 || n_series > (1LL << 30)) return fail(RSV_EINVAL, "n_series out of range");
    if (offsets[0] != 0) return fail(RSV_EINVAL, "offsets[0] must be 0");
    for (int64_t s = 0; s < n_series; ++s)
        if (offsets[s + 1] <= offsets[s]) return fail(RSV_EINVAL, "series %lld is empty", (long long)s);
    if ((st = check_common(n_md, 1.0, prec)) != RSV_OK) return st;
    rsv_plan* p = new rsv_plan();
    p->device = c->device;
    const char* why = "";
    if (!make_plan(offsets, (int)n_series, n_md, c->integrator, c->lambda, prec == RSV_MIXED,
                   with_mass != 0, c->rho != 0.0, c->num_sms, c->sched_nt, c->sched_j,
                   c->sched_tile, p->plan, &why)) {
        delete p;
        return fail(RSV_EINVAL, "%s", why);
    }
    *out = p;
    return RSV_OK;
}

void rsv_plan_destroy(rsv_plan* p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    free_plan(p->plan);
    delete p;
}

rsv_status rsv_plan_info(const rsv_plan* p, int* threads, int* sites_per_thread, int* bins,
                         int* grid, int* split_series)
{
    if (!p) return fail(RSV_EINVAL, "null plan");
    if (threads) *threads = p->plan.nt;
    if (sites_per_thread) *sites_per_thread = p->plan.j;
    if (bins) *bins = p->plan.nbins;
    if (grid) *grid = p->plan.grid;
    if (split_series) *split_series = p->plan.nsplit;
    return RSV_OK;
}

rsv_status rsv_hmc_batched(rsv_ctx* c, rsv_plan* plan, double* h, double* p, const double* y,
                           const double* lnrv, const double* theta, const float* minv,
                           double dtau, uint64_t seed, uint64_t traj0, int64_t n_traj,
                           const double* log_u, double* dH_out, int32_t* accept_out,
                           void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!plan || !h || !y || !lnrv || !theta) return fail(RSV_EINVAL, "null argument");
    if (plan->device != c->device) return fail(RSV_EINVAL, "plan made for another device");
    if (!(dtau > 0.0) || !std::isfinite(dtau)) return fail(RSV_EINVAL, "dtau must be > 0");
    if (n_traj < 0) return fail(RSV_EINVAL, "n_traj must be >= 0");
    if ((p || log_u) && n_traj != 1) return fail(RSV_EINVAL, "p and log_u need n_traj = 1");
    if ((minv != nullptr) != plan->plan.mass) return fail(RSV_EINVAL, "minv does not match the plan");
    if ((c->rho != 0.0) != plan->plan.lev)
        return fail(RSV_EINVAL, "the plan was made for another leverage setting");
    RunOpts o;
    memset(&o, 0, sizeof(o));
    o.h = h;
    o.p = p;
    o.y = y;
    o.lnrv = lnrv;
    o.theta = theta;
    o.minv = minv;
    o.dtau = dtau;
    o.seed = seed;
    o.traj0 = traj0;
    o.n_traj = n_traj;
    o.log_u = log_u;
    o.dH_out = dH_out;
    o.acc_out = accept_out;
    o.commit_only_accepted = n_traj == 1;
    return run(c, plan->plan, o, (cudaStream_t)stream);
}

}  // extern "C"
