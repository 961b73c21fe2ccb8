/*
 * rsv.h -- C ABI of librsv: the Hybrid Monte Carlo (HMC) volatility update of
 * the realized stochastic volatility (RSV) model on one NVIDIA GB300 (sm_103a).
 *
 * Method: T. Takaishi, "GPU Computing in Bayesian Inference of Realized
 * Stochastic Volatility Model", arXiv:1603.08114.
 *   model            eqs. (1)-(3)   y_t = e^{h_t/2} eps_t,  lnRV_t = xi + h_t + u_t,
 *                                   h_{t+1} = mu + phi (h_t - mu) + eta_t
 *   parameters       Sec. 2         theta = (phi, mu, xi, sigma_eta^2, sigma_u^2)
 *   Hamiltonian      Sec. 3         H(p, h) = 1/2 sum_t p_t^2 + S(h),  S = -ln f(h | theta)
 *   leapfrog         eqs. (6)-(8)   h += dtau/2 p;  p -= dtau dS/dh;  h += dtau/2 p
 *   trajectory       Sec. 3         k = n_md repetitions, length l = n_md * dtau
 *   Metropolis       Sec. 3         accept h' with probability min{1, e^{-dH}}
 * S(h) (the paper defers f to its ref. [RSV]) is, constants dropped,
 *   S = sum_t [h_t/2 + (y_t^2/2) e^{-h_t} + (lnRV_t - xi - h_t)^2/(2 sigma_u^2)]
 *     + (1 - phi^2)(h_1 - mu)^2/(2 sigma_eta^2)
 *     + sum_{t<T} (h_{t+1} - mu - phi (h_t - mu))^2/(2 sigma_eta^2).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers on the context's device, owned by the
 *    caller; the library never frees them.  Arrays are dense, 0-based, indexed
 *    by site t = 0..T-1 (the paper's t = 1..T).  Scalars marked "host" are host
 *    values.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream; outputs are valid after the stream
 *    is synchronised.
 *  - Arguments are checked before any launch; on RSV_EINVAL nothing is launched
 *    and no output is touched.  The library never aborts or traps.
 *  - Conditions found on the device (a non-finite dH, a wait that ran out of
 *    time) are recorded in a status word of the context and returned by
 *    rsv_sync_status().
 *  - rsv_last_error() gives a text for the last non-OK status of the calling
 *    thread.
 *  - A context is bound to one device and must not be used from two host
 *    threads at once.
 */
#ifndef RSV_H_
#define RSV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSV_ABI_VERSION 1

/* theta of Sec. 2.  Valid: |phi| < 1, sig_eta2 > 0, sig_u2 > 0, all finite. */
typedef struct rsv_theta {
    double phi, mu, xi, sig_eta2, sig_u2;
} rsv_theta;

typedef enum rsv_status {
    RSV_OK = 0,
    RSV_EINVAL = 1,       /* bad argument; nothing launched                     */
    RSV_ENOMEM = 2,       /* workspace allocation failed                        */
    RSV_ECUDA = 3,        /* a CUDA call failed (text in rsv_last_error)        */
    RSV_ENONFINITE = 4,   /* a dH was NaN/Inf; that trajectory was rejected     */
    RSV_ETIMEOUT = 5      /* a device-side wait gave up; results are invalid    */
} rsv_status;

/* RSV_FP64: every step in FP64.
 * RSV_MIXED: leapfrog force and updates in FP32 on a compensated (hi, lo)
 * FP32 state; dH in double-float: the kinetic energy at both ends per site
 * and, without leverage, the potential energy from double-float sums of the
 * state kept per series and buffer (with leverage, per site at both ends);
 * the Metropolis comparison decides as in FP64.  The theta-derived constants
 * are prepared in FP64, or in FP32 when every component of theta is an FP32
 * value (as the mixed theta update leaves it). */
typedef enum rsv_precision { RSV_FP64 = 0, RSV_MIXED = 1 } rsv_precision;

typedef struct rsv_ctx rsv_ctx;

/* ---- context --------------------------------------------------------------
 * rsv_create: bind a context to CUDA device `device` (makes it current).
 * Owns a small workspace (reduction partials, counters, a status word) that
 * grows on demand; rsv_reserve() grows it ahead of time so that later calls
 * allocate nothing (needed before CUDA-graph capture).
 * rsv_destroy: frees the workspace; NULL is a no-op. */
rsv_status rsv_create(rsv_ctx** ctx, int device);
void rsv_destroy(rsv_ctx* ctx);
rsv_status rsv_reserve(rsv_ctx* ctx, int64_t max_T, int64_t max_series);
const char* rsv_last_error(void);
int rsv_abi_version(void);
/* Synchronise `stream`, return and clear the device status word. */
rsv_status rsv_sync_status(rsv_ctx* ctx, void* stream);
/* Fix the tiling of single-series trajectories (rsv_hmc_trajectory,
 * rsv_hmc_chain) and of plans created afterwards: `threads` per block
 * (multiple of 32; <= 256 FP64, <= 384 mixed), `sites_per_thread` (FP64: 4, 8,
 * 16, 28; mixed: 4, 8, 16, 20) and `tile` owned sites per tile of a series cut
 * into tiles (tile + 2 (n_md + 1) + 3 <= threads * sites_per_thread, else the
 * call that uses it fails with RSV_EINVAL).  A single series no longer than
 * `tile` is kept whole (it then needs only T <= threads * sites_per_thread).
 * All zero restores the automatic plan.  Results depend on the tiling only
 * through rounding (the order of the sums). */
rsv_status rsv_set_schedule(rsv_ctx* ctx, int threads, int sites_per_thread, int64_t tile);
/* rsv_set_persistent: 1 (the default) runs an rsv_hmc_chain call in RSV_MIXED
 * precision on the model without leverage as ONE persistent cooperative
 * launch when the tiles of its plan can all be resident on the GPU at once
 * (else, or with 0, one trajectory kernel per trajectory and a theta-sweep
 * kernel after it).  Every tile stays on its SM for the whole chain; after
 * each trajectory one grid barrier, then every block sums all tiles' records
 * in the same order and takes the same Metropolis decision and theta sweep.
 * The results are bit for bit those of the per-trajectory launches. */
rsv_status rsv_set_persistent(rsv_ctx* ctx, int enable);
/* rsv_set_wait_limit: the clock cycles (per SM) a device-side wait of the
 * persistent chain may spin before it gives up: it then records a timeout,
 * which rsv_sync_status() returns as RSV_ETIMEOUT, and the kernel ends (the
 * chain's results are invalid; the context stays usable).  0 restores the
 * default, 2^31 cycles (about one second at 2 GHz); cycles < 0: RSV_EINVAL. */
rsv_status rsv_set_wait_limit(rsv_ctx* ctx, int64_t cycles);
/* rsv_chain_schedule: the block shape an rsv_hmc_chain call of this context
 * with these arguments uses (threads per block, sites per thread, and the
 * owned sites per tile: T when the series is not cut), and whether it runs as
 * one persistent launch (1) or one kernel per trajectory (0).  Builds and
 * caches the call's plan; any output may be NULL. */
rsv_status rsv_chain_schedule(rsv_ctx* ctx, int64_t T, int n_md, rsv_precision prec, int with_mass,
                              int* threads, int* sites_per_thread, int64_t* tile, int* persistent);

/* ---- integrator -------------------------------------------------------------
 * The molecular-dynamics integrator of the trajectories run afterwards through
 * this context (rsv_hmc_trajectory, rsv_hmc_chain) and of plans created
 * afterwards (a plan keeps the integrator it was made with):
 *  RSV_LEAPFROG  eqs. (6)-(8), one force evaluation per step (the default);
 *  RSV_OMELYAN2  the second-order minimum-norm integrator of Omelyan, Mryglod
 *                and Folk (Phys. Rev. E 65, 056706, 2002), one of the
 *                higher-order integrators Sec. 3 cites: per step
 *                h += lambda dtau p/m; p -= dtau/2 dS/dh; h += (1-2 lambda) dtau p/m;
 *                p -= dtau/2 dS/dh; h += lambda dtau p/m -- two force
 *                evaluations per step, an energy error far smaller than the
 *                leapfrog's at equal cost.  lambda <= 0 selects the minimum-norm
 *                value RSV_OMELYAN2_LAMBDA; lambda = 1/2 is the leapfrog with its
 *                force step split in two.
 * With RSV_OMELYAN2 a tile's halo and the `tile` bound of rsv_set_schedule
 * count 2 n_md force evaluations instead of n_md.  lambda > 1/2 or NaN gives
 * RSV_EINVAL (RSV_OMELYAN2 only). */
typedef enum rsv_integrator { RSV_LEAPFROG = 0, RSV_OMELYAN2 = 1, RSV_OMELYAN4 = 2 } rsv_integrator;
#define RSV_OMELYAN2_LAMBDA 0.19318332750378357
/* RSV_OMELYAN4: the fourth-order force-gradient-free integrator of Omelyan,
 * Mryglod and Folk (Comput. Phys. Commun. 146, 188, 2002), their minimum-norm
 * position-extended Forest-Ruth-like scheme: per step
 *   h += XI dtau p/m;  p -= (1 - 2 LAMBDA)/2 dtau dS/dh;  h += CHI dtau p/m;
 *   p -= LAMBDA dtau dS/dh;  h += (1 - 2 (CHI + XI)) dtau p/m;  p -= LAMBDA dtau dS/dh;
 *   h += CHI dtau p/m;  p -= (1 - 2 LAMBDA)/2 dtau dS/dh;  h += XI dtau p/m
 * with the constants below -- four force evaluations per step, energy error
 * O(dtau^4).  Its `lambda` argument is ignored; a tile's halo and the `tile`
 * bound of rsv_set_schedule count 4 n_md force evaluations. */
#define RSV_OMELYAN4_XI 0.1786178958448091
#define RSV_OMELYAN4_LAMBDA (-0.2123418310626054)
#define RSV_OMELYAN4_CHI (-0.06626458266981849)
rsv_status rsv_set_integrator(rsv_ctx* ctx, rsv_integrator kind, double lambda);

/* ---- model: leverage -------------------------------------------------------
 * The RSV model with leverage: eqs. (1)-(3) of Sec. 2 with corr(eps_t, eta_t)
 * = rho, the form of the RSV model in the reference the paper cites for it
 * (Takahashi, Omori and Watanabe, Comput. Stat. Data Anal. 53 (2009) 2404).
 * Given eps_t = y_t e^{-h_t/2}, eta_t is N(rho s_eta eps_t, s_eta^2 (1-rho^2)),
 * so the AR term of S becomes
 *   sum_{t<T} d_t^2 / (2 s_eta^2 (1 - rho^2)),
 *   d_t = h_{t+1} - mu - phi (h_t - mu) - rho s_eta y_t e^{-h_t/2},
 * and dS/dh follows term by term; the law of h_1 is unchanged.  rho applies to
 * every later rsv_action, rsv_force, rsv_hmc_trajectory and rsv_hmc_chain call
 * of this context, and to plans created afterwards (a plan made with rho = 0
 * cannot run with rho != 0 or the reverse: RSV_EINVAL).  rho = 0 restores
 * eqs. (1)-(3) exactly.  The theta update (rsv_gibbs_theta, update_theta of
 * rsv_hmc_chain) draws from the conditionals of the rho = 0 model and returns
 * RSV_EINVAL while rho != 0.  rsv_action_noalloc has no context and is always
 * the rho = 0 model.  |rho| >= 1 or NaN gives RSV_EINVAL. */
rsv_status rsv_set_leverage(rsv_ctx* ctx, double rho);

/* ---- S(h) -----------------------------------------------------------------
 * S(h) of Sec. 3 (see above), FP64, deterministic reduction order.
 * h, y, lnrv: [T] FP64.  S_out: device FP64 scalar.  T >= 1. */
rsv_status rsv_action(rsv_ctx* ctx, const double* h, const double* y, const double* lnrv,
                      int64_t T, rsv_theta theta, double* S_out, void* stream);

/* ---- S(h) without allocation ----------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: code running while a CUDA graph is being
 * captured (an allocation there is not part of the graph and breaks its
 * replay), plug-ins inside a host application that owns the device memory
 * pool, and real-time loops that must not wait on the allocator.
 * It computes the same S(h) as rsv_action, on the CURRENT device and without a
 * context.  Its scratch (one FP64 partial sum per block of 2048 sites and an
 * arrival counter, 33 KB) is a fixed array in device memory that every device
 * which loads the library holds until the process exits; nothing is allocated
 * or freed.  Limits and behaviour:
 *  - T must be 1 .. 8,388,608 (4096 blocks of 2048 sites); larger T returns
 *    RSV_EINVAL before any launch (use rsv_action).
 *  - The first call on a device looks up the array's device address (one-time
 *    set-up); make that first call before any stream capture.  The address
 *    is kept with the id of the device's context: after a cudaDeviceReset the
 *    next call looks it up again in the new context (so that call, too, must
 *    come before any capture).
 *  - All calls share the one array: calls that can overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 *    The arrival counter is cleared by each call before its launch.
 *  - Errors are returned as by rsv_action; rsv_last_error() gives the text. */
rsv_status rsv_action_noalloc(const double* h, const double* y, const double* lnrv, int64_t T,
                              rsv_theta theta, double* S_out, void* stream);

/* ---- dS/dh ----------------------------------------------------------------
 * F_t = dS/dh_t, the derivative in eq. (7):
 *   F_t = 1/2 - (y_t^2/2) e^{-h_t} - (lnRV_t - xi - h_t)/sigma_u^2 + AR_t,
 *   AR_t = [(1+phi^2) x_t - phi (x_{t-1} + x_{t+1})]/sigma_eta^2 inside,
 *   AR_0 = (x_0 - phi x_1)/sigma_eta^2, AR_{T-1} = (x_{T-1} - phi x_{T-2})/sigma_eta^2,
 *   AR_0 = (1 - phi^2) x_0/sigma_eta^2 if T = 1, with x_t = h_t - mu.
 * F_out: [T] FP64 (must not alias h). */
rsv_status rsv_force(rsv_ctx* ctx, const double* h, const double* y, const double* lnrv,
                     int64_t T, rsv_theta theta, double* F_out, void* stream);

/* ---- one HMC trajectory (Sec. 3) ------------------------------------------
 * n_md leapfrog steps of size dtau (eqs. (6)-(8)) from (h, p), then
 * dH = H(p', h') - H(p, h) and the Metropolis test: accept iff ln u < -dH
 * (a NaN dH rejects and sets RSV_ENONFINITE in the status word).
 *  h     [T] FP64 in/out: on accept h', else unchanged.
 *  p     [T] FP64 in/out or NULL.  Non-NULL: the initial momenta p, replaced
 *        by p' (the end of the trajectory, accepted or not).  NULL: momenta
 *        p_t ~ N(0, m_t) are drawn from Philox4x64-10 with key {seed, 0} and
 *        counter {t/4, traj, 0, 0}, Box-Muller on 53-bit (FP64) or 23-bit
 *        (MIXED, computed in FP32) uniforms (k + 1/2) 2^-bits from the top
 *        bits of each 64-bit word.
 *  minv  [T] FP32 inverse diagonal mass 1/m_t > 0, or NULL for m = 1.  With a
 *        mass, eq. (6) reads h += dtau/2 p/m and H = 1/2 sum p^2/m + S.
 *  log_u device FP64 scalar ln u, or NULL to draw u from Philox counter
 *        {0, traj, 1, 0} (53-bit uniform).
 *  dH_out device FP64 scalar; accept_out device int32 scalar (1 accepted).
 * Requires T >= 1, n_md >= 1, dtau > 0 finite. */
rsv_status rsv_hmc_trajectory(rsv_ctx* ctx, double* h, double* p, const double* y,
                              const double* lnrv, int64_t T, rsv_theta theta, const float* minv,
                              int n_md, double dtau, rsv_precision prec, uint64_t seed,
                              uint64_t traj, const double* log_u, double* dH_out,
                              int32_t* accept_out, void* stream);

/* ---- a chain of trajectories ----------------------------------------------
 * n_traj HMC trajectories (Sec. 3) with indices traj0 .. traj0+n_traj-1 and
 * Philox draws as in rsv_hmc_trajectory; if update_theta != 0 each trajectory
 * is followed by a Gibbs sweep of theta (xi, sigma_u^2, mu, sigma_eta^2, phi;
 * the paper does not describe its theta update) drawing from Philox counter
 * {block, traj, 2, 0}.
 *  h       [T] FP64 in/out: chain state.
 *  theta   device FP64 [5] = (phi, mu, xi, sigma_eta^2, sigma_u^2), in/out.
 *  dH_out, accept_out: device [n_traj] FP64 / int32, or NULL.
 *  theta_out: device [n_traj][5] FP64 (theta after each sweep), or NULL.
 *  snaps:  device FP32 [n_traj/thin][T]: h after every thin-th trajectory
 *          (thin >= 1), or NULL.
 *  fallback_window: if > 0 and minv != NULL, after every fallback_window
 *          trajectories the mass is switched to m = 1 for the rest of the
 *          call when that window's acceptance rate is below 0.6.
 *  mass_used_out: device int32 scalar (1 while the mass is in use), or NULL.
 * In RSV_MIXED precision on the model without leverage the whole call runs as
 * one persistent cooperative launch when the plan's tiles can all be resident
 * (see rsv_set_persistent, rsv_chain_schedule); the results equal those of
 * one launch per trajectory bit for bit. */
rsv_status rsv_hmc_chain(rsv_ctx* ctx, double* h, const double* y, const double* lnrv, int64_t T,
                         double* theta, const float* minv, int n_md, double dtau,
                         rsv_precision prec, uint64_t seed, uint64_t traj0, int64_t n_traj,
                         int update_theta, double* dH_out, int32_t* accept_out,
                         double* theta_out, float* snaps, int64_t thin, int fallback_window,
                         int32_t* mass_used_out, void* stream);

/* ---- many independent series ----------------------------------------------
 * A plan packs n independent series, stored end to end (series s occupies
 * [offsets[s], offsets[s+1]) of every packed array), into the register
 * windows of persistent blocks: series that fit a window are placed whole on
 * whole warps, side by side; longer ones are cut into halo tiles.  Building a
 * plan synchronises the device and allocates; running it does neither once the
 * context workspace has grown (rsv_reserve), so rsv_hmc_batched can be
 * captured in a CUDA graph.
 *  offsets: HOST int64 [n_series + 1], offsets[0] = 0, increasing (T_s >= 1).
 *  with_mass: 1 if rsv_hmc_batched will pass minv.
 * rsv_plan_info reports the chosen block shape, bins, grid and the number of
 * series cut into tiles (any output may be NULL). */
typedef struct rsv_plan rsv_plan;
rsv_status rsv_plan_create(rsv_ctx* ctx, const int64_t* offsets, int64_t n_series, int n_md,
                           rsv_precision prec, int with_mass, rsv_plan** plan);
void rsv_plan_destroy(rsv_plan* plan);
rsv_status rsv_plan_info(const rsv_plan* plan, int* threads, int* sites_per_thread, int* bins,
                         int* grid, int* split_series);

/* n_traj HMC trajectories (Sec. 3) of every series of the plan, each with its
 * own theta, all series advancing together in one persistent launch per
 * trajectory.  Series s draws its momenta and Metropolis uniform from Philox
 * with key {seed, 0} and counters {t/4, traj, 0, s} and {0, traj, 1, s}.
 *  h        packed FP64 in/out (accepted states).
 *  p        packed FP64 initial momenta (replaced by p'), or NULL to draw;
 *           non-NULL only with n_traj = 1.
 *  y, lnrv  packed FP64.   theta: device FP64 [n_series][5].
 *  minv     packed FP32 inverse masses or NULL (the plan must match).
 *  log_u    device FP64 [n_series] or NULL (draw); non-NULL only with n_traj = 1.
 *  dH_out, accept_out: device [n_traj][n_series] FP64 / int32, or NULL.
 * With RSV_MIXED the state of a series is carried as a (hi, lo) FP32 pair
 * between trajectories (about 48 significant bits); with n_traj = 1 the h of a
 * rejected series is left bit-for-bit unchanged. */
rsv_status rsv_hmc_batched(rsv_ctx* ctx, rsv_plan* plan, double* h, double* p, const double* y,
                           const double* lnrv, const double* theta, const float* minv,
                           double dtau, uint64_t seed, uint64_t traj0, int64_t n_traj,
                           const double* log_u, double* dH_out, int32_t* accept_out,
                           void* stream);

/* ---- theta update ---------------------------------------------------------
 * One Gibbs sweep of theta given h (the paper does not describe its theta
 * update): xi ~ N(mean(lnRV - h), s_u^2/T); s_u^2 ~ IG(T/2, sum(lnRV-xi-h)^2/2);
 * mu ~ N(m, s_eta^2/P) from eq. (3) and the stationary law of h_1;
 * s_eta^2 ~ IG(T/2, Q/2); phi by independence Metropolis from the Gaussian
 * part truncated to (-1,1) with ratio sqrt(1-phi'^2)/sqrt(1-phi^2).  Flat
 * priors on phi, mu, xi; 1/sigma^2 priors on the variances.  Draws come in
 * this order from Philox counter {block, traj, 2, series}, key {seed, 0}.
 *  h [T] FP64, lnrv [T] FP64, theta device FP64 [5] in/out.
 *  mask: bit 0 xi, 1 s_u^2, 2 mu, 3 s_eta^2, 4 phi (31 = all).
 *  prec: RSV_FP64 -- statistics and draws in FP64 (53-bit uniforms);
 *        RSV_MIXED -- h and lnRV as (hi, lo) FP32 pairs, statistics in
 *        double-float, the draws in FP32 from 23-bit uniforms of the same
 *        stream positions (the mixed chain draws the same way, its sums taken
 *        from the statistics of the state it keeps); theta comes out
 *        FP32-valued.
 *  phi_acc_out: device int32 scalar (1 if the phi proposal was accepted) or NULL. */
rsv_status rsv_gibbs_theta(rsv_ctx* ctx, const double* h, const double* lnrv, int64_t T,
                           double* theta, uint64_t seed, uint64_t series, uint64_t traj,
                           int mask, rsv_precision prec, int32_t* phi_acc_out, void* stream);

/* ---- learned diagonal mass ---------------------------------------------------
 * The paper has no learned part; these calls build the per-site mass m_t used
 * through `minv` above.  m_t = s (softplus(z_t) + 1e-3), z_t a 20 -> 32 -> 32 -> 1
 * MLP (tanh hidden units) on 20 standardised features of site t computed from
 * a FROZEN posterior mean hbar (never from the current h, so HMC stays exact),
 * trained by Adam (b1 0.9, b2 0.999, eps 1e-8) on the mean squared error of
 * log m_t against log(1 / Var(h_t)).  Matmuls in BF16 with FP32 accumulation
 * (tensor cores), everything else FP32; FP32 master weights.
 * Parameters: FP32 [RSV_MLP_NPARAM] = W1[32][20] b1[32] W2[32][32] b2[32]
 * W3[32] b3 (row-major W[out][in]).
 *
 * rsv_welford_update: fold the n rows of x ([n][T] FP32 sampler snapshots)
 *   into running per-site (count, mean, M2) (FP64 [T] each; count = rows
 *   already folded in; mean/M2 are ignored when count = 0).
 * rsv_welford_target: hbar_out (FP64 [T], may be NULL) = mean; target_out
 *   (FP32 [T]) = log((count - 1) / M2); log_scale_out (FP32 scalar, may be
 *   NULL) = the mean over the sites of target_out, the log of the output
 *   scale s.  count >= 2.
 * log_scale (in rsv_mlp_grad, _train, _mass): device FP32 scalar log s, fixed
 *   during training; NULL means s = 1.  s sets the scale of the network's
 *   output so that softplus works near unit slope (without it the tanh
 *   layers saturate to reach precisions of O(30) and the fit goes flat).
 * rsv_mass_features: feat_out [T][20] FP32 = standardised features
 *   (y^2, lnRV, hbar_{t-4..t+4} zero-padded, phi, mu, xi, s_eta^2, s_u^2,
 *   edge proximity 2^-d with d the distance to the nearer end,
 *   (1+phi^2)/s_eta^2, 1/s_u^2, (y^2/2) e^{-hbar}), each standardised over
 *   the sites except the edge proximity, clipped to [-8, 8]; stats_out [40]
 *   FP32 = per-feature mean and 1/sd (0 for a constant feature; 0 and 1 for
 *   the edge proximity).
 * rsv_mlp_grad: loss (FP32 scalar, may be NULL) and gradient grad_out
 *   [RSV_MLP_NPARAM] of the minibatch of Adam step `step`: batch sites drawn
 *   as floor(hi32(w) T / 2^32), w = word k%4 of Philox block k/4 with counter
 *   {k/4, step, 3, 0}, key {seed, 0}.  batch: multiple of 64.  T < 2^32.
 * rsv_mlp_train: n_steps Adam steps (steps step0 .. step0+n_steps-1, Adam time
 *   step+1) on params with state adam_m, adam_v (FP32 [RSV_MLP_NPARAM], zero
 *   before step 0); loss_out [n_steps] or NULL.
 * rsv_mlp_mass: minv_out [T] = 1/m_t and, if m_out != NULL, m_out [T] = m_t,
 *   with m_t clamped to [1/s_u^2, A_t/s_eta^2 + 1/s_u^2 + (y_t^2/2) e^{-hbar_t}]
 *   (the observation precision, a floor of the posterior precision, and the
 *   diagonal of the Hessian of S at hbar; A_t = 1 + phi^2 inside, 1 at the
 *   ends, 1 - phi^2 if T = 1), so the mass cannot destabilise the leapfrog.
 *   y, hbar: [T] FP64 (the data and frozen mean the features came from). */
#define RSV_MLP_NPARAM 1761
rsv_status rsv_welford_update(rsv_ctx* ctx, const float* x, int64_t n, int64_t T, int64_t count,
                              double* mean, double* m2, void* stream);
rsv_status rsv_welford_target(rsv_ctx* ctx, const double* mean, const double* m2, int64_t T,
                              int64_t count, double* hbar_out, float* target_out,
                              float* log_scale_out, void* stream);
rsv_status rsv_mass_features(rsv_ctx* ctx, const double* y, const double* lnrv, const double* hbar,
                             int64_t T, rsv_theta theta, float* feat_out, float* stats_out,
                             void* stream);
rsv_status rsv_mlp_grad(rsv_ctx* ctx, const float* feat, const float* target, int64_t T,
                        const float* params, const float* log_scale, uint64_t seed, uint64_t step,
                        int batch, float* grad_out, float* loss_out, void* stream);
rsv_status rsv_mlp_train(rsv_ctx* ctx, const float* feat, const float* target, int64_t T,
                         float* params, const float* log_scale, float* adam_m, float* adam_v,
                         int64_t step0, int n_steps, int batch, uint64_t seed, float lr,
                         float* loss_out, void* stream);
rsv_status rsv_mlp_mass(rsv_ctx* ctx, const float* feat, int64_t T, const float* params,
                        const float* log_scale, const double* y, const double* hbar,
                        rsv_theta theta, float* minv_out, float* m_out, void* stream);

/* ---- Philox momenta (exposed for tests of the generator) -----------------
 * p_t exactly as rsv_hmc_trajectory draws them for (seed, series, traj);
 * bits = 53 (FP64 path) or 23 (MIXED path). p_out [T] FP64. */
rsv_status rsv_draw_momenta(rsv_ctx* ctx, uint64_t seed, uint64_t series, uint64_t traj,
                            int64_t T, const float* minv, int bits, double* p_out, void* stream);

/* ---- double-float exponential (exposed for tests of the mixed energies) ----
 * The exponential the MIXED path takes in its energies and state statistics
 * (the return term (y^2/2) e^{-h} of S, Sec. 3), in double-float arithmetic:
 * t = tk ln2/32 + r, |r| <= ln2/64, a degree-5 Taylor polynomial of e^r, the
 * table value 2^{(k mod 32)/32} and an exact power of two.  t: [n] device
 * FP64, each rounded to a double-float (hi = (float)t, lo = (float)(t - hi))
 * as the kernels hold their arguments; out: [n] device FP64 = hi + lo of the
 * scalar form; out2: [n] the two-lane form the end-of-trajectory statistics
 * use (equal to out bit for bit); either may be NULL.  |t| < 80 keeps the
 * result finite and normal (outside it the result is undefined; no error is
 * raised); below t ~ -70 its small part is subnormal and the relative error
 * grows past ~1e-11.  n >= 0, else RSV_EINVAL. */
rsv_status rsv_ff_exp(rsv_ctx* ctx, const double* t, double* out, double* out2, int64_t n,
                      void* stream);
/* rsv_fp64_exp: the exponential of the FP64 path's force and energies
 * (exp_tab): Tang's table-driven method, t = k ln2/64 + r, |r| <= ln2/128,
 * e^t = 2^(k div 64) 2^((k mod 64)/64) (1 + p(r)), p the degree-5 Taylor
 * polynomial of e^r - 1, the table 2^(j/64) rounded to double; |t| >= 512
 * falls back to CUDA's exp.  t, out: [n] device FP64.  n >= 0 and non-NULL
 * pointers when n > 0, else RSV_EINVAL. */
rsv_status rsv_fp64_exp(rsv_ctx* ctx, const double* t, double* out, int64_t n, void* stream);

/* ---- measurement -----------------------------------------------------------
 * rsv_ess: effective sample size of every column t of x, a [n][T] FP32 matrix
 * of n chain samples (row k = sample k), by Geyer's initial monotone sequence
 * estimator (Statistical Science 7, 1992) on the plain autocovariances; ESS is
 * capped at n log10(n).  ess_out [T] FP32.  n >= 2.  (Not part of the paper's
 * method; used to report ESS/s.)
 * rsv_timing: enable (1) / disable (0) CUDA-event timing of every trajectory
 * kernel launch (skipped while the stream is being captured).
 * rsv_stats: kernel launches made by the library, trajectory-kernel launches
 * (a persistent chain launch counts each of its trajectories) and their summed
 * device time (ms) since the last reset; synchronises the recorded events;
 * reset != 0 clears the counters after reading. */
rsv_status rsv_ess(rsv_ctx* ctx, const float* x, int64_t n, int64_t T, float* ess_out,
                   void* stream);
/* rsv_pipe_probe: launch one probe kernel that keeps one on-chip unit busy on
 * every SM with independent dependency chains, and set *ops_out (host) to the
 * number of operations that launch performs; the caller times the launch on
 * `stream` (CUDA events) and divides.  Not part of the paper's method: it
 * measures the peaks the trajectory kernels are reported against.
 *   RSV_PROBE_FFMA   scalar FP32 FMA               (ops = FMAs)
 *   RSV_PROBE_FFMA2  packed FP32 FMA, 2 per instruction (ops = FMAs)
 *   RSV_PROBE_EX2    ex2.approx.f32 on the special-function unit, each
 *                    followed by one dependent FP32 FMA   (ops = ex2)
 *   RSV_PROBE_LDS    16-byte shared-memory loads    (ops = bytes loaded)
 *   RSV_PROBE_DFMA   FP64 FMA                       (ops = FMAs)
 * iters: 1 .. 2^40 (each thread runs 16 iters x 8 chains of its kind). */
enum { RSV_PROBE_FFMA = 0, RSV_PROBE_FFMA2 = 1, RSV_PROBE_EX2 = 2, RSV_PROBE_LDS = 3,
       RSV_PROBE_DFMA = 4 };
rsv_status rsv_pipe_probe(rsv_ctx* ctx, int kind, int64_t iters, double* ops_out, void* stream);
rsv_status rsv_timing(rsv_ctx* ctx, int enable);
rsv_status rsv_stats(rsv_ctx* ctx, int reset, int64_t* launches, int64_t* traj_launches,
                     double* traj_ms);

#ifdef __cplusplus
}
#endif

#endif /* RSV_H_ */
