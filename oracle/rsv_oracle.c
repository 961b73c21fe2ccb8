/*
 * rsv_oracle.c -- plain, slow, FP64 CPU oracle for the Hybrid Monte Carlo
 * volatility update of the realized stochastic volatility (RSV) model
 * (Takaishi, "GPU Computing in Bayesian Inference of Realized Stochastic
 * Volatility Model", arXiv:1603.08114).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is compared against.  It shares no code, header, table or
 * constant generator with the CUDA path, and the library never calls it.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.
 *
 * Every loop is the definition written out, in the paper's order:
 *   - the model, eqs. (1)-(3) (Sec. 2);
 *   - the Hamiltonian H(p,h) = 1/2 sum p_i^2 - ln f(h,theta) (Sec. 3);
 *   - the leapfrog h-half / p-full / h-half, eqs. (6)-(8), repeated k times
 *     with l = k * dtau (Sec. 3);
 *   - Metropolis acceptance with probability min{1, exp(-dH)} (Sec. 3).
 * The paper does not write f out; S(h) = -ln f below is derived from
 * eqs. (1)-(3) with the stationary AR(1) law for h_1 (a reading: the paper
 * leaves the law of h_1 unstated).  Indices are 0-based here (the paper's
 * t = 1..T is t = 0..T-1).
 *
 * Parity status of each function is stated beside it; every one is pinned by a
 * CPU test (finite differences, reversibility, dtau^2 scaling, Kalman smoother,
 * quadrature, numpy's Philox, closed forms).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fused
 * multiply-add contraction, so x86 and Arm give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* theta of eqs. (1)-(3), and rho = corr(eps_t, eta_t) of the RSV model with
 * leverage (Takahashi, Omori and Watanabe, Comput. Stat. Data Anal. 53 (2009)
 * 2404, the RSV model the paper cites in Sec. 2); rho = 0 is eqs. (1)-(3). */
typedef struct {
    double phi, mu, xi, sig_eta2, sig_u2, rho;
} orc_theta;

/* ------------------------------------------------------------------------ */
/* Compensated summation (Neumaier's improvement of Kahan summation).       */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } orc_sum;

static void sum_add(orc_sum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double sum_get(const orc_sum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Action S(h) = -ln f(h | theta, y, lnRV), constants dropped (Sec. 3 with    */
/* the model of eqs. (1)-(3)).  Per-site split used for dH:                  */
/*   s_t = h_t/2 + (y_t^2/2) e^{-h_t} + (lnRV_t - xi - h_t)^2 / (2 s_u^2)     */
/*       + [t < T-1] d_t^2 / (2 s_eta^2 (1 - rho^2))                          */
/*       + [t = 0]   (1 - phi^2) x_0^2 / (2 s_eta^2),      x_t = h_t - mu,    */
/*   d_t = x_{t+1} - phi x_t - rho s_eta eps_t,  eps_t = y_t e^{-h_t/2}.      */
/* With leverage (rho != 0) the pair (eps_t, eta_t) is bivariate normal with  */
/* correlation rho, so eta_t | eps_t ~ N(rho s_eta eps_t, s_eta^2 (1-rho^2)); */
/* the marginal of eta_t, hence the stationary law of h_1, is unchanged.      */
/* rho = 0 gives the d_t = x_{t+1} - phi x_t of eq. (3).                      */
/* ------------------------------------------------------------------------ */
/* rho s_eta eps_t, the leverage shift of eta_t's conditional mean (exactly
 * 0 for rho = 0, where the exponential is not needed). */
static double lev_shift(const double* h, const double* y, orc_theta th, long t)
{
    if (th.rho == 0.0) return 0.0;
    return th.rho * sqrt(th.sig_eta2) * (y[t] * exp(-0.5 * h[t]));
}

double orc_site_action(const double* h, const double* y, const double* lnrv,
                       long T, orc_theta th, long t)
{
    double ht = h[t];
    /* eq. (1): y_t ~ N(0, e^{h_t}) */
    double s = 0.5 * ht + 0.5 * y[t] * y[t] * exp(-ht);
    /* eq. (2): lnRV_t ~ N(xi + h_t, s_u^2) */
    double r = lnrv[t] - th.xi - ht;
    s += r * r / (2.0 * th.sig_u2);
    /* eq. (3): h_{t+1} ~ N(mu + phi (h_t - mu), s_eta^2), given eps_t with
     * leverage: N(mu + phi (h_t - mu) + rho s_eta eps_t, s_eta^2 (1 - rho^2)) */
    double x = ht - th.mu;
    if (t + 1 < T) {
        double d = (h[t + 1] - th.mu) - th.phi * x - lev_shift(h, y, th, t);
        s += d * d / (2.0 * th.sig_eta2 * (1.0 - th.rho * th.rho));
    }
    /* stationary law of h_1: N(mu, s_eta^2 / (1 - phi^2)) */
    if (t == 0) s += (1.0 - th.phi * th.phi) * x * x / (2.0 * th.sig_eta2);
    return s;
}

void orc_action_sites(const double* h, const double* y, const double* lnrv,
                      long T, orc_theta th, double* s_out)
{
    for (long t = 0; t < T; ++t) s_out[t] = orc_site_action(h, y, lnrv, T, th, t);
}

double orc_action(const double* h, const double* y, const double* lnrv,
                  long T, orc_theta th)
{
    orc_sum acc = {0.0, 0.0};
    for (long t = 0; t < T; ++t) sum_add(&acc, orc_site_action(h, y, lnrv, T, th, t));
    return sum_get(&acc);
}

/* ------------------------------------------------------------------------ */
/* Gradient dS/dh_t (the dH/dh_i of eq. (7)), term by term from s_t above:   */
/*   dS/dh_t = 1/2 - (y_t^2/2) e^{-h_t} - (lnRV_t - xi - h_t)/s_u^2 + AR_t,   */
/*   AR_t = [t = 0] (1 - phi^2) x_0 / s_eta^2                                */
/*        + [t < T-1] B d_t (rho s_eta eps_t / 2 - phi)     (from d_t)        */
/*        + [t > 0]   B d_{t-1}                             (from d_{t-1}),   */
/*   B = 1 / (s_eta^2 (1 - rho^2)),  d d_t/d h_t = -phi + rho s_eta eps_t/2.  */
/* With rho = 0 the interior rows are [(1+phi^2) x_t - phi (x_{t-1} +        */
/* x_{t+1})] / s_eta^2, the end rows (x_0 - phi x_1) / s_eta^2 and            */
/* (x_{T-1} - phi x_{T-2}) / s_eta^2, and (1 - phi^2) x_0 / s_eta^2 for T = 1.*/
/* ------------------------------------------------------------------------ */
static double innovation(const double* h, const double* y, orc_theta th, long t)
{
    return (h[t + 1] - th.mu) - th.phi * (h[t] - th.mu) - lev_shift(h, y, th, t);
}

void orc_force(const double* h, const double* y, const double* lnrv,
               long T, orc_theta th, double* F)
{
    const double phi = th.phi, mu = th.mu;
    const double B = 1.0 / (th.sig_eta2 * (1.0 - th.rho * th.rho));
    for (long t = 0; t < T; ++t) {
        double x = h[t] - mu, ar = 0.0;
        if (t == 0) ar += (1.0 - phi * phi) * x / th.sig_eta2;
        if (t + 1 < T)  /* d d_t / d h_t = -phi + (rho s_eta eps_t) / 2 */
            ar += B * innovation(h, y, th, t) * (0.5 * lev_shift(h, y, th, t) - phi);
        if (t > 0) ar += B * innovation(h, y, th, t - 1);
        F[t] = 0.5 - 0.5 * y[t] * y[t] * exp(-h[t])
             - (lnrv[t] - th.xi - h[t]) / th.sig_u2 + ar;
    }
}

/* ------------------------------------------------------------------------ */
/* Leapfrog, eqs. (6)-(8), repeated n_md times (l = n_md * dtau).            */
/* With a diagonal mass m_t (minv = 1/m_t, NULL = identity) the kinetic term */
/* is 1/2 sum p_t^2 / m_t, so dh/dtau = p/m in eq. (4).                      */
/* h, p are updated in place.                                                */
/* ------------------------------------------------------------------------ */
void orc_leapfrog(double* h, double* p, const double* y, const double* lnrv,
                  long T, orc_theta th, const double* minv, int n_md, double dtau)
{
    double* F = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    for (int k = 0; k < n_md; ++k) {
        for (long t = 0; t < T; ++t)                      /* eq. (6) */
            h[t] = h[t] + 0.5 * dtau * (minv ? minv[t] * p[t] : p[t]);
        orc_force(h, y, lnrv, T, th, F);
        for (long t = 0; t < T; ++t)                      /* eq. (7) */
            p[t] = p[t] - dtau * F[t];
        for (long t = 0; t < T; ++t)                      /* eq. (8) */
            h[t] = h[t] + 0.5 * dtau * (minv ? minv[t] * p[t] : p[t]);
    }
    free(F);
}

/* n_md steps of the second-order minimum-norm integrator of Omelyan, Mryglod
 * and Folk (Phys. Rev. E 65, 056706 (2002)), one of the higher-order
 * integrators the paper cites (Sec. 3), taken literally: per step
 *   h += lambda dtau p/m;  p -= dtau/2 dS/dh;  h += (1 - 2 lambda) dtau p/m;
 *   p -= dtau/2 dS/dh;  h += lambda dtau p/m.
 * lambda = 1/2 gives eqs. (6)-(8) with the force step split in two halves. */
void orc_omelyan2(double* h, double* p, const double* y, const double* lnrv,
                  long T, orc_theta th, const double* minv, int n_md, double dtau,
                  double lambda)
{
    double* F = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    const double c[3] = {lambda * dtau, (1.0 - 2.0 * lambda) * dtau, lambda * dtau};
    for (int k = 0; k < n_md; ++k) {
        for (int s = 0; s < 3; ++s) {
            for (long t = 0; t < T; ++t) h[t] = h[t] + c[s] * (minv ? minv[t] * p[t] : p[t]);
            if (s == 2) break;
            orc_force(h, y, lnrv, T, th, F);
            for (long t = 0; t < T; ++t) p[t] = p[t] - 0.5 * dtau * F[t];
        }
    }
    free(F);
}

/* n_md steps of the fourth-order force-gradient-free integrator of Omelyan,
 * Mryglod and Folk (Comput. Phys. Commun. 146, 188 (2002)), their
 * position-extended Forest-Ruth-like scheme with the minimum error norm,
 * taken literally: per step five drifts and four kicks
 *   h += xi dtau p/m;  p -= (1 - 2 lambda)/2 dtau dS/dh;  h += chi dtau p/m;
 *   p -= lambda dtau dS/dh;  h += (1 - 2 (chi + xi)) dtau p/m;
 *   p -= lambda dtau dS/dh;  h += chi dtau p/m;
 *   p -= (1 - 2 lambda)/2 dtau dS/dh;  h += xi dtau p/m,
 * with their published constants xi, lambda, chi (the drifts and the kicks
 * each sum to 1; the scheme is symmetric, so reversible). */
#define ORC_PEFRL_XI 0.1786178958448091
#define ORC_PEFRL_LAMBDA (-0.2123418310626054)
#define ORC_PEFRL_CHI (-0.06626458266981849)
void orc_omelyan4(double* h, double* p, const double* y, const double* lnrv,
                  long T, orc_theta th, const double* minv, int n_md, double dtau)
{
    double* F = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    const double xi = ORC_PEFRL_XI, lam = ORC_PEFRL_LAMBDA, chi = ORC_PEFRL_CHI;
    const double a[5] = {xi, chi, 1.0 - 2.0 * (chi + xi), chi, xi};
    const double b[4] = {0.5 * (1.0 - 2.0 * lam), lam, lam, 0.5 * (1.0 - 2.0 * lam)};
    for (int k = 0; k < n_md; ++k) {
        for (int s = 0; s < 5; ++s) {
            const double cd = a[s] * dtau;
            for (long t = 0; t < T; ++t) h[t] = h[t] + cd * (minv ? minv[t] * p[t] : p[t]);
            if (s == 4) break;
            orc_force(h, y, lnrv, T, th, F);
            const double ck = b[s] * dtau;
            for (long t = 0; t < T; ++t) p[t] = p[t] - ck * F[t];
        }
    }
    free(F);
}

/* The integrator of a trajectory: 0 = leapfrog (eqs. (6)-(8)), 1 = the
 * minimum-norm integrator above with the given lambda, 2 = the fourth-order
 * scheme above. */
static void orc_integrate(double* h, double* p, const double* y, const double* lnrv, long T,
                          orc_theta th, const double* minv, int n_md, double dtau,
                          int integrator, double lambda)
{
    if (integrator == 2) orc_omelyan4(h, p, y, lnrv, T, th, minv, n_md, dtau);
    else if (integrator == 1) orc_omelyan2(h, p, y, lnrv, T, th, minv, n_md, dtau, lambda);
    else orc_leapfrog(h, p, y, lnrv, T, th, minv, n_md, dtau);
}

/* dH = H(p', h') - H(p, h), summed as per-site differences with compensation
 * so that the O(1) result is not lost against the O(T) action (Sec. 3). */
double orc_delta_H(const double* h0, const double* p0, const double* h1, const double* p1,
                   const double* y, const double* lnrv, long T, orc_theta th,
                   const double* minv)
{
    orc_sum acc = {0.0, 0.0};
    for (long t = 0; t < T; ++t) {
        double w = minv ? minv[t] : 1.0;
        double dk = 0.5 * w * (p1[t] * p1[t] - p0[t] * p0[t]);
        double ds = orc_site_action(h1, y, lnrv, T, th, t) - orc_site_action(h0, y, lnrv, T, th, t);
        sum_add(&acc, dk + ds);
    }
    return sum_get(&acc);
}

/* Metropolis test of Sec. 3: accept with probability min{1, e^{-dH}},
 * i.e. accept iff ln u < -dH for u ~ U(0,1).  A NaN dH rejects. */
int orc_metropolis(double dH, double log_u)
{
    if (!(dH == dH)) return 0;
    return log_u < -dH ? 1 : 0;
}

/* One HMC trajectory (Sec. 3): leapfrog from (h, p), dH, Metropolis.
 * On accept h <- h'; on reject h is left as it was.  p is overwritten by p'.
 * Returns the accept flag; *dH_out receives dH. */
int orc_trajectory(double* h, double* p, const double* y, const double* lnrv,
                   long T, orc_theta th, const double* minv, int n_md, double dtau,
                   double log_u, double* dH_out, int integrator, double lambda)
{
    size_t n = (size_t)(T > 0 ? T : 1);
    double* h1 = (double*)malloc(sizeof(double) * n);
    double* p0 = (double*)malloc(sizeof(double) * n);
    memcpy(h1, h, sizeof(double) * (size_t)T);
    memcpy(p0, p, sizeof(double) * (size_t)T);
    orc_integrate(h1, p, y, lnrv, T, th, minv, n_md, dtau, integrator, lambda);
    double dH = orc_delta_H(h, p0, h1, p, y, lnrv, T, th, minv);
    int acc = orc_metropolis(dH, log_u);
    if (acc) memcpy(h, h1, sizeof(double) * (size_t)T);
    if (dH_out) *dH_out = dH;
    free(h1);
    free(p0);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of                                    */
/*   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))*/
/* with the key bumped by the Weyl constants between rounds.                 */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    /* 64x64 -> 128 by 32-bit halves (portable C, no compiler extension). */
    uint64_t a0 = a & 0xffffffffULL, a1 = a >> 32;
    uint64_t b0 = b & 0xffffffffULL, b1 = b >> 32;
    uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffULL) + (p10 & 0xffffffffULL);
    *lo = (mid << 32) | (p00 & 0xffffffffULL);
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout shared by both sides of the parity tests (a convention,
 * not arithmetic): counter = {block, trajectory, stream, series},
 * key = {seed, 0}.  Streams: 0 momenta, 1 Metropolis uniform, 2 theta draws. */
enum { ORC_STREAM_MOM = 0, ORC_STREAM_MH = 1, ORC_STREAM_THETA = 2 };

static void philox_block(uint64_t seed, uint64_t series, uint64_t traj, uint64_t stream,
                         uint64_t block, uint64_t out[4])
{
    uint64_t ctr[4] = {block, traj, stream, series};
    uint64_t key[2] = {seed, 0};
    orc_philox4x64_10(ctr, key, out);
}

/* Uniform in (0,1) from the top `bits` bits of a 64-bit word: (k + 1/2) 2^-bits. */
double orc_u01(uint64_t w, int bits)
{
    uint64_t k = w >> (64 - bits);
    return ((double)k + 0.5) * ldexp(1.0, -bits);
}

/* Box-Muller (Box & Muller 1958): (u1, u2) -> r cos(2 pi u2), r sin(2 pi u2),
 * r = sqrt(-2 ln u1). */
void orc_box_muller(double u1, double u2, double* z0, double* z1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(two_pi * u2);
    *z1 = r * sin(two_pi * u2);
}

/* Momenta p_t ~ N(0, m_t) for one trajectory: Philox block q gives the four
 * words of sites 4q..4q+3; words (0,1) -> sites 4q, 4q+1 and (2,3) -> 4q+2,
 * 4q+3 by Box-Muller.  bits = 53 for the FP64 path, 24 for the FP32 path. */
void orc_draw_momenta(uint64_t seed, uint64_t series, uint64_t traj, long T,
                      const double* minv, int bits, double* p)
{
    for (long q = 0; 4 * q < T; ++q) {
        uint64_t w[4];
        double z[4];
        philox_block(seed, series, traj, ORC_STREAM_MOM, (uint64_t)q, w);
        orc_box_muller(orc_u01(w[0], bits), orc_u01(w[1], bits), &z[0], &z[1]);
        orc_box_muller(orc_u01(w[2], bits), orc_u01(w[3], bits), &z[2], &z[3]);
        for (int i = 0; i < 4; ++i) {
            long t = 4 * q + i;
            if (t < T) p[t] = minv ? z[i] / sqrt(minv[t]) : z[i];
        }
    }
}

/* ln u for the Metropolis test of one trajectory: first word of block 0 of
 * the Metropolis stream, 53 bits. */
double orc_draw_log_u(uint64_t seed, uint64_t series, uint64_t traj)
{
    uint64_t w[4];
    philox_block(seed, series, traj, ORC_STREAM_MH, 0, w);
    return log(orc_u01(w[0], 53));
}

/* ------------------------------------------------------------------------ */
/* Sequential draws for the theta update: words are consumed in order from   */
/* blocks 0, 1, 2, ... of the theta stream of one trajectory.                */
/* ------------------------------------------------------------------------ */
/* margin: the smallest distance of any accept/reject decision taken from    */
/* the stream to its boundary (relative to 1 + |boundary|), for tests that   */
/* compare with a lower-precision sampler of the same stream.               */
typedef struct {
    uint64_t seed, series, traj, block;
    uint64_t w[4];
    int pos;
    int bits;      /* uniforms (k + 1/2) 2^-bits from the top bits of each word */
    double margin;
} orc_stream;

static void stream_init(orc_stream* s, uint64_t seed, uint64_t series, uint64_t traj)
{
    s->seed = seed; s->series = series; s->traj = traj; s->block = 0; s->pos = 4;
    s->bits = 53;
    s->margin = INFINITY;
}
static void stream_margin(orc_stream* s, double lhs, double rhs)
{
    double m = fabs(lhs - rhs) / (1.0 + fabs(rhs));
    if (m < s->margin) s->margin = m;
}
static double stream_u01(orc_stream* s)
{
    if (s->pos == 4) {
        philox_block(s->seed, s->series, s->traj, ORC_STREAM_THETA, s->block++, s->w);
        s->pos = 0;
    }
    return orc_u01(s->w[s->pos++], s->bits);
}
/* One standard normal per call: the cosine branch of Box-Muller. */
static double stream_normal(orc_stream* s)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = stream_u01(s), u2 = stream_u01(s);
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}
/* Gamma(alpha, 1), Marsaglia & Tsang (2000) for alpha >= 1; alpha < 1 by
 * Gamma(alpha + 1) * u^(1/alpha).  Gives up after 1000 rounds (returns NaN). */
static double stream_gamma(orc_stream* s, double alpha)
{
    if (alpha < 1.0) {
        double g = stream_gamma(s, alpha + 1.0);
        double u = stream_u01(s);
        return g * pow(u, 1.0 / alpha);
    }
    double d = alpha - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (int it = 0; it < 1000; ++it) {
        double z = stream_normal(s);
        double v = 1.0 + c * z;
        stream_margin(s, v, 0.0);
        if (v <= 0.0) continue;
        v = v * v * v;
        double u = stream_u01(s);
        double bound = 0.5 * z * z + d - d * v + d * log(v);
        stream_margin(s, log(u), bound);
        if (log(u) < bound) return d * v;
    }
    return NAN;
}

/* ------------------------------------------------------------------------ */
/* theta update.  The paper uses the code of its ref. [Takaishi4] and does   */
/* not describe it (Sec. 2); this is an exact Gibbs sweep under flat priors  */
/* on phi in (-1,1), mu, xi and 1/sigma^2 priors on both variances:          */
/*   xi      ~ N(mean(lnRV - h), s_u^2 / T)                                  */
/*   s_u^2   ~ IG(T/2, sum (lnRV - xi - h)^2 / 2)                            */
/*   mu      ~ N(m_mu, 1/P_mu) from the quadratic form of eq. (3) + h_1 law */
/*   s_eta^2 ~ IG(T/2, Q/2), Q = (1-phi^2) x_1^2 + sum (x_{t+1} - phi x_t)^2 */
/*   phi     : independence Metropolis from N(sum x_t x_{t+1} / D,          */
/*             s_eta^2 / D) truncated to (-1,1), D = sum_{t=2}^{T-1} x_t^2, */
/*             accepted with ratio sqrt(1-phi'^2)/sqrt(1-phi^2).             */
/* Every sum is taken directly over the series with the current values.     */
/* mask selects the components updated (bit 0 xi, 1 s_u^2, 2 mu, 3 s_eta^2, */
/* 4 phi); the draws of a skipped component are not consumed.               */
/* Returns 1 if the phi proposal was accepted, -1 (theta untouched) under   */
/* leverage, where these conditionals are not the model's.                  */
/* ------------------------------------------------------------------------ */
static int gibbs_theta(const double* h, const double* lnrv, long T, orc_theta* th,
                       uint64_t seed, uint64_t series, uint64_t traj, int mask,
                       int bits, double* margin_out)
{
    if (th->rho != 0.0) return -1;
    orc_stream st;
    stream_init(&st, seed, series, traj);
    st.bits = bits;
    double Td = (double)T;

    /* xi */
    if (mask & 1) {
        orc_sum a = {0, 0};
        for (long t = 0; t < T; ++t) sum_add(&a, lnrv[t] - h[t]);
        double mean_r = sum_get(&a) / Td;
        th->xi = mean_r + sqrt(th->sig_u2 / Td) * stream_normal(&st);
    }

    /* s_u^2 */
    if (mask & 2) {
        orc_sum ss = {0, 0};
        for (long t = 0; t < T; ++t) {
            double r = lnrv[t] - th->xi - h[t];
            sum_add(&ss, r * r);
        }
        double g = stream_gamma(&st, 0.5 * Td);
        /* a degenerate state (zero residuals) keeps the old value */
        if (g > 0.0 && sum_get(&ss) > 0.0) th->sig_u2 = 0.5 * sum_get(&ss) / g;
    }

    /* mu */
    if (mask & 4) {
        double phi = th->phi;
        double w0 = 1.0 - phi * phi, w1 = (1.0 - phi) * (1.0 - phi);
        orc_sum num = {0, 0};
        sum_add(&num, w0 * h[0]);
        for (long t = 0; t + 1 < T; ++t) sum_add(&num, (1.0 - phi) * (h[t + 1] - phi * h[t]));
        double prec = (w0 + (Td - 1.0) * w1) / th->sig_eta2;
        double m = sum_get(&num) / (w0 + (Td - 1.0) * w1);
        th->mu = m + stream_normal(&st) / sqrt(prec);
    }

    /* s_eta^2 */
    if (mask & 8) {
        double phi = th->phi, mu = th->mu;
        orc_sum q = {0, 0};
        double x0 = h[0] - mu;
        sum_add(&q, (1.0 - phi * phi) * x0 * x0);
        for (long t = 0; t + 1 < T; ++t) {
            double e = (h[t + 1] - mu) - phi * (h[t] - mu);
            sum_add(&q, e * e);
        }
        double g2 = stream_gamma(&st, 0.5 * Td);
        if (g2 > 0.0 && sum_get(&q) > 0.0) th->sig_eta2 = 0.5 * sum_get(&q) / g2;
    }

    /* phi */
    int acc = 0;
    if (mask & 16) {
        double mu = th->mu;
        orc_sum num = {0, 0}, den = {0, 0};
        for (long t = 0; t + 1 < T; ++t) sum_add(&num, (h[t] - mu) * (h[t + 1] - mu));
        for (long t = 1; t + 1 < T; ++t) sum_add(&den, (h[t] - mu) * (h[t] - mu));
        double D = sum_get(&den);
        if (D > 0.0) {
            double m = sum_get(&num) / D, sd = sqrt(th->sig_eta2 / D);
            double prop = NAN;
            for (int it = 0; it < 1000; ++it) {
                double c = m + sd * stream_normal(&st);
                stream_margin(&st, fabs(c), 1.0);
                if (c > -1.0 && c < 1.0) { prop = c; break; }
            }
            double u = stream_u01(&st);
            if (prop == prop) {
                double lr = 0.5 * log(1.0 - prop * prop) - 0.5 * log(1.0 - th->phi * th->phi);
                stream_margin(&st, log(u), lr);
                if (log(u) < lr) { th->phi = prop; acc = 1; }
            }
        }
    }
    if (margin_out) *margin_out = st.margin;
    return acc;
}

int orc_gibbs_theta(const double* h, const double* lnrv, long T, orc_theta* th,
                    uint64_t seed, uint64_t series, uint64_t traj, int mask)
{
    return gibbs_theta(h, lnrv, T, th, seed, series, traj, mask, 53, NULL);
}

/* The same sweep from uniforms of `bits` bits (53, or 23 as a sampler that   */
/* draws in FP32 takes them from the same words), also reporting the        */
/* stream's smallest decision margin.                                       */
int orc_gibbs_theta_margin(const double* h, const double* lnrv, long T, orc_theta* th,
                           uint64_t seed, uint64_t series, uint64_t traj, int mask, int bits,
                           double* margin_out)
{
    if (bits < 1 || bits > 53) return -2;
    return gibbs_theta(h, lnrv, T, th, seed, series, traj, mask, bits, margin_out);
}

/* ------------------------------------------------------------------------ */
/* A chain of n_traj HMC trajectories (Sec. 3), each with Philox momenta and */
/* Metropolis uniform for trajectory index traj0 + n, optionally followed by */
/* the theta update.  Records dH, accept and theta per trajectory, and h    */
/* after every `thin`-th trajectory into snaps (n_traj/thin rows of T).      */
/* bits selects the uniform width used for the momenta (53 FP64, 24 FP32).   */
/* Returns -1 if a theta update is asked for under leverage.                */
/* ------------------------------------------------------------------------ */
long orc_chain(double* h, const double* y, const double* lnrv, long T, orc_theta* th,
               const double* minv, int n_md, double dtau, uint64_t seed, uint64_t series,
               uint64_t traj0, long n_traj, int update_theta, int bits,
               double* dH_out, int* acc_out, double* theta_out, double* snaps, long thin,
               int integrator, double lambda)
{
    if (update_theta && th->rho != 0.0) return -1;
    size_t n = (size_t)(T > 0 ? T : 1);
    double* p = (double*)malloc(sizeof(double) * n);
    long n_acc = 0;
    for (long i = 0; i < n_traj; ++i) {
        uint64_t traj = traj0 + (uint64_t)i;
        orc_draw_momenta(seed, series, traj, T, minv, bits, p);
        double log_u = orc_draw_log_u(seed, series, traj);
        double dH;
        int acc = orc_trajectory(h, p, y, lnrv, T, *th, minv, n_md, dtau, log_u, &dH,
                                 integrator, lambda);
        n_acc += acc;
        if (update_theta) orc_gibbs_theta(h, lnrv, T, th, seed, series, traj, 31);
        if (dH_out) dH_out[i] = dH;
        if (acc_out) acc_out[i] = acc;
        if (theta_out) {
            theta_out[5 * i + 0] = th->phi;
            theta_out[5 * i + 1] = th->mu;
            theta_out[5 * i + 2] = th->xi;
            theta_out[5 * i + 3] = th->sig_eta2;
            theta_out[5 * i + 4] = th->sig_u2;
        }
        if (snaps && thin > 0 && (i + 1) % thin == 0)
            memcpy(snaps + (size_t)((i + 1) / thin - 1) * (size_t)T, h, sizeof(double) * (size_t)T);
    }
    free(p);
    return n_acc;
}
