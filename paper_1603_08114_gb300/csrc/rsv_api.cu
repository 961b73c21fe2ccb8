// rsv_api.cu -- the extern "C" entry points of librsv (declared in include/rsv.h).
//
// Argument checks, the context's workspace and the order of launches on the
// caller's stream.  All arithmetic of the method runs in the kernels of
// rsv_traj.cu, rsv_simple.cu and the other .cu files of this directory.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "rsv.h"
#include "rsv_ctx.cuh"
#include "rsv_ess.cuh"
#include "rsv_gibbs.cuh"
#include "rsv_simple.cuh"
#include "rsv_traj.cuh"
#include "rsv_api_common.cuh"

using namespace rsv;

namespace rsv {

thread_local std::string g_last_error;

rsv_status fail(rsv_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

rsv_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(RSV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool theta_ok(const rsv_theta& t)
{
    return std::isfinite(t.phi) && std::isfinite(t.mu) && std::isfinite(t.xi) &&
           std::isfinite(t.sig_eta2) && std::isfinite(t.sig_u2) && std::fabs(t.phi) < 1.0 &&
           t.sig_eta2 > 0.0 && t.sig_u2 > 0.0;
}

ThetaD to_dev(const rsv_theta& t) { return ThetaD{t.phi, t.mu, t.xi, t.sig_eta2, t.sig_u2}; }

// Grow a workspace buffer to at least `bytes`; never shrinks.
rsv_status Buf::ensure(size_t bytes)
{
    if (bytes <= cap) return RSV_OK;
    if (capture_active())
        return fail(RSV_EINVAL, "workspace must grow during stream capture; call rsv_reserve first");
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    size_t b = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&ptr, b);
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        return fail(RSV_ENOMEM, "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    }
    cap = b;
    return RSV_OK;
}
void Buf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
}

bool capture_active_on(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

thread_local cudaStream_t g_cur_stream = nullptr;
bool capture_active() { return capture_active_on(g_cur_stream); }

rsv_status ctx_begin(rsv_ctx* c, void* stream)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    g_cur_stream = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return RSV_OK;
}

rsv_status ctx_ensure_partials(rsv_ctx* c, int64_t n)
{
    return c->partials.ensure((size_t)n * kPartialWords * sizeof(double));
}

// Count a kernel launch made through launcher f.

}  // namespace rsv

extern "C" {

const char* rsv_last_error(void) { return g_last_error.c_str(); }
int rsv_abi_version(void) { return RSV_ABI_VERSION; }

rsv_status rsv_create(rsv_ctx** out, int device)
{
    if (!out) return fail(RSV_EINVAL, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(RSV_EINVAL, "device %d out of range", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    rsv_ctx* c = new rsv_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    g_cur_stream = nullptr;
    rsv_status st = c->ints.ensure(kIntSlots * sizeof(int));
    if (st == RSV_OK) st = c->partials.ensure(4096 * sizeof(double));
    if (st == RSV_OK) st = c->scalars.ensure(64 * sizeof(double));
    if (st != RSV_OK) {
        rsv_destroy(c);
        return st;
    }
    e = cudaMemset(c->ints.ptr, 0, kIntSlots * sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rsv_destroy(c);
        return cuda_fail(e, "workspace init");
    }
    *out = c;
    return RSV_OK;
}

void rsv_destroy(rsv_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (auto& e : c->plans) free_plan(e.plan);
    for (Buf* b : c->all_bufs()) b->release();
    delete c;
}

rsv_status rsv_reserve(rsv_ctx* c, int64_t max_T, int64_t max_series)
{
    rsv_status st = ctx_begin(c, nullptr);
    if (st != RSV_OK) return st;
    if (max_T < 0 || max_series < 0) return fail(RSV_EINVAL, "negative reserve size");
    const size_t T = (size_t)max_T;
    if ((st = c->dbuf0.ensure(T * 8)) != RSV_OK) return st;
    if ((st = c->dbuf1.ensure(T * 8)) != RSV_OK) return st;
    if ((st = c->fbuf0.ensure(T * 8)) != RSV_OK) return st;
    if ((st = c->fbuf1.ensure(T * 8)) != RSV_OK) return st;
    if ((st = c->a_f.ensure(T * 4)) != RSV_OK) return st;
    if ((st = c->lr_f.ensure(T * 8)) != RSV_OK) return st;
    if ((st = ctx_ensure_partials(c, (max_T / 64 + 4096))) != RSV_OK) return st;
    const size_t n = (size_t)(max_series > 1 ? max_series : 1);
    if ((st = c->ser_cur.ensure(n * sizeof(int))) != RSV_OK) return st;
    if ((st = c->ser_cnt.ensure(n * sizeof(unsigned))) != RSV_OK) return st;
    if ((st = c->ser_dh.ensure(n * sizeof(double))) != RSV_OK) return st;
    if ((st = c->ser_acc.ensure(n * sizeof(int))) != RSV_OK) return st;
    if ((st = c->theta_f.ensure(n * sizeof(MixedTheta))) != RSV_OK) return st;
    if ((st = c->rstats.ensure(n * 2 * sizeof(StatsRec))) != RSV_OK) return st;
    if ((st = c->gibbs.ensure((size_t)gibbs_grid(max_T) * 8 * sizeof(double))) != RSV_OK) return st;
    return RSV_OK;
}

rsv_status rsv_set_integrator(rsv_ctx* c, rsv_integrator kind, double lambda)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    if (kind == RSV_LEAPFROG) {
        c->integrator = 0;
        c->lambda = 0.0;
        return RSV_OK;
    }
    if (kind == RSV_OMELYAN4) {
        c->integrator = 2;
        c->lambda = 0.0;
        return RSV_OK;
    }
    if (kind != RSV_OMELYAN2) return fail(RSV_EINVAL, "unknown integrator");
    if (!(lambda <= 0.5) || lambda != lambda) return fail(RSV_EINVAL, "lambda must be <= 1/2");
    c->integrator = 1;
    c->lambda = lambda > 0.0 ? lambda : RSV_OMELYAN2_LAMBDA;
    return RSV_OK;
}

rsv_status rsv_set_persistent(rsv_ctx* c, int enable)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    c->persistent = enable != 0;
    return RSV_OK;
}

rsv_status rsv_set_wait_limit(rsv_ctx* c, int64_t cycles)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    if (cycles < 0) return fail(RSV_EINVAL, "wait limit must be >= 0");
    c->wait_limit = cycles > 0 ? (long long)cycles : (1LL << 31);
    return RSV_OK;
}

rsv_status rsv_set_leverage(rsv_ctx* c, double rho)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    if (!(rho > -1.0 && rho < 1.0)) return fail(RSV_EINVAL, "rho must be in (-1, 1)");
    c->rho = rho;
    return RSV_OK;
}

rsv_status rsv_set_schedule(rsv_ctx* c, int threads, int sites_per_thread, int64_t tile)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    if (threads == 0 && sites_per_thread == 0 && tile == 0) {
        c->sched_nt = c->sched_j = 0;
        c->sched_tile = 0;
        return RSV_OK;
    }
    if (threads < 32 || threads % 32 || sites_per_thread < 1 || tile < 1)
        return fail(RSV_EINVAL, "bad schedule");
    c->sched_nt = threads;
    c->sched_j = sites_per_thread;
    c->sched_tile = tile;
    return RSV_OK;
}

rsv_status rsv_sync_status(rsv_ctx* c, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int w = 0;
    e = cudaMemcpy(&w, c->ints.as<int>() + kStatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read status");
    e = cudaMemset(c->ints.as<int>() + kStatus, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    if (w & ST_TIMEOUT) return fail(RSV_ETIMEOUT, "a device-side wait ran out of time");
    if (w & ST_NONFINITE) return fail(RSV_ENONFINITE, "a dH was not finite (trajectory rejected)");
    return RSV_OK;
}

rsv_status rsv_action(rsv_ctx* c, const double* h, const double* y, const double* lnrv,
                      int64_t T, rsv_theta theta, double* S_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!h || !y || !lnrv || !S_out) return fail(RSV_EINVAL, "null array argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    if ((st = ctx_ensure_partials(c, action_grid(T))) != RSV_OK) return st;
    ThetaD th = to_dev(theta);
    th.rho = c->rho;
    cudaError_t e = counted(c, launch_action, h, y, lnrv, T, th, c->partials.as<double>(),
                                  reinterpret_cast<unsigned*>(c->ints.as<int>() + kActionCounter),
                                  S_out, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "action kernel");
}

rsv_status rsv_force(rsv_ctx* c, const double* h, const double* y, const double* lnrv,
                     int64_t T, rsv_theta theta, double* F_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!h || !y || !lnrv || !F_out) return fail(RSV_EINVAL, "null array argument");
    if (F_out == h) return fail(RSV_EINVAL, "F_out must not alias h");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    ThetaD th = to_dev(theta);
    th.rho = c->rho;
    cudaError_t e = counted(c, launch_force, h, y, lnrv, T, th, F_out, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "force kernel");
}

rsv_status rsv_draw_momenta(rsv_ctx* c, uint64_t seed, uint64_t series, uint64_t traj,
                            int64_t T, const float* minv, int bits, double* p_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!p_out) return fail(RSV_EINVAL, "null p_out");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1");
    if (bits != 53 && bits != 23) return fail(RSV_EINVAL, "bits must be 53 or 23");
    cudaError_t e = counted(c, launch_draw_momenta, seed, series, traj, T, minv, bits, p_out,
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "momentum kernel");
}

rsv_status rsv_gibbs_theta(rsv_ctx* c, const double* h, const double* lnrv, int64_t T,
                           double* theta, uint64_t seed, uint64_t series, uint64_t traj,
                           int mask, rsv_precision prec, int32_t* phi_acc_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!h || !lnrv || !theta) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1");
    if (mask < 0 || mask > 31) return fail(RSV_EINVAL, "mask must be in 0..31");
    if (prec != RSV_FP64 && prec != RSV_MIXED) return fail(RSV_EINVAL, "bad precision");
    if (c->rho != 0.0)
        return fail(RSV_EINVAL, "the theta update is for the model without leverage (rho = 0)");
    const bool mixed = prec == RSV_MIXED;
    if ((st = c->gibbs.ensure((size_t)gibbs_grid(T) * 8 * sizeof(double))) != RSV_OK) return st;
    if (mixed && ((st = c->fbuf0.ensure((size_t)T * 8)) != RSV_OK ||
                  (st = c->lr_f.ensure((size_t)T * 8)) != RSV_OK ||
                  (st = c->theta_f.ensure(sizeof(MixedTheta))) != RSV_OK))
        return st;
    GibbsArgs g;
    memset(&g, 0, sizeof(g));
    cudaError_t e;
    if (mixed) {
        // the state and lnRV as (hi, lo) FP32 pairs, theta's constants
        if ((e = counted(c, launch_h_to_ff, h, c->fbuf0.as<float2>(), T,
                         (cudaStream_t)stream)) != cudaSuccess ||
            (e = counted(c, launch_h_to_ff, lnrv, c->lr_f.as<float2>(), T,
                         (cudaStream_t)stream)) != cudaSuccess ||
            (e = counted(c, launch_theta_prep, (const double*)theta, ThetaD{}, 1, 0.0,
                         c->theta_f.as<MixedTheta>(), (cudaStream_t)stream)) != cudaSuccess)
            return cuda_fail(e, "theta update set-up");
        g.h0f = c->fbuf0.as<float2>();
        g.lr_f = c->lr_f.as<float2>();
        g.theta_f = c->theta_f.as<MixedTheta>();
    } else {
        g.h0d = h;
        g.lnrv = lnrv;
    }
    g.T = T;
    g.theta = theta;
    g.seed = seed;
    g.series = series;
    g.traj = traj;
    g.mask = mask;
    g.partials = c->gibbs.as<double>();
    g.counter = reinterpret_cast<unsigned*>(c->ints.as<int>() + kGibbsCounter);
    g.phi_acc = phi_acc_out;
    e = counted(c, launch_gibbs, g, mixed, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "theta kernel");
}

rsv_status rsv_ess(rsv_ctx* c, const float* x, int64_t n, int64_t T, float* ess_out,
                   void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!x || !ess_out) return fail(RSV_EINVAL, "null argument");
    if (n < 2 || T < 1) return fail(RSV_EINVAL, "need n >= 2 samples and T >= 1");
    ++c->launches;
    cudaError_t e = launch_ess(x, n, T, ess_out, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "ess kernel");
}

rsv_status rsv_timing(rsv_ctx* c, int enable)
{
    if (!c) return fail(RSV_EINVAL, "null context");
    c->timing = enable != 0;
    return RSV_OK;
}

rsv_status rsv_stats(rsv_ctx* c, int reset, int64_t* launches, int64_t* traj_launches,
                     double* traj_ms)
{
    rsv_status st = ctx_begin(c, nullptr);
    if (st != RSV_OK) return st;
    double ms = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(c->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event sync");
        float m = 0.f;
        e = cudaEventElapsedTime(&m, c->ev[i], c->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event elapsed");
        ms += m;
    }
    if (launches) *launches = c->launches;
    if (traj_launches) *traj_launches = c->traj_launches;
    if (traj_ms) *traj_ms = ms;
    if (reset) {
        c->launches = 0;
        c->traj_launches = 0;
        c->ev_used = 0;
    }
    return RSV_OK;
}

}  // extern "C"
