// rsv_api_mlp.cu -- entry points of the learned diagonal mass (include/rsv.h).
#include <cstring>

#include "rsv.h"
#include "rsv_api_common.cuh"
#include "rsv_ctx.cuh"
#include "rsv_mlp.cuh"

using namespace rsv;

extern "C" {

rsv_status rsv_welford_update(rsv_ctx* c, const float* x, int64_t n, int64_t T, int64_t count,
                              double* mean, double* m2, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!x || !mean || !m2) return fail(RSV_EINVAL, "null argument");
    if (n < 1 || T < 1 || count < 0) return fail(RSV_EINVAL, "need n >= 1, T >= 1, count >= 0");
    cudaError_t e = counted(c, launch_welford, x, n, T, count, mean, m2, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "welford kernel");
}

rsv_status rsv_welford_target(rsv_ctx* c, const double* mean, const double* m2, int64_t T,
                              int64_t count, double* hbar_out, float* target_out,
                              float* log_scale_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!mean || !m2 || !target_out) return fail(RSV_EINVAL, "null argument");
    if (T < 1 || count < 2) return fail(RSV_EINVAL, "need T >= 1 and count >= 2");
    cudaError_t e = counted(c, launch_welford_target, mean, m2, T, count, hbar_out, target_out,
                            log_scale_out, (cudaStream_t)stream);
    if (log_scale_out) ++c->launches;
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "welford target kernel");
}

rsv_status rsv_mass_features(rsv_ctx* c, const double* y, const double* lnrv, const double* hbar,
                             int64_t T, rsv_theta theta, float* feat_out, float* stats_out,
                             void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!y || !lnrv || !hbar || !feat_out || !stats_out) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1");
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    const int g = feat_grid(T);
    if ((st = c->batch.ensure((size_t)(g * 20 + 32) * sizeof(double))) != RSV_OK) return st;
    double* part = c->batch.as<double>();
    c->launches += 4;
    cudaError_t e = launch_features(y, lnrv, hbar, T, to_dev(theta), feat_out, stats_out, part + 32,
                                    reinterpret_cast<unsigned*>(c->ints.as<int>() + kBatchCounter + 1),
                                    part, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "feature kernels");
}

static rsv_status mlp_common(rsv_ctx* c, const float* feat, const float* target, int64_t T,
                             int batch)
{
    if (!feat || !target) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1");
    if (T > 0xffffffffLL) return fail(RSV_EINVAL, "T must be < 2^32 for minibatch sampling");
    if (batch < mlp_sites_per_block() || batch % mlp_sites_per_block() || batch > (1 << 24))
        return fail(RSV_EINVAL, "batch must be a positive multiple of %d", mlp_sites_per_block());
    const size_t need = (size_t)(batch / mlp_sites_per_block()) * (mlp_nparam() + 1) * sizeof(float);
    return c->extra.ensure(need);
}

rsv_status rsv_mlp_grad(rsv_ctx* c, const float* feat, const float* target, int64_t T,
                        const float* params, const float* log_scale, uint64_t seed, uint64_t step,
                        int batch, float* grad_out, float* loss_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!params || !grad_out) return fail(RSV_EINVAL, "null argument");
    if ((st = mlp_common(c, feat, target, T, batch)) != RSV_OK) return st;
    cudaError_t e = counted(c, launch_mlp_step, feat, target, T, const_cast<float*>(params),
                            (float*)nullptr, (float*)nullptr, grad_out, c->extra.as<float>(),
                            reinterpret_cast<unsigned*>(c->ints.as<int>() + kBatchCounter),
                            seed, step, (int64_t)1, 0.f, 0.f, 0.f, 0.f, batch, 0, loss_out,
                            log_scale, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "mlp gradient kernel");
}

rsv_status rsv_mlp_train(rsv_ctx* c, const float* feat, const float* target, int64_t T,
                         float* params, const float* log_scale, float* adam_m, float* adam_v,
                         int64_t step0, int n_steps, int batch, uint64_t seed, float lr,
                         float* loss_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!params || !adam_m || !adam_v) return fail(RSV_EINVAL, "null argument");
    if (step0 < 0 || n_steps < 0) return fail(RSV_EINVAL, "negative step");
    if (!(lr > 0.f)) return fail(RSV_EINVAL, "lr must be > 0");
    if ((st = mlp_common(c, feat, target, T, batch)) != RSV_OK) return st;
    for (int i = 0; i < n_steps; ++i) {
        const uint64_t step = (uint64_t)(step0 + i);
        cudaError_t e = counted(c, launch_mlp_step, feat, target, T, params, adam_m, adam_v,
                                (float*)nullptr, c->extra.as<float>(),
                                reinterpret_cast<unsigned*>(c->ints.as<int>() + kBatchCounter),
                                seed, step, (int64_t)(step + 1), lr, 0.9f, 0.999f, 1e-8f, batch, 1,
                                loss_out ? loss_out + i : (float*)nullptr, log_scale,
                                (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "mlp step kernel");
    }
    return RSV_OK;
}

rsv_status rsv_mlp_mass(rsv_ctx* c, const float* feat, int64_t T, const float* params,
                        const float* log_scale, const double* y, const double* hbar,
                        rsv_theta theta, float* minv_out, float* m_out, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!feat || !params || !y || !hbar || !minv_out) return fail(RSV_EINVAL, "null argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1");
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    cudaError_t e = counted(c, launch_mlp_mass, feat, T, params, y, hbar, to_dev(theta), log_scale,
                            minv_out, m_out, (cudaStream_t)stream);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "mlp mass kernel");
}

}  // extern "C"
