// rsv_dfexp.cu -- the exponentials of the trajectory kernels, exposed for
// tests: the mixed path's double-float ff_exp (one double-float) and its
// two-lane form ff2_exp (the end-of-trajectory statistics), and the FP64
// path's table-driven exp_tab, evaluated at given arguments.  Not steps of
// the method; the tests compare them with exp in FP64.
#include <algorithm>
#include <cstdint>

#include "rsv.h"
#include "rsv_api_common.cuh"
#include "rsv_traj_dev.cuh"

namespace rsv {
namespace {

constexpr int kDfThreads = 256;

// Thread i takes arguments 2i and 2i + 1: ff_exp of each, and ff2_exp of the
// two as one pair (an odd n leaves the last pair's second lane at t = 0).
__global__ void __launch_bounds__(kDfThreads) k_ff_exp(const double* __restrict__ t, int64_t n,
                                                       double* __restrict__ out,
                                                       double* __restrict__ out2)
{
    __shared__ float2 tab[32];
    if (threadIdx.x < 32) {
        const ff v = ff_from_double(exp2((double)threadIdx.x / 32.0));
        tab[threadIdx.x] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    const int64_t npair = (n + 1) / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npair;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = 2 * i, i1 = 2 * i + 1;
        const ff a = ff_from_double(t[i0]);
        const ff b = i1 < n ? ff_from_double(t[i1]) : ff{0.f, 0.f};
        if (out) {
            const ff ea = ff_exp(a, tab);
            out[i0] = ff_to_double(ea);
            if (i1 < n) out[i1] = ff_to_double(ff_exp(b, tab));
        }
        if (out2) {
            const ff2 e = ff2_exp(ff2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}, tab);
            out2[i0] = (double)e.hi.x + (double)e.lo.x;
            if (i1 < n) out2[i1] = (double)e.hi.y + (double)e.lo.y;
        }
    }
}

// exp_tab (the FP64 trajectory kernel's exponential) at each argument.
__global__ void __launch_bounds__(kDfThreads) k_exp_tab(const double* __restrict__ t, int64_t n,
                                                        double* __restrict__ out)
{
    __shared__ double tab[kExpTabN];
    if (threadIdx.x < kExpTabN) tab[threadIdx.x] = kExp2Tab[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = exp_tab(t[i], tab);
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_ff_exp(rsv_ctx* c, const double* t, double* out, double* out2, int64_t n,
                                 void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (n < 0) return fail(RSV_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return RSV_OK;
    if (!t) return fail(RSV_EINVAL, "null t");
    const int64_t npair = (n + 1) / 2;
    const int grid = (int)std::min<int64_t>((npair + kDfThreads - 1) / kDfThreads, 4 * (int64_t)c->num_sms);
    k_ff_exp<<<grid, kDfThreads, 0, (cudaStream_t)stream>>>(t, n, out, out2);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "k_ff_exp");
}

extern "C" rsv_status rsv_fp64_exp(rsv_ctx* c, const double* t, double* out, int64_t n, void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (n < 0) return fail(RSV_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return RSV_OK;
    if (!t || !out) return fail(RSV_EINVAL, "null t or out");
    const int grid = (int)std::min<int64_t>((n + kDfThreads - 1) / kDfThreads, 4 * (int64_t)c->num_sms);
    k_exp_tab<<<grid, kDfThreads, 0, (cudaStream_t)stream>>>(t, n, out);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "k_exp_tab");
}
