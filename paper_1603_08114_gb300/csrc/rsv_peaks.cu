// rsv_peaks.cu -- probe kernels that measure the on-chip peaks the trajectory
// kernels are reported against (not part of the paper's method).
//
// The device-wide copy bandwidth and the BF16 tensor rate are measured
// elsewhere; the mixed trajectory kernel is bound by neither, but by the FP32
// pipe (scalar FFMA and packed FFMA2), the special-function unit (ex2) and
// shared memory, and the FP64 kernel by the FP64 pipe.  Each probe fills every
// SM (four blocks of 512 threads) with independent dependency chains of one
// instruction kind, so that its rate is the pipe's throughput and not its
// latency; the caller times a launch with CUDA events and divides the count of
// operations the call reports by that time.  A result is written only if it
// equals a value no chain reaches, so the chains cannot be removed.
#include <cstdint>

#include "rsv.h"
#include "rsv_api_common.cuh"

namespace rsv {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kChains = 8;               // independent chains per thread
constexpr int kLdsFloat4PerThread = 4;   // shared-memory words a thread cycles over

// FP32 FMA: x = x a + b on kChains chains; one FMA per chain and iteration.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_probe_ffma(int64_t iters, float a, float b, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5f) sink[threadIdx.x] = s;
}

// Packed FP32 FMA (FFMA2): two FP32 FMAs per instruction.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_probe_ffma2(int64_t iters, float a, float b, float* sink)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c - 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1234.5f) sink[threadIdx.x] = s;
}

// 2^x on the special-function unit: x = b - 2^x / 2 (a contraction onto a
// fixed point near -0.15), one ex2 and one FP32 FMA per chain and iteration.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_probe_ex2(int64_t iters, float a, float b, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -0.01f * (c + 1) - threadIdx.x * 1e-6f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float e[kChains];
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e[c]) : "f"(x[c]));
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(e[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5f) sink[threadIdx.x] = s;
}

// Shared-memory loads: each thread reads 16-byte words from a block-wide
// array at an index that moves with the iteration (consecutive lanes,
// consecutive words: no bank conflicts), adding them with packed FP32 adds.
// The loads are volatile: the same four addresses repeat, and plain loads of
// an unchanged address may be merged by the compiler.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_probe_lds(int64_t iters, float a, float b, float* sink)
{
    __shared__ float4 buf[kProbeThreads * kLdsFloat4PerThread];
    for (int i = threadIdx.x; i < kProbeThreads * kLdsFloat4PerThread; i += blockDim.x)
        buf[i] = make_float4(a * i, b, a, b * i);
    __syncthreads();
    float2 s0 = make_float2(0.f, 0.f), s1 = s0;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int idx = (threadIdx.x + (int)((i * 16 + k) & (kLdsFloat4PerThread - 1)) *
                                               kProbeThreads);
            float4 v;
            asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "r"((unsigned)__cvta_generic_to_shared(buf + idx)));
            s0 = __fadd2_rn(s0, make_float2(v.x, v.y));
            s1 = __fadd2_rn(s1, make_float2(v.z, v.w));
        }
    }
    const float s = s0.x + s0.y + s1.x + s1.y;
    if (s == -1234.5f) sink[threadIdx.x] = s;
}

// FP64 FMA on kChains chains.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_probe_dfma(int64_t iters, float a, float b, float* sink)
{
    double x[kChains];
    const double ad = a, bd = b;
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], ad, bd);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5) sink[threadIdx.x] = (float)s;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_pipe_probe(rsv_ctx* c, int kind, int64_t iters, double* ops_out,
                                     void* stream)
{
    rsv_status st = ctx_begin(c, stream);
    if (st != RSV_OK) return st;
    if (!ops_out) return fail(RSV_EINVAL, "null ops_out");
    if (iters < 1 || iters > (int64_t(1) << 40)) return fail(RSV_EINVAL, "iters out of range");
    if (kind < RSV_PROBE_FFMA || kind > RSV_PROBE_DFMA) return fail(RSV_EINVAL, "unknown probe kind");
    if ((st = c->extra.ensure(kProbeThreads * sizeof(float))) != RSV_OK) return st;
    float* sink = c->extra.as<float>();
    const int grid = c->num_sms * kProbeBlocksPerSm;
    const double threads = (double)grid * kProbeThreads;
    const double per_iter = 16.0 * threads;  // instructions per chain slot and iteration
    cudaStream_t s = (cudaStream_t)stream;
    // a < 1 and b keep every chain bounded
    const float a = 0.999f, b = 1e-3f;
    switch (kind) {
        case RSV_PROBE_FFMA:
            k_probe_ffma<<<grid, kProbeThreads, 0, s>>>(iters, a, b, sink);
            *ops_out = per_iter * kChains * (double)iters;
            break;
        case RSV_PROBE_FFMA2:
            k_probe_ffma2<<<grid, kProbeThreads, 0, s>>>(iters, a, b, sink);
            *ops_out = 2.0 * per_iter * kChains * (double)iters;
            break;
        case RSV_PROBE_EX2:
            k_probe_ex2<<<grid, kProbeThreads, 0, s>>>(iters, -0.5f, 0.25f, sink);
            *ops_out = per_iter * kChains * (double)iters;
            break;
        case RSV_PROBE_LDS:
            k_probe_lds<<<grid, kProbeThreads, 0, s>>>(iters, a, b, sink);
            *ops_out = 16.0 * per_iter * (double)iters;  // bytes
            break;
        default:
            k_probe_dfma<<<grid, kProbeThreads, 0, s>>>(iters, a, b, sink);
            *ops_out = per_iter * kChains * (double)iters;
            break;
    }
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "probe kernel");
}
