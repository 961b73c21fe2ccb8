// rsv_noalloc.cu -- S(h) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is
// being captured (an allocation there is not captured and breaks the graph's
// replay), plug-ins that run inside a host application that owns the device
// memory pool and forbids other allocations, and hard real-time loops that must
// not block on the allocator.  rsv_action_noalloc gives them the action S(h)
// without a context: the reduction's scratch (one partial sum per block and
// the arrival counter of the last-block reduction) lives in a fixed array in
// device memory, created when the library is loaded on a device and kept until
// the process exits.  The sum is the same as rsv_action's; only the scratch
// and the number of blocks (one per 2048 sites) differ.
#include <cmath>
#include <mutex>

#include "rsv.h"
#include "rsv_api_common.cuh"
#include "rsv_device.cuh"

namespace rsv {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int64_t kNoallocSitesPerBlock = 2048;    // 8 sites per thread
constexpr int kNoallocMaxBlocks = 4096;            // => T <= 8,388,608
constexpr size_t kNoallocBytes = kNoallocMaxBlocks * sizeof(double) + 256;

// One partial sum per block, then (at byte offset kNoallocMaxBlocks * 8) the
// arrival counter.  Every call on a device shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The array's device address is looked up once per device context and
// cached with that context's unique id: cudaDeviceReset destroys the device's
// context, the module is loaded again into the next one and the array may move,
// so a cached address is used only while the current context is the one it was
// looked up in.
std::mutex g_noalloc_mu;
struct NoallocSlot {
    unsigned long long ctx_id;  // 0 = none
    void* ptr;
};
NoallocSlot g_noalloc_slot[64] = {};

// Driver entry points for the current context's id (cuCtxGetCurrent and
// cuCtxGetId, CUDA >= 12.0), fetched through the runtime so that the library
// does not link libcuda itself.  Their CUresult is returned as int (0 = OK).
typedef int (*PfnCtxGetCurrent)(void** ctx);
typedef int (*PfnCtxGetId)(void* ctx, unsigned long long* id);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
bool g_ctx_fns_tried = false;

// Unique id of the calling thread's current context, or 0 when there is none
// or the driver cannot tell (then the address is looked up on every call).
unsigned long long current_ctx_id()
{
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f);
        (void)cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || ctx == nullptr) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

__global__ void __launch_bounds__(kNoallocThreads) k_action_noalloc(
    const double* __restrict__ h, const double* __restrict__ y, const double* __restrict__ lnrv,
    int64_t T, ThetaD th, unsigned char* __restrict__ scratch, double* __restrict__ S_out)
{
    __shared__ double red[32];
    __shared__ int s_last;
    double* partials = reinterpret_cast<double*>(scratch);
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoallocMaxBlocks * sizeof(double));
    const double phi = th.phi, mu = th.mu, ie = 1.0 / th.se2, iu = 1.0 / th.su2;
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double ht = h[t], yt = y[t];
        const double r = lnrv[t] - th.xi - ht;
        double s = 0.5 * ht + 0.5 * yt * yt * exp(-ht) + 0.5 * iu * r * r;
        const double x = ht - mu;
        if (t + 1 < T) {
            const double e = (h[t + 1] - mu) - phi * x;
            s += 0.5 * ie * e * e;
        }
        if (t == 0) s += 0.5 * ie * (1.0 - phi * phi) * x * x;
        acc += s;
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
    const double S = block_sum(v, red);
    if (threadIdx.x == 0) {
        *S_out = S;
        *counter = 0u;
    }
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_action_noalloc(const double* h, const double* y, const double* lnrv,
                                         int64_t T, rsv_theta theta, double* S_out, void* stream)
{
    if (!h || !y || !lnrv || !S_out) return fail(RSV_EINVAL, "null array argument");
    if (T < 1) return fail(RSV_EINVAL, "T must be >= 1 (got %lld)", (long long)T);
    const int64_t max_T = kNoallocSitesPerBlock * kNoallocMaxBlocks;
    if (T > max_T)
        return fail(RSV_EINVAL, "T = %lld exceeds the %lld sites that the fixed scratch of "
                    "rsv_action_noalloc covers; use rsv_action", (long long)T, (long long)max_T);
    if (!theta_ok(theta)) return fail(RSV_EINVAL, "invalid theta");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(RSV_EINVAL, "device index %d not supported", dev);
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        NoallocSlot& slot = g_noalloc_slot[dev];
        const unsigned long long id = current_ctx_id();
        if (id != 0 && slot.ctx_id == id) {
            ptr = slot.ptr;
        } else {
            // set-up on this device (the current one): the first call, or the
            // first in a new context (after a device reset)
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                slot = NoallocSlot{0, nullptr};
                return cuda_fail(e, "cudaGetSymbolAddress of the fixed scratch");
            }
            // the lookup made the device's context current if none was
            slot = NoallocSlot{current_ctx_id(), ptr};
        }
    }
    unsigned char* scratch = static_cast<unsigned char*>(ptr);
    cudaStream_t st = (cudaStream_t)stream;
    // the arrival counter must start at zero (a previous call leaves it at 0,
    // but an interrupted one may not)
    e = cudaMemsetAsync(scratch + kNoallocMaxBlocks * sizeof(double), 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    const int grid = (int)((T + kNoallocSitesPerBlock - 1) / kNoallocSitesPerBlock);
    k_action_noalloc<<<grid, kNoallocThreads, 0, st>>>(h, y, lnrv, T, to_dev(theta), scratch,
                                                       S_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "action kernel (fixed scratch)");
}
