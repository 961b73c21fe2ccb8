// rsv_api_common.cuh -- helpers shared by the entry-point files of librsv.
#pragma once

#include <cuda_runtime.h>

#include "rsv.h"
#include "rsv_ctx.cuh"
#include "rsv_device.cuh"

namespace rsv {

bool theta_ok(const rsv_theta& t);
ThetaD to_dev(const rsv_theta& t);
// Bind the context's device and remember the caller's stream (for capture checks).
rsv_status ctx_begin(rsv_ctx* c, void* stream);
rsv_status ctx_ensure_partials(rsv_ctx* c, int64_t n);

// Count a kernel launch made through launcher f.
template <class F, class... A>
cudaError_t counted(rsv_ctx* c, F f, A... a)
{
    ++c->launches;
    return f(a...);
}

}  // namespace rsv
