// rsv_ctx.cuh -- the opaque context behind rsv_ctx* (workspace of one device).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "rsv.h"
#include "rsv_traj.cuh"

namespace rsv {

// A device buffer that only grows.
struct Buf {
    void* ptr = nullptr;
    size_t cap = 0;
    rsv_status ensure(size_t bytes);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Slots of the small int workspace.
enum IntSlot : int {
    kCur = 0,            // chain double-buffer selector
    kFbState = 1,        // [2] mass fallback window counters
    kMassOn = 3,         // 1 while the mass is used
    kStatus = 4,         // status bits (ST_*)
    kTrajCounter = 5,    // arrival counter of trajectory blocks
    kActionCounter = 6,  // arrival counter of the action reduction
    kScratchAcc = 7,     // accept flag when the caller gives none
    kGibbsCounter = 8,   // arrival counter of the theta reduction
    kChainBarrier = 9,   // grid barrier counter of the persistent chain
    kBatchCounter = 16,  // [..] per-call counters of other kernels
    kIntSlots = 64
};
enum ScalSlot : int { kScalDH = 0 };

}  // namespace rsv

struct rsv_plan {
    rsv::Plan plan;
    int device = 0;
};

struct rsv_ctx {
    int device = 0;
    int num_sms = 0;
    // single-series plans, keyed by (T, n_md, precision, mass, schedule)
    struct Cached {
        int64_t T;
        int n_md;
        int integrator;
        double lambda;
        bool mixed, mass, lev;
        int nt, j;
        int64_t tile;
        bool chain;
        rsv::Plan plan;
    };
    std::vector<Cached> plans;
    rsv::Buf ser_cur, ser_cnt, ser_dh, ser_acc;  // per-series scratch
    int sched_nt = 0, sched_j = 0;  // rsv_set_schedule override (0 = automatic)
    int integrator = 0;             // rsv_set_integrator (0 leapfrog)
    double lambda = 0.0;
    double rho = 0.0;               // rsv_set_leverage (0: no leverage)
    int64_t sched_tile = 0;
    bool persistent = true;             // rsv_set_persistent
    long long wait_limit = 1LL << 31;   // rsv_set_wait_limit (clock cycles)
    // accounting: kernel launches, and CUDA events around trajectory kernels
    int64_t launches = 0;
    int64_t traj_launches = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    size_t ev_used = 0;
    rsv::Buf ints;      // int slots
    rsv::Buf scalars;   // double scratch scalars
    rsv::Buf partials;  // per-block partial sums
    rsv::Buf dbuf0, dbuf1;  // FP64 [T] scratch (proposal h', p')
    rsv::Buf fbuf0, fbuf1;  // (hi, lo) FP32 state double buffer
    rsv::Buf a_f, lr_f;  // mixed-path per-site constants
    rsv::Buf theta_f;    // mixed-path per-series theta constants
    rsv::Buf rstats;     // mixed-path statistics of each series' two state buffers
    rsv::Buf gibbs;     // theta-update partial sums
    rsv::Buf batch;     // batched-path scratch
    rsv::Buf extra;     // other kernels' scratch
    std::vector<rsv::Buf*> all_bufs()
    {
        return {&ints, &scalars, &partials, &dbuf0, &dbuf1, &fbuf0, &fbuf1, &a_f, &lr_f, &theta_f,
                &rstats, &gibbs, &batch, &extra, &ser_cur, &ser_cnt, &ser_dh, &ser_acc};
    }
};

namespace rsv {
rsv_status fail(rsv_status st, const char* fmt, ...);
rsv_status cuda_fail(cudaError_t e, const char* what);
bool capture_active();
}  // namespace rsv
