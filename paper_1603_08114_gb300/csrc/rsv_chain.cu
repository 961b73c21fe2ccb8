// rsv_chain.cu -- a whole chain of mixed-precision HMC trajectories of one
// series (Sec. 3), each followed by the theta sweep, in ONE persistent
// cooperative launch.
//
// The per-trajectory path (rsv_api_hmc.cu) launches the trajectory kernel once
// per trajectory and the theta sweep after it; at T = 2^20 every launch pays
// the launch and tail latency, the last tile of the split series sums all
// tiles' records alone, and the sweep is a launch of its own.  Here every tile
// of the series stays on its SM for the whole chain:
//   per trajectory  the tile's leapfrog (traj_mixed_bin, the same device code
//                   as the per-trajectory kernel), its record (kinetic
//                   difference and end-state statistics) to partials and its
//                   end state as a proposal into the other state buffer;
//   grid barrier    one per trajectory (an arrival counter with a bounded
//                   spin, RSV_ETIMEOUT when it runs out);
//   every block     sums all tiles' records in tile order and takes the
//                   Metropolis decision itself -- the same bits in every block,
//                   so no second barrier broadcasts it -- and the theta sweep
//                   from the statistics of the accepted state (one warp, the
//                   same draws in every block) while its other warps draw the
//                   next trajectory's momenta.
// The records are double-buffered by trajectory parity, so a block that is a
// trajectory ahead never overwrites a record another block is still summing,
// and the state buffers alternate as in the per-trajectory path (a proposal is
// written only to the buffer no block reads in that trajectory).  The results
// are those of the per-trajectory path bit for bit.
#include "rsv_chain.cuh"
#include "rsv_gibbs_dev.cuh"
#include "rsv_traj_dev.cuh"

namespace rsv {
namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: thread 0 of every block adds one to *bar and waits until it
// reaches `target` (the counter only grows: target = generation x grid).  A
// wait longer than `limit` clock cycles sets ST_TIMEOUT and returns false in
// every thread of the block; the kernel then stops.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, long long limit,
                                             int* status, int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        int ok = 1;
        while (ld_acquire_u32(bar) < target) {
            if (clock64() - t0 > limit) {
                ok = 0;
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Momenta of trajectory `traj` for every slot of the block's segment (standard
// normals; the load pass scales them by the mass), drawn by threads t0,
// t0 + step, ...: the slots of owner thread o are sites wlo + o J .. + J - 1,
// Philox4x64-10 counter {site / 4, traj, STREAM_MOM, series}, 23-bit uniforms
// and Box-Muller in FP32, exactly as the per-trajectory kernel draws them.
// Only the Philox blocks idx in [lo, hi) of the segment's owners * J / 4 are
// drawn (hi < 0: all from lo).
template <int J>
__device__ __forceinline__ void draw_slots(const TrajArgs& A, uint64_t traj, const Seg& g,
                                           float* s_ph, int NS, int t0, int step, int lo = 0,
                                           int hi = -1)
{
    constexpr int Q = J / 4;
    const int owners = g.nwarp * 32;
    const int end = hi < 0 ? owners * Q : hi;
    for (int idx = lo + t0; idx < end; idx += step) {
        const int o = idx / Q, q = idx - o * Q;
        const int64_t s0 = g.wlo + (int64_t)o * J + 4 * q;
        const u64x4 r = philox_block(A.seed, (uint64_t)g.series, traj, STREAM_MOM,
                                     (uint64_t)(s0 >> 2));
        float z[4];
        box_muller_f(u01_23(r.w[0]), u01_23(r.w[1]), z[0], z[1]);
        box_muller_f(u01_23(r.w[2]), u01_23(r.w[3]), z[2], z[3]);
        const int owner = g.warp0 * 32 + o;
#pragma unroll
        for (int i = 0; i < 4; ++i) s_ph[(4 * q + i) * NS + owner] = z[i];
    }
}

// The chain's state besides the trajectory body's (shared memory, so that no
// value lives in registers across the body: the body's register pressure
// stays that of the per-trajectory kernel).
struct ChainShared {
    StatsRec rec;          // statistics of the current state
    float th[5];           // theta (FP32-valued once swept)
    double thd[5];         // theta as given (recorded while it is not swept)
    float2 red[kRecWords];
    int ok, fb[2];
    long long i;           // the trajectory about to run / just run
    double u[2];           // the Metropolis uniforms of trajectories of each parity
    Seg g;                 // the block's segment
    int64_t T;
    int nseg, seg0;
};

// s_ph, the momentum rows of the dynamic shared memory (see traj_mixed_bin).
template <int J, bool MASS>
__device__ __forceinline__ float* chain_s_ph(unsigned char* smem_raw)
{
    const int NT = blockDim.x, NS = mixed_row(NT, J);
    return reinterpret_cast<float*>(reinterpret_cast<float2*>(smem_raw) +
                                    (size_t)(2 + (MASS ? 1 : 0)) * (J / 2) * mixed_ntp(NT)) +
           (size_t)2 * NS * J;
}

template <int J, bool MASS>
__device__ __noinline__ void chain_setup(const ChainArgs& C, MixedSmem<false>& S,
                                         ChainShared& Q, unsigned char* smem_raw)
{
    const TrajArgs& A = C.A;
    const int tid = threadIdx.x, NT = blockDim.x;
    const Seg g = A.segs[A.bin_seg[A.bin_first[blockIdx.x]]];
    if (tid < 32) {
        const ff v = ff_from_double(exp2((double)tid / 32.0));
        S.exptab[tid] = make_float2(v.hi, v.lo);
    }
    for (int i = tid; i < NWMAX * 32; i += NT)
        reinterpret_cast<float*>(S.mt)[i] = reinterpret_cast<const float*>(A.theta_f)[i & 31];
    if (tid < 5) {
        Q.thd[tid] = C.theta[tid];
        Q.th[tid] = (float)C.theta[tid];
    }
    if (tid == 0) {
        Q.rec = A.rstats[0];
        Q.fb[0] = Q.fb[1] = 0;
        Q.i = 0;
        Q.g = g;
        Q.T = A.ser[g.series].T;
        Q.nseg = A.ser[g.series].nseg;
        Q.seg0 = A.ser[g.series].seg0;
        Q.u[0] = metropolis_u(A.seed, g.series, C.traj0);
        S.cur = 0;
        S.mass_on = MASS ? 1 : 0;
    }
    draw_slots<J>(A, C.traj0, g, chain_s_ph<J, MASS>(smem_raw), mixed_row(NT, J), tid, NT);
    // the block's view, filed for every trajectory of the chain
    View v;
    load_bin<false>(A, blockIdx.x, S.wseg, S.wacc, v, S.wg, S.wsi, S.wcur);
    __syncthreads();
}

// After trajectory Q.i: the grid barrier, the decision, the theta sweep and
// the next momenta; returns false if a barrier wait ran out.  Warps 0..7 sum
// the tiles' records (one value each; named barrier 1 joins them), thread 0
// decides and warp 0 then sweeps theta, while warps 8.. and then 1..7 draw
// the next trajectory's momenta (a block of fewer than 9 warps does the steps
// one after the other).  Not inlined: inside the trajectory loop its
// loop-invariant values (Philox and sweep constants, addresses) would be
// hoisted out of the loop and held in registers through the leapfrog, which
// then runs ~10 % slower.
template <int J, bool MASS>
__device__ __noinline__ bool chain_after(const ChainArgs& C, MixedSmem<false>& S,
                                         ChainShared& Q, unsigned char* smem_raw)
{
    static_assert(kRecWords == 8, "warps 0..7 sum one record value each");
    const TrajArgs& A = C.A;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const int nw = NT >> 5;
    const bool split = nw > kRecWords;  // warps 8.. draw momenta meanwhile
    const long long i = Q.i;
    const bool more = i + 1 < C.n_traj;
    const uint64_t traj = C.traj0 + (uint64_t)i;
    float* s_ph = chain_s_ph<J, MASS>(smem_raw);
    const int NS = mixed_row(NT, J);
    if (!grid_barrier(C.bar, (unsigned)(i + 1) * gridDim.x, C.wait_limit, A.status, &Q.ok))
        return false;
    // the next momenta (Philox blocks [0, mom_split) by warps 8.., which start
    // at once, the rest by warps 1..7 after their share of the record sum):
    // twice the blocks per thread for the early warps
    const int mom_total = Q.g.nwarp * 32 * (J / 4);
    const int n_early = NT - 32 * kRecWords, n_late = 32 * (kRecWords - 1);
    const int mom_split =
        split ? (int)((int64_t)mom_total * 2 * n_early / (2 * n_early + n_late)) : mom_total;
    if (warp < kRecWords) {
        // every tile's record value f in tile order (lane l takes tiles l,
        // l + 32, ...; then a butterfly) -- the same order in every block;
        // warp w sums the values f = w, w + nw, ... (one each when the block
        // has 8 warps or more)
        const float2* pf = reinterpret_cast<const float2*>(S.partials);
        const int nseg = Q.nseg, seg0 = Q.seg0;
        for (int f = warp; f < kRecWords; f += nw) {
            ff sum = {0.f, 0.f};
            for (int i0 = lane; i0 < nseg; i0 += 32 * 8) {
                float2 w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    w[u] = i0 + 32 * u < nseg
                               ? __ldcg(pf + (int64_t)(seg0 + i0 + 32 * u) * kPartialWords + f)
                               : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + 32 * u < nseg) sum = ff_add(sum, ff{w[u].x, w[u].y});
            }
            sum = warp_sum_ff(sum);
            if (lane == 0) Q.red[f] = make_float2(sum.hi, sum.lo);
        }
        if (split) asm volatile("bar.sync 1, %0;" ::"r"(kRecWords * 32) : "memory");
        else __syncthreads();
        // warps 1..7 then join the momenta (warp 0 decides and sweeps)
        if (split && more && warp > 0)
            draw_slots<J>(A, traj + 1, Q.g, s_ph, NS, tid - 32, 32 * (kRecWords - 1), mom_split);
    } else {
        if (more) draw_slots<J>(A, traj + 1, Q.g, s_ph, NS, tid - 32 * kRecWords,
                                NT - 32 * kRecWords, 0, mom_split);
    }
    if (!split) __syncthreads();  // (the reducing warps passed one already)
    if (tid == 0) {
        const MixedTheta& mt = S.mt[0];
        ff dk;
        StatsRec r1;
        rec_from(Q.red, dk, r1.s);
        r1.mu = mt.mu;
        r1.ximu = mt.ximu;
        r1.sl = Q.rec.sl;
        r1.sll = Q.rec.sll;
        const double dH = stats_dH(dk, r1.s, Q.rec, mt, Q.T);
        const int acc = metropolis_accept_u(Q.u[i & 1], dH);
        if (acc) {
            Q.rec = r1;
            S.cur ^= 1;
        }
        if (blockIdx.x == 0) {
            if (!isfinite(dH)) atomicOr(A.status, ST_NONFINITE);
            if (C.dH_out) C.dH_out[i] = dH;
            if (C.acc_out) C.acc_out[i] = acc;
        }
        if (MASS && C.fallback_window > 0) {
            int na = Q.fb[0] + acc, nt = Q.fb[1] + 1;
            if (nt >= C.fallback_window) {
                if (S.mass_on && 10 * na < 6 * nt) S.mass_on = 0;
                na = nt = 0;
            }
            Q.fb[0] = na;
            Q.fb[1] = nt;
        }
    }
    if (warp == 0) {
        __syncwarp();
        if (C.update_theta) {
            // the theta sweep from the accepted state's statistics
            float th[5], tot[NSTAT], x0;
#pragma unroll
            for (int k = 0; k < 5; ++k) th[k] = Q.th[k];
            record_sums(Q.rec, th, Q.T, tot, x0);
            WarpDrawsF st;
            st.seed = A.seed;
            st.series = (uint64_t)Q.g.series;
            st.traj = traj;
            st.fill(Q.T);
            int phi_acc = 0;
            gibbs_draws_f(tot, x0, Q.T, th, st, 31, &phi_acc);
            if (lane < 5) {
                float v = th[0];
#pragma unroll
                for (int k = 1; k < 5; ++k)
                    if (lane == k) v = th[k];
                Q.th[lane] = v;
                if (blockIdx.x == 0) {
                    C.theta[lane] = (double)v;
                    if (C.theta_out) C.theta_out[5 * i + lane] = (double)v;
                }
            }
            if (lane == 0) S.mt[0] = mixed_theta_f(th);
        } else if (blockIdx.x == 0 && C.theta_out && lane < 5) {
            C.theta_out[5 * i + lane] = Q.thd[lane];
        }
    }
    // the next test's uniform, off the critical path where there is a warp 1
    if (more && tid == (nw > 1 ? 32 : 0))
        Q.u[(i + 1) & 1] = metropolis_u(A.seed, Q.g.series, traj + 1);
    __syncthreads();
    if (!split && more) {  // a small block draws the momenta after the sweep
        draw_slots<J>(A, traj + 1, Q.g, s_ph, NS, tid, NT);
        __syncthreads();
    }
    if (C.update_theta)
        for (int k = tid + 32; k < nw * 32; k += NT)
            reinterpret_cast<float*>(S.mt)[k] = reinterpret_cast<const float*>(S.mt)[k & 31];
    if (tid == 0) Q.i = i + 1;
    __syncthreads();
    return true;
}

template <int J, bool MASS>
__global__ void __launch_bounds__(mixed_ntmax<J, MASS>(), 1)
    k_chain_mixed(const __grid_constant__ ChainArgs C)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MixedSmem<false> S;
    __shared__ ChainShared Q;
    chain_setup<J, MASS>(C, S, Q, smem_raw);
    for (;;) {
        const long long i = Q.i;
        if (i >= C.n_traj) break;
        // this trajectory's records go to the half of partials of its parity
        // (set before the body's first block barrier, read after its last)
        if (threadIdx.x == 0) S.partials = C.partials + (i & 1) * (int64_t)C.nsegs * kPartialWords;
        // the snapshot of the state this trajectory starts from, if due
        float* snap_prev = (C.snaps && i > 0 && i % C.thin == 0)
                               ? C.snaps + (size_t)(i / C.thin - 1) * (size_t)Q.T
                               : nullptr;
        traj_mixed_bin<J, MASS, false, true>(C.A, blockIdx.x, S, smem_raw, snap_prev);
        if (!chain_after<J, MASS>(C, S, Q, smem_raw)) return;
    }
    // the last snapshot, if due, and the final state selector and mass flag
    if (C.snaps && C.n_traj > 0 && C.n_traj % C.thin == 0) {
        const float2* hc = S.cur ? C.A.h1f : C.A.h0f;
        float* dst = C.snaps + (size_t)(C.n_traj / C.thin - 1) * (size_t)Q.T;
        const int64_t off = C.A.ser[Q.g.series].off;
        for (int64_t s = Q.g.lo + threadIdx.x; s < Q.g.hi; s += blockDim.x) {
            const float2 hv = __ldcg(hc + off + s);
            dst[off + s] = hv.x + hv.y;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        C.ser_cur_out[Q.g.series] = S.cur;
        if (C.mass_on_out) *C.mass_on_out = S.mass_on;
    }
}

// Whether every block of the plan can be resident at once (the grid barrier
// waits for all of them).
template <int J, bool MASS>
cudaError_t chain_fits_j(const Plan& p, int num_sms, bool* fits)
{
    auto k = k_chain_mixed<J, MASS>;
    *fits = false;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p.nt, p.smem);
    if (e != cudaSuccess) return e;
    *fits = (int64_t)per_sm * num_sms >= p.nbins;
    return cudaSuccess;
}

template <int J, bool MASS>
cudaError_t launch_chain_j(const ChainArgs& c, const Plan& p, int num_sms, cudaStream_t st,
                           bool* launched)
{
    auto k = k_chain_mixed<J, MASS>;
    bool fits = false;
    cudaError_t e = chain_fits_j<J, MASS>(p, num_sms, &fits);
    if (e != cudaSuccess) return e;
    if (!fits) {
        *launched = false;
        return cudaSuccess;
    }
    ChainArgs a = c;
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)k, dim3(p.nbins), dim3(p.nt), args, p.smem, st);
    *launched = e == cudaSuccess;
    return e;
}

}  // namespace

bool chain_supported(const Plan& p)
{
    return p.mixed && !p.lev && p.nseries == 1 && p.grid == p.nbins &&
           (p.j == 4 || p.j == 8 || p.j == 12 || p.j == 16 || p.j == 20);
}

cudaError_t chain_fits(const Plan& p, int num_sms, bool* fits)
{
    *fits = false;
    if (!chain_supported(p)) return cudaSuccess;
#define RSV_CF(JJ)                                                                        \
    case JJ:                                                                              \
        return p.mass ? chain_fits_j<JJ, true>(p, num_sms, fits)                          \
                      : chain_fits_j<JJ, false>(p, num_sms, fits);
    switch (p.j) {
        RSV_CF(4)
        RSV_CF(8)
        RSV_CF(12)
        RSV_CF(16)
        RSV_CF(20)
        default: return cudaSuccess;
    }
#undef RSV_CF
}

cudaError_t launch_chain(const ChainArgs& c, const Plan& p, int num_sms, cudaStream_t st,
                         bool* launched)
{
    *launched = false;
#define RSV_CH(JJ)                                                                        \
    case JJ:                                                                              \
        return p.mass ? launch_chain_j<JJ, true>(c, p, num_sms, st, launched)             \
                      : launch_chain_j<JJ, false>(c, p, num_sms, st, launched);
    switch (p.j) {
        RSV_CH(4)
        RSV_CH(8)
        RSV_CH(12)
        RSV_CH(16)
        RSV_CH(20)
        default: return cudaSuccess;
    }
#undef RSV_CH
}

}  // namespace rsv
