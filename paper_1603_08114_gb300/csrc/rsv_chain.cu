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
template <int J>
__device__ __forceinline__ void draw_slots(const TrajArgs& A, uint64_t traj, const Seg& g,
                                           float* s_ph, int NS, int t0, int step)
{
    constexpr int Q = J / 4;
    const int owners = g.nwarp * 32;
    for (int idx = t0; idx < owners * Q; idx += step) {
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

template <int J, bool MASS>
__global__ void __launch_bounds__(mixed_ntmax<J, MASS>(), 1) k_chain_mixed(const ChainArgs C)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MixedSmem<false> S;
    __shared__ StatsRec s_rec;   // statistics of the current state
    __shared__ float s_th[5];    // theta (FP32-valued once swept)
    __shared__ double s_thd[5];  // theta as given (recorded while it is not swept)
    __shared__ float2 s_red[kRecWords];
    __shared__ int s_ok, s_fb[2];
    const TrajArgs& A = C.A;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const int nw = NT >> 5, NS = mixed_row(NT, J);
    constexpr int P = J / 2;
    // s_ph, the momentum row of the dynamic shared memory (see traj_mixed_bin)
    float* s_ph = reinterpret_cast<float*>(reinterpret_cast<float2*>(smem_raw) +
                                           (size_t)(2 + (MASS ? 1 : 0)) * P * NT) +
                  (size_t)2 * NS * J;
    const int b = blockIdx.x;
    const Seg g = A.segs[A.bin_seg[A.bin_first[b]]];
    const int64_t T = A.ser[g.series].T;
    const int nseg = A.ser[g.series].nseg, seg0 = A.ser[g.series].seg0;

    if (tid < 32) {
        const ff v = ff_from_double(exp2((double)tid / 32.0));
        S.exptab[tid] = make_float2(v.hi, v.lo);
    }
    for (int i = tid; i < NWMAX * 32; i += NT)
        reinterpret_cast<float*>(S.mt)[i] = reinterpret_cast<const float*>(A.theta_f)[i & 31];
    if (tid < 5) {
        s_thd[tid] = C.theta[tid];
        s_th[tid] = (float)C.theta[tid];
    }
    if (tid == 0) {
        s_rec = A.rstats[0];
        S.cur = 0;
        S.mass_on = MASS ? 1 : 0;
        s_fb[0] = s_fb[1] = 0;
    }
    draw_slots<J>(A, C.traj0, g, s_ph, NS, tid, NT);
    __syncthreads();

    for (int64_t i = 0; i < C.n_traj; ++i) {
        const uint64_t traj = C.traj0 + (uint64_t)i;
        // records of this trajectory: the half of partials of its parity (set
        // before the trajectory's first block barrier, read after its last)
        if (tid == 0) S.partials = C.partials + (i & 1) * (int64_t)C.nsegs * kPartialWords;
        // the snapshot of the state this trajectory starts from, if due
        float* snap_prev = (C.snaps && i > 0 && i % C.thin == 0)
                               ? C.snaps + (size_t)(i / C.thin - 1) * (size_t)T
                               : nullptr;
        traj_mixed_bin<J, MASS, false, true>(A, b, S, smem_raw, snap_prev);
        if (!grid_barrier(C.bar, (unsigned)(i + 1) * gridDim.x, C.wait_limit, A.status, &s_ok))
            return;
        // every tile's record in tile order (warp f sums value f; lane l takes
        // tiles l, l + 32, ...; then a butterfly) -- the same order in every block
        {
            const float2* pf = reinterpret_cast<const float2*>(S.partials);
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
                if (lane == 0) s_red[f] = make_float2(sum.hi, sum.lo);
            }
        }
        __syncthreads();
        if (tid == 0) {
            const MixedTheta& mt = S.mt[0];
            ff dk;
            StatsRec r1;
            rec_from(s_red, dk, r1.s);
            r1.mu = mt.mu;
            r1.ximu = mt.ximu;
            r1.sl = s_rec.sl;
            r1.sll = s_rec.sll;
            const double dH = stats_dH(dk, r1.s, s_rec, mt, T);
            const int acc = metropolis_accept(nullptr, A.seed, g.series, traj, dH);
            if (acc) {
                s_rec = r1;
                S.cur ^= 1;
            }
            if (b == 0) {
                if (!isfinite(dH)) atomicOr(A.status, ST_NONFINITE);
                if (C.dH_out) C.dH_out[i] = dH;
                if (C.acc_out) C.acc_out[i] = acc;
            }
            if (MASS && C.fallback_window > 0) {
                int na = s_fb[0] + acc, nt = s_fb[1] + 1;
                if (nt >= C.fallback_window) {
                    if (S.mass_on && 10 * na < 6 * nt) S.mass_on = 0;
                    na = nt = 0;
                }
                s_fb[0] = na;
                s_fb[1] = nt;
            }
        }
        __syncthreads();
        const bool more = i + 1 < C.n_traj;
        if (C.update_theta) {
            // warp 0: the theta sweep from the accepted state's statistics;
            // the other warps: the next trajectory's momenta meanwhile
            if (warp == 0) {
                float th[5], tot[NSTAT], x0;
#pragma unroll
                for (int k = 0; k < 5; ++k) th[k] = s_th[k];
                record_sums(s_rec, th, T, tot, x0);
                WarpDrawsF st;
                st.seed = A.seed;
                st.series = (uint64_t)g.series;
                st.traj = traj;
                st.fill(T);
                int phi_acc = 0;
                gibbs_draws_f(tot, x0, T, th, st, 31, &phi_acc);
                if (lane < 5) {
                    float v = th[0];
#pragma unroll
                    for (int k = 1; k < 5; ++k)
                        if (lane == k) v = th[k];
                    s_th[lane] = v;
                    if (b == 0) {
                        C.theta[lane] = (double)v;
                        if (C.theta_out) C.theta_out[5 * i + lane] = (double)v;
                    }
                }
                if (lane == 0) S.mt[0] = mixed_theta_f(th);
                if (!more || nw == 1) {
                    if (more) draw_slots<J>(A, traj + 1, g, s_ph, NS, lane, 32);
                }
            } else if (more) {
                draw_slots<J>(A, traj + 1, g, s_ph, NS, tid - 32, NT - 32);
            }
            __syncthreads();
            for (int k = tid + 32; k < nw * 32; k += NT)
                reinterpret_cast<float*>(S.mt)[k] = reinterpret_cast<const float*>(S.mt)[k & 31];
        } else {
            if (b == 0 && C.theta_out && tid < 5) C.theta_out[5 * i + tid] = s_thd[tid];
            if (more) draw_slots<J>(A, traj + 1, g, s_ph, NS, tid, NT);
        }
        __syncthreads();
    }

    // the last snapshot, if due, and the final state selector and mass flag
    if (C.snaps && C.n_traj > 0 && C.n_traj % C.thin == 0) {
        const float2* hc = S.cur ? A.h1f : A.h0f;
        float* dst = C.snaps + (size_t)(C.n_traj / C.thin - 1) * (size_t)T;
        const int64_t off = A.ser[g.series].off;
        for (int64_t s = g.lo + tid; s < g.hi; s += NT) {
            const float2 hv = __ldcg(hc + off + s);
            dst[off + s] = hv.x + hv.y;
        }
    }
    if (b == 0 && tid == 0) {
        C.ser_cur_out[g.series] = S.cur;
        if (C.mass_on_out) *C.mass_on_out = S.mass_on;
    }
}

template <int J, bool MASS>
cudaError_t launch_chain_j(const ChainArgs& c, const Plan& p, int num_sms, cudaStream_t st,
                           bool* launched)
{
    auto k = k_chain_mixed<J, MASS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p.nt, p.smem);
    if (e != cudaSuccess) return e;
    // every tile must be resident at once (the grid barrier waits for all)
    if ((int64_t)per_sm * num_sms < p.nbins) {
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
