// rsv_plan.cu -- host-side work plan of the trajectory kernels.
//
// A plan fixes the block shape (threads nt, sites per thread j; the window of
// a block is W = nt * j sites) and cuts the series into segments placed in
// bins:
//  - a series that fits a window (and, for a single series, that the cost
//    model keeps whole) is one segment on ceil(T / (32 j)) whole warps; such
//    segments are packed side by side into bins first-fit-decreasing;
//  - a longer series is cut into tiles of `tile` owned sites, each with a
//    halo of K = (force evaluations per trajectory) + 1 sites per side, one
//    tile per bin.
// Segment ids run series by series so that the tiles of one series are
// consecutive (their partial dH are summed in that order).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "rsv_traj.cuh"

namespace rsv {

namespace {

const int kJ_fp64[] = {4, 8, 16, 28};
const int kJ_mixed[] = {4, 8, 12, 16, 20};
const int kNJ_fp64 = 4, kNJ_mixed = 5;

// mixed: (a, k) float2 + x0 (hi, lo) + p0 per site (+ dtau/m with a mass,
// + the leverage v with leverage), the start state in j rows of
// mixed_row(nt, j) slots each; FP64:
// a' (or y e^{-mu/2}), kc (+ 1/m) per site
size_t smem_for(bool mixed, bool mass, bool lev, int nt, int j)
{
    if (mixed)
        return ((2 + (mass ? 1 : 0) + (lev ? 1 : 0)) * (size_t)mixed_ntp(nt) +
                3 * (size_t)mixed_row(nt, j)) *
               (size_t)j * sizeof(float);
    return (2 + (mass ? 1 : 0)) * (size_t)nt * (size_t)j * sizeof(double);
}

bool valid_j(bool mixed, int j)
{
    const int* js = mixed ? kJ_mixed : kJ_fp64;
    const int n = mixed ? kNJ_mixed : kNJ_fp64;
    for (int i = 0; i < n; ++i)
        if (js[i] == j) return true;
    return false;
}

int ntmax(bool mixed, bool mass, int j) { return mixed ? mixed_max_threads(j, mass) : 256; }

}  // namespace

void free_plan(Plan& p)
{
    if (p.d_segs) cudaFree(p.d_segs);
    if (p.d_bin_first) cudaFree(p.d_bin_first);
    if (p.d_bin_seg) cudaFree(p.d_bin_seg);
    if (p.d_ser) cudaFree(p.d_ser);
    p = Plan();
}

bool make_plan(const int64_t* off, int n, int n_md, int integrator, double lambda, bool mixed,
               bool mass, bool lev, int num_sms, int sched_nt, int sched_j, int64_t sched_tile,
               Plan& P, const char** why, bool chain)
{
    // one site of staleness per force evaluation
    const int64_t K = (int64_t)n_md * make_scheme(integrator, lambda).nk + 1;
    const size_t smem_cap = 227 * 1024;
    if (n < 1) {
        *why = "no series";
        return false;
    }
    int64_t Tmax = 0;
    for (int s = 0; s < n; ++s) {
        const int64_t T = off[s + 1] - off[s];
        if (T < 1) {
            *why = "every series needs T >= 1";
            return false;
        }
        Tmax = std::max(Tmax, T);
    }

    // ---- block shape and tile ----------------------------------------------
    int nt = 0, j = 0;
    int64_t tile = 0;
    if (sched_nt > 0) {
        // a single series no longer than the tile is kept whole: it needs the
        // window only, no halo
        const bool whole1 = n == 1 && sched_tile >= Tmax && Tmax <= (int64_t)sched_nt * sched_j;
        if (!valid_j(mixed, sched_j) || sched_nt % 32 || sched_nt > ntmax(mixed, mass, sched_j) ||
            sched_tile < 1 || (!whole1 && sched_tile + 2 * K + 3 > (int64_t)sched_nt * sched_j) ||
            smem_for(mixed, mass, lev, sched_nt, sched_j) > smem_cap) {
            *why = "the fixed schedule does not fit this call";
            return false;
        }
        nt = sched_nt;
        j = sched_j;
        tile = sched_tile;
    } else if (n == 1) {
        // one series: fewest waves of the smallest windows (latency per
        // trajectory ~ sites per thread), whole if one window holds it
        const int64_t T = Tmax;
        double best = 1e300;
        const int* js = mixed ? kJ_mixed : kJ_fp64;
        const int nj = mixed ? kNJ_mixed : kNJ_fp64;
        for (int ji = 0; ji < nj; ++ji) {
            const int tmax = ntmax(mixed, mass, js[ji]);
            for (int t = 32; t <= tmax; t += 32) {
                const int64_t cap = (int64_t)t * js[ji];
                if (smem_for(mixed, mass, lev, t, js[ji]) > smem_cap) continue;
                const int64_t tl = cap - 2 * K - 3;
                int64_t bins;
                int64_t use_tile;
                if (T <= cap) {
                    bins = 1;
                    use_tile = T;
                } else {
                    if (tl < 1) continue;
                    bins = (T + tl - 1) / tl;
                    use_tile = tl;
                }
                // also consider splitting a series that would fit
                for (int pass = 0; pass < 2; ++pass) {
                    int64_t b = bins, ut = use_tile;
                    if (pass == 1) {
                        if (T <= cap && tl >= 1 && tl < T) {
                            b = (T + tl - 1) / tl;
                            ut = tl;
                        } else {
                            continue;
                        }
                    }
                    // blocks resident per SM share it: an SM's work per wave
                    // is bps windows
                    int bps = blocks_per_sm(mixed, mass, lev, js[ji], t,
                                            smem_for(mixed, mass, lev, t, js[ji]));
                    if (bps < 1) continue;
                    const int64_t waves = (b + (int64_t)num_sms * bps - 1) / ((int64_t)num_sms * bps);
                    double cost = (double)waves * (double)cap * bps;
                    // measured on the mixed kernel at T = 2^20 (fixed and
                    // per-step cost per block shape): J = 12 with ~600
                    // threads is the fastest, J = 20 close, J = 16 and 8
                    // slower; inside the persistent chain (78 steps, mass,
                    // every state recorded) J = 20 with 384 threads is the
                    // fastest, 89.5 us per trajectory against 92.1 for
                    // J = 16 (448 threads) and 91.9 for J = 12 (608): per
                    // site of a window 0.0117, 0.0128 and 0.0126 us
                    if (mixed && chain)
                        cost *= js[ji] == 20 ? 0.91 : js[ji] == 16 ? 1.0 : js[ji] == 12 ? 0.98 : 1.1;
                    else if (mixed)
                        cost *= js[ji] == 12 ? 1.0 : js[ji] == 20 ? 1.03 : 1.08;
                    // a series cut into tiles runs at the throughput of
                    // its blocks, which falls with fewer warps (the
                    // leapfrog is latency-bound): measured on the mixed
                    // kernel at T = 2^22, 384 x 20 takes 0.382 ms a
                    // trajectory in 4 waves, 288 x 20 0.449 ms in 5 (25 %
                    // more per site); a whole series keeps the smallest
                    // window (a tie-break toward more threads only)
                    cost *= 1.0 + (b > 1 ? 1.0 : 1e-3) * (double)(tmax - t) / tmax;
                    if (cost < best) {
                        best = cost;
                        nt = t;
                        j = js[ji];
                        tile = ut;
                    }
                }
            }
        }
        if (nt == 0) {
            *why = "n_md too large for an on-chip window";
            return false;
        }
    } else {
        // many series: the largest window, so that most series are whole
        j = mixed ? 20 : 28;
        nt = ntmax(mixed, mass, j);
        tile = (int64_t)nt * j - 2 * K - 3;
        if (tile < 1) {
            *why = "n_md too large for an on-chip window";
            return false;
        }
    }
    const int64_t cap = (int64_t)nt * j;
    const int NW = nt / 32;
    const int64_t per_warp = 32LL * j;

    // ---- segments --------------------------------------------------------------
    std::vector<Seg> segs;
    std::vector<SerInfo> ser(n);
    for (int s = 0; s < n; ++s) {
        const int64_t T = off[s + 1] - off[s];
        ser[s].off = off[s];
        ser[s].T = T;
        ser[s].seg0 = (int)segs.size();
        const bool whole = (n == 1) ? (tile >= T && T <= cap) : (T <= cap);
        if (whole) {
            Seg g;
            g.lo = 0;
            g.hi = T;
            g.wlo = 0;
            g.whi = T;
            g.series = s;
            g.warp0 = 0;
            g.nwarp = (int)((T + per_warp - 1) / per_warp);
            g.split = 0;
            segs.push_back(g);
            ser[s].nseg = 1;
        } else {
            int cnt = 0;
            for (int64_t lo = 0; lo < T; lo += tile) {
                Seg g;
                g.lo = lo;
                g.hi = std::min(T, lo + tile);
                g.wlo = std::max(lo - K, (int64_t)0) & ~(int64_t)3;
                g.whi = std::min(T, g.hi + K);
                g.series = s;
                g.warp0 = 0;
                g.nwarp = NW;
                g.split = 1;
                if (g.whi - g.wlo > cap) {
                    *why = "internal: tile window exceeds the block";
                    return false;
                }
                segs.push_back(g);
                ++cnt;
            }
            ser[s].nseg = cnt;
        }
    }

    // ---- bins ------------------------------------------------------------------
    std::vector<int> bin_first{0};
    std::vector<int> bin_seg;
    int nsplit = 0;
    for (int s = 0; s < n; ++s) {
        if (ser[s].nseg > 1 || segs[ser[s].seg0].split) {
            ++nsplit;
            for (int k = 0; k < ser[s].nseg; ++k) {
                bin_seg.push_back(ser[s].seg0 + k);
                bin_first.push_back((int)bin_seg.size());
            }
        }
    }
    std::vector<int> whole;
    for (int i = 0; i < (int)segs.size(); ++i)
        if (!segs[i].split) whole.push_back(i);
    std::stable_sort(whole.begin(), whole.end(),
                     [&](int a, int b) { return segs[a].nwarp > segs[b].nwarp; });
    std::vector<std::vector<int>> bins;
    std::vector<int> room;
    for (int id : whole) {
        const int need = segs[id].nwarp;
        int b = -1;
        for (int k = 0; k < (int)bins.size(); ++k)
            if (room[k] >= need) {
                b = k;
                break;
            }
        if (b < 0) {
            bins.emplace_back();
            room.push_back(NW);
            b = (int)bins.size() - 1;
        }
        segs[id].warp0 = NW - room[b];
        room[b] -= need;
        bins[b].push_back(id);
    }
    for (auto& b : bins) {
        for (int id : b) bin_seg.push_back(id);
        bin_first.push_back((int)bin_seg.size());
    }
    const int nbins = (int)bin_first.size() - 1;

    // ---- launch shape ----------------------------------------------------------
    Plan p;
    p.nt = nt;
    p.j = j;
    p.nbins = nbins;
    p.smem = smem_for(mixed, mass, lev, nt, j);
    p.nsegs = (int64_t)segs.size();
    p.nseries = n;
    p.nsplit = nsplit;
    p.total = off[n];
    p.n_md = n_md;
    p.integrator = integrator;
    p.lambda = lambda;
    p.mixed = mixed;
    p.mass = mass;
    p.lev = lev;
    const int bps = blocks_per_sm(mixed, mass, lev, j, nt, p.smem);
    if (bps < 1) {  // a fixed schedule whose block does not fit on an SM
        *why = "the block shape does not fit on one SM (shared memory or registers)";
        return false;
    }
    p.grid = std::min(nbins, num_sms * bps);

    // ---- device copy -----------------------------------------------------------
    cudaError_t e = cudaMalloc(&p.d_segs, sizeof(Seg) * segs.size());
    if (e == cudaSuccess) e = cudaMalloc(&p.d_bin_first, sizeof(int) * bin_first.size());
    if (e == cudaSuccess) e = cudaMalloc(&p.d_bin_seg, sizeof(int) * std::max<size_t>(1, bin_seg.size()));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_ser, sizeof(SerInfo) * ser.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_segs, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_bin_first, bin_first.data(), sizeof(int) * bin_first.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !bin_seg.empty())
        e = cudaMemcpy(p.d_bin_seg, bin_seg.data(), sizeof(int) * bin_seg.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_ser, ser.data(), sizeof(SerInfo) * ser.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_plan(p);
        *why = "plan upload failed (out of device memory?)";
        return false;
    }
    P = p;
    return true;
}

}  // namespace rsv
