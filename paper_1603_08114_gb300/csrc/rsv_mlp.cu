// rsv_mlp.cu -- the learned diagonal mass: sampler moments, features, a BF16
// MLP trained by Adam, and mass inference.
//
// Not part of the paper (which has no learned component): this library adds a
// per-site mass m_t = s (softplus(z_t) + eps) for HMC, where z_t is a 20 -> 32 ->
// 32 -> 1 MLP (tanh hidden units) on 20 features of site t computed from a
// FROZEN state (the posterior mean hbar of a plain sampler), so the mass never
// depends on the current h and HMC stays exact.  The network is trained on
// log(1 / Var(h_t)) with the squared error in log space.  s is a fixed output
// scale, the geometric mean of the target precisions: it keeps softplus near
// its unit-slope range so that the tanh layers need not saturate to reach
// precisions of O(30).
//
// Tensor cores: the matmuls (layer 1 and 2 forward, the back-propagation
// through layer 2 and the weight gradients of layers 1 and 2) run as
// mma.sync m16n8k16 BF16 tiles with FP32 accumulation; a warp owns 16 sites.
// These GEMMs are 16 x 32 x 32 per warp; tcgen05's 128-row tiles and TMEM
// staging would idle on them, so the warp-level MMA is the right size here.
//
// Parameter vector (FP32, 1761): W1[32][20] b1[32] W2[32][32] b2[32] W3[32] b3.
#include <cmath>

#include <cuda_bf16.h>

#include "rsv_device.cuh"
#include "rsv_mlp.cuh"

namespace rsv {

namespace {

constexpr int NF = 20, NH = 32, KP = 32;  // features, hidden, padded K of layer 1
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH,
              NPARAM = OFF_B3 + 1;
static_assert(NPARAM == 1761, "parameter layout");
constexpr float EPS_M = 1e-3f;
constexpr int EDGE = 16;       // the edge proximity 2^-d is not standardised
constexpr float CLIP = 8.0f;   // standardised features are clipped to [-8, 8]
constexpr int SITES_PER_BLOCK = 64;  // 4 warps x 16 sites

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
__device__ __forceinline__ float round_bf16(float x)
{
    return __bfloat162float(__float2bfloat16_rn(x));
}

// D = A(16x16, row) * B(16x8, col) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float softplus_f(float z)
{
    return z > 20.f ? z : log1pf(expf(z));
}
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + expf(-z)); }

// Shared parameter copies of one block.
struct SParams {
    float w1[NH * KP];  // BF16-rounded, K padded with zeros
    float w2[NH * NH];  // BF16-rounded
    float b1[NH], b2[NH], w3[NH];
    float b3;
};

__device__ void load_params(const float* __restrict__ P, SParams& s)
{
    for (int i = threadIdx.x; i < NH * KP; i += blockDim.x) {
        const int n = i / KP, k = i % KP;
        s.w1[i] = k < NF ? round_bf16(P[OFF_W1 + n * NF + k]) : 0.f;
    }
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) s.w2[i] = round_bf16(P[OFF_W2 + i]);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        s.b1[i] = P[OFF_B1 + i];
        s.b2[i] = P[OFF_B2 + i];
        s.w3[i] = P[OFF_W3 + i];
    }
    if (threadIdx.x == 0) s.b3 = P[OFF_B3];
}

// B fragment (16 x 8, "col") of a matrix stored as M[n][k] (row n, K
// consecutive): element (k, n) = M[n0 + n][k0 + k].
__device__ __forceinline__ void b_frag_nk(const float* M, int ld, int n0, int k0, uint32_t& b0,
                                          uint32_t& b1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float* r = M + (n0 + g) * ld + k0;
    b0 = pack_bf16(r[2 * t], r[2 * t + 1]);
    b1 = pack_bf16(r[2 * t + 8], r[2 * t + 9]);
}
// B fragment of a matrix stored as M[k][n]: element (k, n) = M[k0 + k][n0 + n].
__device__ __forceinline__ void b_frag_kn(const float* M, int ld, int k0, int n0, uint32_t& b0,
                                          uint32_t& b1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    b0 = pack_bf16(M[(k0 + 2 * t) * ld + n0 + g], M[(k0 + 2 * t + 1) * ld + n0 + g]);
    b1 = pack_bf16(M[(k0 + 2 * t + 8) * ld + n0 + g], M[(k0 + 2 * t + 9) * ld + n0 + g]);
}
// A fragment (16 x 16, row) of a matrix stored as M[m][k]: (m, k) = M[m0 + m][k0 + k].
__device__ __forceinline__ void a_frag_mk(const float* M, int ld, int m0, int k0, uint32_t (&a)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float* r0 = M + (m0 + g) * ld + k0;
    const float* r1 = M + (m0 + g + 8) * ld + k0;
    a[0] = pack_bf16(r0[2 * t], r0[2 * t + 1]);
    a[1] = pack_bf16(r1[2 * t], r1[2 * t + 1]);
    a[2] = pack_bf16(r0[2 * t + 8], r0[2 * t + 9]);
    a[3] = pack_bf16(r1[2 * t + 8], r1[2 * t + 9]);
}
// A fragment of the TRANSPOSE of M[k][m]: (m, k) = M[k0 + k][m0 + m].
__device__ __forceinline__ void a_frag_t(const float* M, int ld, int m0, int k0, uint32_t (&a)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    a[0] = pack_bf16(M[(k0 + 2 * t) * ld + m0 + g], M[(k0 + 2 * t + 1) * ld + m0 + g]);
    a[1] = pack_bf16(M[(k0 + 2 * t) * ld + m0 + g + 8], M[(k0 + 2 * t + 1) * ld + m0 + g + 8]);
    a[2] = pack_bf16(M[(k0 + 2 * t + 8) * ld + m0 + g], M[(k0 + 2 * t + 9) * ld + m0 + g]);
    a[3] = pack_bf16(M[(k0 + 2 * t + 8) * ld + m0 + g + 8],
                     M[(k0 + 2 * t + 9) * ld + m0 + g + 8]);
}
// A fragment of a 16 x 32 activation held as C fragments c[ntile][4] (k-step kk).
__device__ __forceinline__ void a_from_c(const float (&c)[4][4], int kk, uint32_t (&a)[4])
{
    a[0] = pack_bf16(c[2 * kk][0], c[2 * kk][1]);
    a[1] = pack_bf16(c[2 * kk][2], c[2 * kk][3]);
    a[2] = pack_bf16(c[2 * kk + 1][0], c[2 * kk + 1][1]);
    a[3] = pack_bf16(c[2 * kk + 1][2], c[2 * kk + 1][3]);
}

// Site index of minibatch entry k of Adam step `step`: word k%4 of Philox
// block k/4 (counter {k/4, step, 3, 0}, key {seed, 0}), floor(hi32(w) T / 2^32).
__device__ __forceinline__ int64_t batch_site(uint64_t seed, uint64_t step, int64_t k, int64_t T)
{
    const u64x4 w = philox_block(seed, 0, step, 3, (uint64_t)(k >> 2));
    const uint64_t hi = w.w[k & 3] >> 32;
    return (int64_t)((hi * (uint64_t)T) >> 32);
}

// Forward of the 16 sites of this warp.  fs: [16][KP] BF16-rounded features
// (shared).  Outputs: a1, a2 in C-fragment form, z3 for rows g and g+8.
__device__ __forceinline__ void mlp_forward(const SParams& sp, const float* fs, float (&a1)[4][4],
                                            float (&a2)[4][4], float& z3g, float& z3g8)
{
    const int lane = threadIdx.x & 31, t = lane & 3;
    float z1[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        uint32_t a[4];
        a_frag_mk(fs, KP, 0, 16 * kk, a);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0, b1;
            b_frag_nk(sp.w1, KP, 8 * nt, 16 * kk, b0, b1);
            mma_bf16(z1[nt], a, b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        a1[nt][0] = tanhf(z1[nt][0] + sp.b1[n0]);
        a1[nt][1] = tanhf(z1[nt][1] + sp.b1[n0 + 1]);
        a1[nt][2] = tanhf(z1[nt][2] + sp.b1[n0]);
        a1[nt][3] = tanhf(z1[nt][3] + sp.b1[n0 + 1]);
    }
    float z2[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        uint32_t a[4];
        a_from_c(a1, kk, a);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0, b1;
            b_frag_nk(sp.w2, NH, 8 * nt, 16 * kk, b0, b1);
            mma_bf16(z2[nt], a, b0, b1);
        }
    }
    float pg = 0.f, pg8 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        a2[nt][0] = tanhf(z2[nt][0] + sp.b2[n0]);
        a2[nt][1] = tanhf(z2[nt][1] + sp.b2[n0 + 1]);
        a2[nt][2] = tanhf(z2[nt][2] + sp.b2[n0]);
        a2[nt][3] = tanhf(z2[nt][3] + sp.b2[n0 + 1]);
        pg = fmaf(a2[nt][0], sp.w3[n0], fmaf(a2[nt][1], sp.w3[n0 + 1], pg));
        pg8 = fmaf(a2[nt][2], sp.w3[n0], fmaf(a2[nt][3], sp.w3[n0 + 1], pg8));
    }
    // the 4 lanes of a group hold the 32 columns of rows g and g+8
    pg += __shfl_xor_sync(0xffffffffu, pg, 1);
    pg += __shfl_xor_sync(0xffffffffu, pg, 2);
    pg8 += __shfl_xor_sync(0xffffffffu, pg8, 1);
    pg8 += __shfl_xor_sync(0xffffffffu, pg8, 2);
    z3g = pg + sp.b3;
    z3g8 = pg8 + sp.b3;
}

// One minibatch: loss and gradient partials of this block; the last block to
// arrive sums the partials in block order and (update != 0) takes an Adam
// step of the FP32 master parameters.
struct StepArgs {
    const float* feat;    // [T][NF] standardised features
    const float* target;  // [T]
    int64_t T;
    float* params;        // [NPARAM] FP32 master, updated in place
    float* adam_m;
    float* adam_v;
    float* grad_out;      // optional: the gradient of this batch [NPARAM]
    float* partials;      // [gridDim.x][NPARAM + 1]
    unsigned* counter;
    uint64_t seed, step;  // minibatch of Adam step `step`
    int64_t adam_t;       // 1-based Adam time of this step
    float lr, b1, b2, eps;
    int batch;
    int update;
    float* loss_out;      // optional
    const float* log_scale;  // optional device scalar: log s
};

__global__ void __launch_bounds__(128) k_mlp_step(const StepArgs A)
{
    __shared__ SParams sp;
    __shared__ float fs[4][16][KP];   // features of the warp's sites (BF16-rounded)
    __shared__ float st_a1[4][16][NH];  // a1 (BF16-rounded) for dW2
    __shared__ float st_d[4][16][NH];   // dz2, then dz1 (BF16-rounded)
    __shared__ float gsum[NPARAM + 1];  // block gradient (+ loss in the last slot)
    __shared__ int s_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    load_params(A.params, sp);
    for (int i = tid; i < NPARAM + 1; i += blockDim.x) gsum[i] = 0.f;
    // gather this warp's 16 sites
    const int64_t k0 = (int64_t)blockIdx.x * SITES_PER_BLOCK + warp * 16;
    if (lane < 16) {
        const int64_t site = batch_site(A.seed, A.step, k0 + lane, A.T);
        for (int f = 0; f < KP; ++f)
            fs[warp][lane][f] = f < NF ? round_bf16(A.feat[site * NF + f]) : 0.f;
    }
    __syncthreads();
    float a1[4][4], a2[4][4], z3g, z3g8;
    mlp_forward(sp, &fs[warp][0][0], a1, a2, z3g, z3g8);
    // loss gradient at rows g and g+8
    float yg, yg8;
    {
        const int64_t sg = batch_site(A.seed, A.step, k0 + g, A.T);
        const int64_t sg8 = batch_site(A.seed, A.step, k0 + g + 8, A.T);
        yg = A.target[sg];
        yg8 = A.target[sg8];
    }
    const float ls = A.log_scale ? *A.log_scale : 0.f;
    const float mg = softplus_f(z3g) + EPS_M, mg8 = softplus_f(z3g8) + EPS_M;
    const float lg = logf(mg) + ls - yg, lg8 = logf(mg8) + ls - yg8;
    const float invB = 1.f / (float)A.batch;
    const float g3g = 2.f * lg * invB * sigmoid_f(z3g) / mg;
    const float g3g8 = 2.f * lg8 * invB * sigmoid_f(z3g8) / mg8;
    // dz2 = g3 W3 (1 - a2^2); dW3 = sum g3 a2; db2 = sum dz2
    float dz2[4][4];
    float pw3[4][2], pb2[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float w = sp.w3[n0 + c];
            dz2[nt][c] = g3g * w * (1.f - a2[nt][c] * a2[nt][c]);
            dz2[nt][2 + c] = g3g8 * w * (1.f - a2[nt][2 + c] * a2[nt][2 + c]);
            pw3[nt][c] = g3g * a2[nt][c] + g3g8 * a2[nt][2 + c];
            pb2[nt][c] = dz2[nt][c] + dz2[nt][2 + c];
        }
    }
    // sum over the 8 groups of the warp (rows), then one lane per column adds
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                pw3[nt][c] += __shfl_xor_sync(0xffffffffu, pw3[nt][c], o);
                pb2[nt][c] += __shfl_xor_sync(0xffffffffu, pb2[nt][c], o);
            }
    // stage a1 and dz2 (BF16-rounded) for the weight gradient of layer 2
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        st_a1[warp][g][n0] = round_bf16(a1[nt][0]);
        st_a1[warp][g][n0 + 1] = round_bf16(a1[nt][1]);
        st_a1[warp][g + 8][n0] = round_bf16(a1[nt][2]);
        st_a1[warp][g + 8][n0 + 1] = round_bf16(a1[nt][3]);
        st_d[warp][g][n0] = round_bf16(dz2[nt][0]);
        st_d[warp][g][n0 + 1] = round_bf16(dz2[nt][1]);
        st_d[warp][g + 8][n0] = round_bf16(dz2[nt][2]);
        st_d[warp][g + 8][n0 + 1] = round_bf16(dz2[nt][3]);
    }
    __syncwarp();
    // dW2[n][k] = sum_s dz2[s][n] a1[s][k]: M = n (2 tiles), N = k (4 tiles), K = 16 sites
    float gw2[2][4][4] = {};
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4];
        a_frag_t(&st_d[warp][0][0], NH, 16 * mt, 0, a);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0, b1;
            b_frag_kn(&st_a1[warp][0][0], NH, 0, 8 * nt, b0, b1);
            mma_bf16(gw2[mt][nt], a, b0, b1);
        }
    }
    // da1 = dz2 W2 (A = dz2 rows = sites; B(k=n, n=j) = W2[n][j])
    float da1[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        uint32_t a[4];
        a[0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
        a[1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
        a[2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
        a[3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0, b1;
            b_frag_kn(sp.w2, NH, 16 * kk, 8 * nt, b0, b1);
            mma_bf16(da1[nt], a, b0, b1);
        }
    }
    // dz1 = da1 (1 - a1^2); db1 = sum dz1; stage dz1 for dW1
    float pb1[4][2];
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        float d[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) d[c] = da1[nt][c] * (1.f - a1[nt][c] * a1[nt][c]);
        pb1[nt][0] = d[0] + d[2];
        pb1[nt][1] = d[1] + d[3];
        st_d[warp][g][n0] = round_bf16(d[0]);
        st_d[warp][g][n0 + 1] = round_bf16(d[1]);
        st_d[warp][g + 8][n0] = round_bf16(d[2]);
        st_d[warp][g + 8][n0 + 1] = round_bf16(d[3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1)
                pb1[nt][c] += __shfl_xor_sync(0xffffffffu, pb1[nt][c], o);
    __syncwarp();
    // dW1[n][f] = sum_s dz1[s][n] F[s][f]: M = n (2 tiles), N = f (4 tiles over KP)
    float gw1[2][4][4] = {};
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4];
        a_frag_t(&st_d[warp][0][0], NH, 16 * mt, 0, a);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0, b1;
            b_frag_kn(&fs[warp][0][0], KP, 0, 8 * nt, b0, b1);
            mma_bf16(gw1[mt][nt], a, b0, b1);
        }
    }
    // loss of the warp's sites
    float lsum = (t == 0) ? (lg * lg + lg8 * lg8) : 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    const float g3sum_part = (t == 0) ? (g3g + g3g8) : 0.f;
    float g3sum = g3sum_part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) g3sum += __shfl_xor_sync(0xffffffffu, g3sum, o);

    // block sums in warp order (deterministic): warp w adds after warp w-1
    for (int w = 0; w < 4; ++w) {
        __syncthreads();
        if (warp != w) continue;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = 16 * mt + g, k = 8 * nt + 2 * t;
                gsum[OFF_W2 + n * NH + k] += gw2[mt][nt][0];
                gsum[OFF_W2 + n * NH + k + 1] += gw2[mt][nt][1];
                gsum[OFF_W2 + (n + 8) * NH + k] += gw2[mt][nt][2];
                gsum[OFF_W2 + (n + 8) * NH + k + 1] += gw2[mt][nt][3];
                if (k < NF) {
                    gsum[OFF_W1 + n * NF + k] += gw1[mt][nt][0];
                    gsum[OFF_W1 + (n + 8) * NF + k] += gw1[mt][nt][2];
                }
                if (k + 1 < NF) {
                    gsum[OFF_W1 + n * NF + k + 1] += gw1[mt][nt][1];
                    gsum[OFF_W1 + (n + 8) * NF + k + 1] += gw1[mt][nt][3];
                }
            }
        if (g == 0) {
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int n = 8 * nt + 2 * t + c;
                    gsum[OFF_W3 + n] += pw3[nt][c];
                    gsum[OFF_B2 + n] += pb2[nt][c];
                    gsum[OFF_B1 + n] += pb1[nt][c];
                }
        }
        if (lane == 0) {
            gsum[OFF_B3] += g3sum;
            gsum[NPARAM] += lsum;
        }
    }
    __syncthreads();
    for (int i = tid; i < NPARAM + 1; i += blockDim.x)
        A.partials[(int64_t)blockIdx.x * (NPARAM + 1) + i] = gsum[i];
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = tid; i < NPARAM + 1; i += blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(A.partials + (int64_t)b * (NPARAM + 1) + i);
        if (i == NPARAM) {
            if (A.loss_out) *A.loss_out = s / (float)A.batch;
            continue;
        }
        if (A.grad_out) A.grad_out[i] = s;
        if (A.update) {
            // Adam (Kingma & Ba 2015), FP32
            const float m = A.b1 * A.adam_m[i] + (1.f - A.b1) * s;
            const float v = A.b2 * A.adam_v[i] + (1.f - A.b2) * s * s;
            A.adam_m[i] = m;
            A.adam_v[i] = v;
            const float mh = m / (1.f - powf(A.b1, (float)A.adam_t));
            const float vh = v / (1.f - powf(A.b2, (float)A.adam_t));
            A.params[i] -= A.lr * mh / (sqrtf(vh) + A.eps);
        }
    }
    if (tid == 0) *A.counter = 0u;
}

// Clamp interval of the mass at site t: [1/s_u^2, diagonal of the Hessian of
// S at hbar] = [1/s_u^2, A_t/s_eta^2 + 1/s_u^2 + (y_t^2/2) e^{-hbar_t}], A_t =
// 1 + phi^2 inside, 1 at the ends, 1 - phi^2 when T = 1.
__device__ __forceinline__ float clamp_mass(float m, int64_t t, int64_t T, const double* y,
                                            const double* hbar, const ThetaD& th)
{
    const double A = T == 1 ? 1.0 - th.phi * th.phi
                   : (t == 0 || t == T - 1) ? 1.0 : 1.0 + th.phi * th.phi;
    const double lo = 1.0 / th.su2;
    const double hi = A / th.se2 + lo + 0.5 * y[t] * y[t] * exp(-hbar[t]);
    return fminf(fmaxf(m, (float)lo), (float)hi);
}

// m_t for every site, clamped; writes 1/m_t (and m_t if m_out).
__global__ void __launch_bounds__(128) k_mlp_mass(const float* __restrict__ feat, int64_t T,
                                                  const float* __restrict__ P,
                                                  const double* __restrict__ y,
                                                  const double* __restrict__ hbar, ThetaD th,
                                                  const float* __restrict__ log_scale,
                                                  float* __restrict__ minv, float* __restrict__ m_out)
{
    __shared__ SParams sp;
    __shared__ float fs[4][16][KP];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const float scale = log_scale ? expf(*log_scale) : 1.f;
    load_params(P, sp);
    __syncthreads();
    for (int64_t base = ((int64_t)blockIdx.x * 4 + warp) * 16; base < T;
         base += (int64_t)gridDim.x * 64) {
        if (lane < 16) {
            const int64_t s = base + lane;
            for (int f = 0; f < KP; ++f)
                fs[warp][lane][f] = (f < NF && s < T) ? round_bf16(feat[s * NF + f]) : 0.f;
        }
        __syncwarp();
        float a1[4][4], a2[4][4], z3g, z3g8;
        mlp_forward(sp, &fs[warp][0][0], a1, a2, z3g, z3g8);
        if (t == 0) {
            const int64_t s0 = base + g, s1 = base + g + 8;
            float m0 = scale * (softplus_f(z3g) + EPS_M), m1 = scale * (softplus_f(z3g8) + EPS_M);
            if (s0 < T) m0 = clamp_mass(m0, s0, T, y, hbar, th);
            if (s1 < T) m1 = clamp_mass(m1, s1, T, y, hbar, th);
            if (s0 < T) {
                minv[s0] = 1.f / m0;
                if (m_out) m_out[s0] = m0;
            }
            if (s1 < T) {
                minv[s1] = 1.f / m1;
                if (m_out) m_out[s1] = m1;
            }
        }
        __syncwarp();
    }
}

// Fold n snapshot rows of x ([n][T] FP32) into running (count, mean, M2).
__global__ void k_welford(const float* __restrict__ x, int64_t n, int64_t T, int64_t count,
                          double* __restrict__ mean, double* __restrict__ m2)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        double m = count ? mean[t] : 0.0, s = count ? m2[t] : 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double v = (double)x[k * T + t];
            const double d = v - m;
            m += d / (double)(count + k + 1);
            s += d * (v - m);
        }
        mean[t] = m;
        m2[t] = s;
    }
}

// target_t = log(1 / Var(h_t)) = log((count - 1) / M2_t); hbar_t = mean_t.
__global__ void k_welford_target(const double* __restrict__ mean, const double* __restrict__ m2,
                                 int64_t T, int64_t count, double* __restrict__ hbar,
                                 float* __restrict__ target)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (hbar) hbar[t] = mean[t];
        const double var = m2[t] / (double)(count - 1);
        target[t] = (float)log(1.0 / fmax(var, 1e-300));
    }
}

// log s = mean over the sites of the target (one block, FP64, fixed order).
__global__ void __launch_bounds__(1024) k_target_mean(const float* __restrict__ target, int64_t T,
                                                      float* __restrict__ out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) s += (double)target[t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = (float)(s / (double)T);
}

// Raw features of each site (see the header of oracle/mlp.py for the list).
__global__ void k_feat_raw(const double* __restrict__ y, const double* __restrict__ lnrv,
                           const double* __restrict__ hbar, int64_t T, ThetaD th,
                           float* __restrict__ F)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        float* f = F + t * NF;
        const double yt = y[t];
        f[0] = (float)(yt * yt);
        f[1] = (float)lnrv[t];
        for (int k = -4; k <= 4; ++k) {
            const int64_t s = t + k;
            f[2 + k + 4] = (s >= 0 && s < T) ? (float)hbar[s] : 0.f;
        }
        f[11] = (float)th.phi;
        f[12] = (float)th.mu;
        f[13] = (float)th.xi;
        f[14] = (float)th.se2;
        f[15] = (float)th.su2;
        const int64_t d = t < T - 1 - t ? t : T - 1 - t;   // distance to the nearer end
        f[16] = ldexpf(1.f, -(int)(d < 64 ? d : 64));
        f[17] = (float)((1.0 + th.phi * th.phi) / th.se2);
        f[18] = (float)(1.0 / th.su2);
        f[19] = (float)(0.5 * yt * yt * exp(-hbar[t]));
    }
}

// Column sums (pass 0: sum f; pass 1: sum (f - mean)^2) with a last-block
// finish; stats = [mean(20), inv_sd(20)].
__global__ void __launch_bounds__(256) k_feat_stats(const float* __restrict__ F, int64_t T,
                                                    int pass, double* __restrict__ partials,
                                                    unsigned* __restrict__ counter,
                                                    double* __restrict__ acc,
                                                    float* __restrict__ stats)
{
    __shared__ double red[32];
    __shared__ int s_last;
    double loc[NF];
    for (int f = 0; f < NF; ++f) loc[f] = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x)
        for (int f = 0; f < NF; ++f) {
            const double v = (double)F[t * NF + f];
            if (pass == 0) {
                loc[f] += v;
            } else {
                const double d = v - acc[f];
                loc[f] += d * d;
            }
        }
    for (int f = 0; f < NF; ++f) {
        const double b = block_sum(loc[f], red);
        if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * NF + f] = b;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < NF) {
        const int f = threadIdx.x;
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + (int64_t)b * NF + f);
        if (pass == 0) {
            acc[f] = s / (double)T;
            stats[f] = f == EDGE ? 0.f : (float)acc[f];
        } else {
            const double sd = sqrt(s / (double)T);
            const double m = acc[f];
            stats[NF + f] = f == EDGE ? 1.f
                          : (sd > 1e-12 * fmax(1.0, fabs(m))) ? (float)(1.0 / sd) : 0.f;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

__global__ void k_feat_norm(float* __restrict__ F, int64_t T, const float* __restrict__ stats)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T * NF;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i % NF);
        F[i] = fminf(fmaxf((F[i] - stats[f]) * stats[NF + f], -CLIP), CLIP);
    }
}

int grid1(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int mlp_nparam() { return NPARAM; }
int mlp_sites_per_block() { return SITES_PER_BLOCK; }

cudaError_t launch_mlp_step(const float* feat, const float* target, int64_t T, float* params,
                            float* adam_m, float* adam_v, float* grad_out, float* partials,
                            unsigned* counter, uint64_t seed, uint64_t step, int64_t adam_t,
                            float lr, float b1, float b2, float eps, int batch, int update,
                            float* loss_out, const float* log_scale, cudaStream_t st)
{
    StepArgs a{feat,  target,  T,    params, adam_m, adam_v, grad_out, partials, counter,
               seed,  step,    adam_t, lr,   b1,     b2,     eps,      batch,    update,
               loss_out, log_scale};
    k_mlp_step<<<batch / SITES_PER_BLOCK, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_mass(const float* feat, int64_t T, const float* params, const double* y,
                            const double* hbar, ThetaD th, const float* log_scale, float* minv,
                            float* m_out, cudaStream_t st)
{
    int64_t g = (T + 63) / 64;
    if (g > 152 * 16) g = 152 * 16;
    k_mlp_mass<<<(int)(g < 1 ? 1 : g), 128, 0, st>>>(feat, T, params, y, hbar, th, log_scale,
                                                      minv, m_out);
    return cudaGetLastError();
}

cudaError_t launch_welford(const float* x, int64_t n, int64_t T, int64_t count, double* mean,
                           double* m2, cudaStream_t st)
{
    k_welford<<<grid1(T), 256, 0, st>>>(x, n, T, count, mean, m2);
    return cudaGetLastError();
}

cudaError_t launch_welford_target(const double* mean, const double* m2, int64_t T, int64_t count,
                                  double* hbar, float* target, float* log_scale, cudaStream_t st)
{
    k_welford_target<<<grid1(T), 256, 0, st>>>(mean, m2, T, count, hbar, target);
    if (log_scale) k_target_mean<<<1, 1024, 0, st>>>(target, T, log_scale);
    return cudaGetLastError();
}

int feat_grid(int64_t T) { return grid1(T); }

cudaError_t launch_features(const double* y, const double* lnrv, const double* hbar, int64_t T,
                            ThetaD th, float* F, float* stats, double* partials, unsigned* counter,
                            double* acc, cudaStream_t st)
{
    const int g = grid1(T);
    k_feat_raw<<<g, 256, 0, st>>>(y, lnrv, hbar, T, th, F);
    k_feat_stats<<<g, 256, 0, st>>>(F, T, 0, partials, counter, acc, stats);
    k_feat_stats<<<g, 256, 0, st>>>(F, T, 1, partials, counter, acc, stats);
    k_feat_norm<<<grid1(T * NF), 256, 0, st>>>(F, T, stats);
    return cudaGetLastError();
}

}  // namespace rsv
