// rsv_device.cuh -- device helpers of librsv (sm_103a).
//
// Counter-based generator, Box-Muller, double-float error-free transforms and
// fixed-order reductions shared by the kernels of this library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsv {

// Status bits written by kernels into the context status word.
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

// Philox counter streams (counter word 2).
enum : uint64_t { STREAM_MOM = 0, STREAM_MH = 1, STREAM_THETA = 2 };

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round maps
// (c0, c1, c2, c3) to (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0))
// with A = 0xD2E7470EE14C6C93, B = 0xCA5A826395121157; between rounds the key
// advances by the Weyl increments 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B.
// ---------------------------------------------------------------------------
struct u64x4 { uint64_t w[4]; };

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1)
{
    const uint64_t A = 0xD2E7470EE14C6C93ULL, B = 0xCA5A826395121157ULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        const uint64_t hiA = __umul64hi(A, c0), loA = A * c0;
        const uint64_t hiB = __umul64hi(B, c2), loB = B * c2;
        const uint64_t n0 = hiB ^ c1 ^ k0, n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
    }
    u64x4 o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// Philox block `blk` of stream `stream` for trajectory `traj` of series `series`.
__device__ __forceinline__ u64x4 philox_block(uint64_t seed, uint64_t series, uint64_t traj,
                                             uint64_t stream, uint64_t blk)
{
    return philox4x64_10(blk, traj, stream, series, seed, 0ULL);
}

// Uniform in (0,1): (k + 1/2) 2^-53 from the top 53 bits.
__device__ __forceinline__ double u01_53(uint64_t w)
{
    return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}
// Uniform in (0,1) exactly representable in FP32: (k + 1/2) 2^-23, k = top 23
// bits.  Built from the bits (1 + k 2^-23 has k as its mantissa) so that no
// integer-to-float conversion runs: conversions share this GPU's slow FP64
// pipe.  Every step is exact: (1 + k 2^-23) - 1 = k 2^-23, + 2^-24 fits 24 bits.
__device__ __forceinline__ float u01_23(uint64_t w)
{
    const uint32_t k = (uint32_t)(w >> 41);
    return (__uint_as_float(0x3F800000u | k) - 1.0f) + 0x1.0p-24f;
}

// Box-Muller: r = sqrt(-2 ln u1); (r cos 2 pi u2, r sin 2 pi u2).
__device__ __forceinline__ void box_muller(double u1, double u2, double& z0, double& z1)
{
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}
__device__ __forceinline__ void box_muller_f(float u1, float u2, float& z0, float& z1)
{
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// two_sum (Knuth), fast_two_sum (Dekker, |a| >= |b|), two_prod by FMA.
// Every add, subtract and multiply is an explicitly rounded intrinsic: the
// error-free transformations need s = fl(a + b) exactly, and the compiler
// would otherwise fuse a product feeding an add into an FMA (a different
// rounding of s).
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// Accumulate a double-float into a double-float (no renormalisation of the
// small part until read).
__device__ __forceinline__ void ff_acc(ff& acc, ff v)
{
    ff s = two_sum(acc.hi, v.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, v.lo));
}
__host__ __device__ __forceinline__ ff ff_from_double(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Table of 2^(j/32), j = 0..31, as double-float pairs (filled by ff_exp_table).
__device__ __forceinline__ void ff_exp_table(float2* tab)
{
    for (int j = threadIdx.x; j < 32; j += blockDim.x) {
        const ff v = ff_from_double(exp2((double)j / 32.0));
        tab[j] = make_float2(v.hi, v.lo);
    }
}

// e^t in double-float (relative error ~1e-12 for |t| < 80, the caller's
// range), table-driven:
// t = k ln2/32 + r with k = rint(32 t / ln2), |r| <= ln2/64; e^t =
// 2^(k div 32) 2^((k mod 32)/32) e^r, e^r = 1 + r + q with the tail
// q = r^2 (1/2 + r/6 + r^2/24 + r^3/120) in FP32 (|q| < 6e-5, so its FP32
// rounding is below 1e-11 of the result).  ln2/32 is split into a 24-bit
// head and a tail so that k * head is exact through two_prod.
// k = rint(32 t / ln2) is taken by adding 1.5 2^23 (the FP32 sum then holds k
// in its low mantissa bits, rounded to nearest even, for |k| < 2^22), which
// needs no float-to-integer conversion.
__device__ __forceinline__ ff ff_exp(ff t, const float2* tab)
{
    const float C_hi = 0x1.62e43p-6f, C_lo = -0x1.05c61p-34f;  // ln2/32
    const float kr = __fmaf_rn(t.hi, 46.166241308446828f, 0x1.8p23f);  // 32/ln2
    const int k = __float_as_int(kr) - 0x4B400000;
    const float kf = __fsub_rn(kr, 0x1.8p23f);
    ff kc = two_prod(kf, C_hi);
    kc.lo = __fmaf_rn(kf, C_lo, kc.lo);
    const ff r = ff_sub(t, kc);
    const float x = r.hi;
    const float q = __fmul_rn(
        __fmul_rn(x, x),
        __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f), 0.5f));
    ff s = two_sum(x, q);
    s.lo = __fadd_rn(s.lo, r.lo);
    ff e = two_sum(1.0f, s.hi);
    e.lo = __fadd_rn(e.lo, s.lo);
    e = fast_two_sum(e.hi, e.lo);
    const float2 tv = tab[k & 31];
    ff res = ff_mul(ff{tv.x, tv.y}, e);
    // 2^(k div 32) as an exact power of two (|t| < 80 keeps it normal)
    const float sc = __int_as_float(((k >> 5) + 127) << 23);
    return ff{__fmul_rn(res.hi, sc), __fmul_rn(res.lo, sc)};
}

// ---------------------------------------------------------------------------
// exp in FP64 for the FP64 trajectory kernel, table-driven after P. T. P. Tang
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15, 1989): a = k ln2/64 + r with k the
// integer nearest to 64 a/ln2 and |r| <= ln2/128 (ln2/64 split in a head of 32
// significant bits, so that k times it is exact, and a tail), and
//   e^a = 2^(k div 64) 2^((k mod 64)/64) (1 + p(r)),
// p the Taylor polynomial of e^r - 1 to degree 5 (remainder < 4e-17 for
// |r| <= ln2/128): 10 FP64 instructions.  kExp2Tab holds 2^(j/64) rounded to
// double (computed to 200 bits).  |a| >= 512 takes exp (the scaling by
// 2^(k div 64) through the exponent field assumes a normal result).
// ---------------------------------------------------------------------------
constexpr int kExpTabN = 64;
static __constant__ double kExp2Tab[kExpTabN] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};
__device__ __forceinline__ double exp_tab(double a, const double* tab)
{
    const long long ab = __double_as_longlong(a);
    if (((ab >> 52) & 0x7ff) >= 1032) return exp(a);  // |a| >= 512
    const double sh = 0x1.8p52;  // adding it rounds to an integer
    const double ks = fma(a, 0x1.71547652b82fep+6, sh);  // 64/ln2
    const int k = (int)(__double_as_longlong(ks) - __double_as_longlong(sh));
    const double kd = ks - sh;
    double r = fma(-kd, 0x1.62e42fee00000p-7, a);  // head of ln2/64
    r = fma(-kd, 0x1.a39ef35793c76p-39, r);          // its tail
    double q = fma(r, 0x1.1111111111111p-7, 0x1.5555555555555p-5);  // 1/120, 1/24
    q = fma(r, q, 0x1.5555555555555p-3);                               // 1/6
    q = fma(r, q, 0.5);
    const double p = fma(r * r, q, r);
    const double t = tab[k & (kExpTabN - 1)];
    const double e = fma(t, p, t);
    return __longlong_as_double(__double_as_longlong(e) + ((long long)(k >> 6) << 52));
}

// ---------------------------------------------------------------------------
// Reductions in a fixed order (deterministic): xor-butterfly inside a warp,
// then warp 0 over the per-warp values in warp order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ ff warp_sum_ff(ff v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}
// Block sum; `red` needs blockDim.x/32 doubles.  Result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        for (int i = lane; i < nw; i += 32) s += red[i];
        s = warp_sum(s);
    }
    return s;
}

// Theta as stored on the device: (phi, mu, xi, sigma_eta^2, sigma_u^2), and
// the leverage rho = corr(eps_t, eta_t) of the RSV model with leverage (a
// context setting, not stored with theta; 0 is the model of eqs. (1)-(3)).
struct ThetaD {
    double phi, mu, xi, se2, su2;
    double rho = 0.0;
};
__device__ __forceinline__ ThetaD load_theta(const double* th, double rho = 0.0)
{
    return {th[0], th[1], th[2], th[3], th[4], rho};
}

}  // namespace rsv
