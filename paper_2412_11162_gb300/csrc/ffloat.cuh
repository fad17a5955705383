// Float-float ("double-float") arithmetic on the FP32 pipe (sm_103a).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2:
// 48 significant bits (relative rounding ~2^-47 per operation), the exponent
// range of float.  The GB300's FP64 pipe retires 2 FMA per SM per clock and
// its FP32 pipe 128, so the sampling loops and transforms of the mixed path
// (S~, K~ at every node pair and angle, Sec. 3.1 / 4.1; the even-sequence
// DFTs of the FFT modal kernels, Sec. 4.1) run in this arithmetic and keep
// near-FP64 accuracy of the modal kernels.
//
// Building blocks: Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based exact
// product (TwoProd), as in the double-double literature (Dekker 1971;
// Hida, Li & Bailey 2001), written for floats.  Elementary functions:
//   exp:   x = n ln2/64 + r (ln2/64 split into three floats, the first with
//          8 significant bits so that n times it is exact for |n| < 2^16),
//          e^x = 2^(n div 64) T[n mod 64] e^r with T[j] = 2^(j/64) in float-float
//          and e^r = 1 + r + r^2/2 + r^3/6 + r^4/24 + r^5/120, |r| <= ln2/128;
//   sin, cos: x = n pi/256 + r (pi/256 in three floats, the first with 8
//          significant bits: exact n times it for |n| < 2^16), angle tables of
//          cos / sin (j pi/256), j = 0..128, and the Taylor series of sin r,
//          cos r to r^5 / r^4 (|r| <= pi/512: remainders < 2^-49);
//   1/sqrt: the hardware float estimate refined by two Newton steps, the
//          second with a float-float residual.
// Tables are float-float roundings of FP64 values computed on the host.
#pragma once

#include <cstdint>

namespace pmlbie {
namespace ffm {

struct ff {
    float hi, lo;
};

// complex float-float, stored as float4 (re.hi, re.lo, im.hi, im.lo)
struct cff {
    ff re, im;
};

__device__ __forceinline__ ff mk(float hi, float lo) { return ff{hi, lo}; }
__device__ __forceinline__ ff from_float(float x) { return ff{x, 0.0f}; }
__host__ __device__ __forceinline__ ff from_double(double x) {
    const float hi = (float)x;
    return ff{hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ float4 pack(cff a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cff unpack(float4 v) { return cff{ff{v.x, v.y}, ff{v.z, v.w}}; }

// ---- error-free transformations ----
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ---- arithmetic ----
__device__ __forceinline__ ff neg(ff a) { return ff{-a.hi, -a.lo}; }
// error ~2^-46 (|a| + |b|)
__device__ __forceinline__ ff add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    fast_two_sum(s, e, s, e);
    return ff{s, e};
}
__device__ __forceinline__ ff sub(ff a, ff b) { return add(a, neg(b)); }
__device__ __forceinline__ ff add_f(ff a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    fast_two_sum(s, e, s, e);
    return ff{s, e};
}
__device__ __forceinline__ ff mul(ff a, ff b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    fast_two_sum(p, e, p, e);
    return ff{p, e};
}
__device__ __forceinline__ ff mul_f(ff a, float b) {
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    fast_two_sum(p, e, p, e);
    return ff{p, e};
}
__device__ __forceinline__ ff sqr(ff a) {
    float p, e;
    two_prod(a.hi, a.hi, p, e);
    e = __fmaf_rn(2.0f * a.hi, a.lo, e);
    fast_two_sum(p, e, p, e);
    return ff{p, e};
}
// a b + c d with one renormalisation (error ~2^-46 (|a b| + |c d|))
__device__ __forceinline__ ff dot2(ff a, ff b, ff c, ff d) {
    float p1, e1, p2, e2, s, t;
    two_prod(a.hi, b.hi, p1, e1);
    two_prod(c.hi, d.hi, p2, e2);
    two_sum(p1, p2, s, t);
    float u = __fadd_rn(e1, e2);
    u = __fmaf_rn(a.hi, b.lo, u);
    u = __fmaf_rn(a.lo, b.hi, u);
    u = __fmaf_rn(c.hi, d.lo, u);
    u = __fmaf_rn(c.lo, d.hi, u);
    t = __fadd_rn(t, u);
    fast_two_sum(s, t, s, t);
    return ff{s, t};
}
// exact scaling by 2^k (no overflow / underflow handling: callers keep values
// in range)
__device__ __forceinline__ ff ldexp_ff(ff a, int k) {
    const float s = __int_as_float((k + 127) << 23);
    return ff{a.hi * s, a.lo * s};
}
// 1 / b
__device__ __forceinline__ ff rcp(ff b) {
    const float y = __frcp_rn(b.hi);
    // r = 1 - b y in float-float, then y (1 + r)
    const ff by = mul_f(b, y);
    const ff r = add_f(neg(by), 1.0f);
    float s, e;
    fast_two_sum(y, __fmul_rn(y, r.hi), s, e);
    const ff y1{s, e};
    // second step with the refined estimate
    const ff r2 = add_f(neg(mul(b, y1)), 1.0f);
    return add(y1, mul_f(y1, r2.hi));
}
__device__ __forceinline__ ff div(ff a, ff b) { return mul(a, rcp(b)); }
// 1 / sqrt(x), x > 0
__device__ __forceinline__ ff rsqrt(ff x) {
    float y = rsqrtf(x.hi);
    // float Newton step: y (3 - x y^2) / 2
    y = __fmul_rn(y, __fmaf_rn(-0.5f * x.hi * y, y, 1.5f));
    // float-float residual r = 1 - x y^2, then y + y r / 2
    const ff y2 = sqr(from_float(y));
    const ff r = add_f(neg(mul(x, y2)), 1.0f);
    float s, e;
    fast_two_sum(y, __fmul_rn(0.5f * y, r.hi), s, e);
    return ff{s, e};
}

// ---- complex ----
__device__ __forceinline__ cff cadd(cff a, cff b) { return cff{add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ cff csub(cff a, cff b) { return cff{sub(a.re, b.re), sub(a.im, b.im)}; }
__device__ __forceinline__ cff cmul(cff a, cff b) {
    return cff{dot2(a.re, b.re, neg(a.im), b.im), dot2(a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ cff cscale(cff a, ff s) { return cff{mul(a.re, s), mul(a.im, s)}; }
__device__ __forceinline__ cff cscale_f(cff a, float s) { return cff{mul_f(a.re, s), mul_f(a.im, s)}; }
__device__ __forceinline__ cff cneg(cff a) { return cff{neg(a.re), neg(a.im)}; }
__device__ __forceinline__ cff cldexp(cff a, int k) { return cff{ldexp_ff(a.re, k), ldexp_ff(a.im, k)}; }

// Principal square root R of z (z != 0) and 1/R = conj(R) / |z|:
// |z| from 1/sqrt(|z|^2), t = sqrt((|z| + |Re z|)/2), s = Im z / (2 t).
// z is first scaled by an even power of two 2^-2k to |z| ~ 1 (|z|^2 of a
// close pair's separation, ~1e-26 in units of the pair's length, would
// underflow), and R, 1/R are scaled back by 2^k, 2^-k.
__device__ __forceinline__ void csqrt_rcp_unit(cff z, cff& R, cff& iR);
__device__ __forceinline__ void csqrt_rcp(cff z, cff& R, cff& iR) {
    const float big = fmaxf(fabsf(z.re.hi), fabsf(z.im.hi));
    const int eb = (int)((__float_as_uint(big) >> 23) & 0xffu);   // biased exponent, 0: zero or denormal
    const int k = eb == 0 ? -63 : (eb - 127) >> 1;                // floor(e / 2)
    // z 2^-2k in two steps (each factor a normal float)
    const cff zs = cldexp(cldexp(z, -k), -k);
    csqrt_rcp_unit(zs, R, iR);
    R = cldexp(R, k);
    iR = cldexp(iR, -k);
}
__device__ __forceinline__ void csqrt_rcp_unit(cff z, cff& R, cff& iR) {
    const ff m2 = dot2(z.re, z.re, z.im, z.im);
    const ff ir = rsqrt(m2);                    // 1/|z|
    const ff r = mul(m2, ir);                   // |z|
    const ff ax = z.re.hi < 0.0f ? neg(z.re) : z.re;
    const ff u = mul_f(add(r, ax), 0.5f);
    const ff it = rsqrt(u);
    const ff t = mul(u, it);                    // sqrt(u)
    const ff s = mul_f(mul(z.im, it), 0.5f);    // Im z / (2 t)
    if (z.re.hi >= 0.0f) {
        R = cff{t, s};
    } else {
        const ff as = s.hi < 0.0f ? neg(s) : s;
        R = cff{as, z.im.hi < 0.0f ? neg(t) : t};
    }
    iR = cff{mul(R.re, ir), neg(mul(R.im, ir))};
}

// ---- tables (shared memory copies of the host-built float-float tables) ----
struct Tables {
    const float2* exp2j;   // 64: 2^(j/64)
    const float4* cs;      // 129: (cos(j pi/256), sin(j pi/256)), j = 0..128
};
constexpr int kExpTab = 64;
constexpr int kTrigTab = 129;

// e^x as a float-float mantissa in [2^-1/128, 2^1/128) times 2^E (E returned
// separately so that callers can keep a common scale); x is float-float,
// clamped to [-700, 700] (|n| < 2^16 keeps n C1 exact).  The reduction error
// is below |x| 2^-48 (relative to e^x), the rounding of the argument itself.
__device__ __forceinline__ ff exp_split(ff x, const Tables& T, int& E) {
    constexpr float kInvC = 92.33248f;             // 64 / ln 2
    constexpr float kC1 = 0x1.62p-7f;              // ln2/64 = C1 + C2 + C3, C1 with 8 bits
    constexpr float kC2 = 0x1.c85fe0p-16f;
    constexpr float kC3 = -0x1.718432p-41f;
    ff xc = x;
    if (x.hi < -700.0f) xc = ff{-700.0f, 0.0f};
    if (x.hi > 700.0f) xc = ff{700.0f, 0.0f};
    // nearest integer by the 1.5 x 2^23 shift (no conversion instruction:
    // this GPU issues conversions to its FP64 pipe); |x / C| < 2^22
    const float sh = __fadd_rn(__fmul_rn(xc.hi, kInvC), 12582912.0f);
    const float nf = __fsub_rn(sh, 12582912.0f);
    const int n = __float_as_int(sh) - 0x4b400000;
    // r = x - n (C1 + C2 + C3): n C1 exact, n C2 by TwoProd, n C3 rounded
    float p2, e2;
    two_prod(nf, kC2, p2, e2);
    ff r = add_f(xc, -nf * kC1);
    r = add(r, ff{-p2, -e2});
    r = add_f(r, -nf * kC3);
    // e^r - 1 = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120), |r| <= ln2/128
    const ff r2 = sqr(r);
    const float rh = r.hi;
    const float tail = r2.hi * rh * __fmaf_rn(rh, __fmaf_rn(rh, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f);
    ff p = add(r, mul_f(r2, 0.5f));
    p = add_f(p, tail);
    const int j = n & 63;
    E = n >> 6;   // floor division (arithmetic shift)
    const float2 t = T.exp2j[j];
    const ff tj{t.x, t.y};
    return add(tj, mul(tj, p));
}

// sin and cos of a float-float argument, |x| < 2^16 pi/256 (~804)
__device__ __forceinline__ void sincos_ff(ff x, const Tables& T, ff& sn, ff& cs) {
    constexpr float kInvD = 81.48733f;             // 256 / pi
    constexpr float kD1 = 0x1.92p-7f;              // pi/256 = D1 + D2 + D3, D1 with 8 bits
    constexpr float kD2 = 0x1.fb5444p-19f;
    constexpr float kD3 = 0x1.68c234p-46f;
    const float shd = __fadd_rn(__fmul_rn(x.hi, kInvD), 12582912.0f);   // as in exp_split
    const float nf = __fsub_rn(shd, 12582912.0f);
    float p2, e2;
    two_prod(nf, kD2, p2, e2);
    ff r = add_f(x, -nf * kD1);
    r = add(r, ff{-p2, -e2});
    r = add_f(r, -nf * kD3);
    // sin r = r - r^3/6 + r^5/120; cos r = 1 - r^2/2 + r^4/24 (|r| <= pi/512)
    const ff r2 = sqr(r);
    const float q = r2.hi;
    const float s3 = r.hi * q * __fmaf_rn(q, 1.0f / 120.0f, -1.0f / 6.0f);
    const ff sr = add_f(r, s3);
    ff cr = add_f(mul_f(r2, -0.5f), q * q * (1.0f / 24.0f));
    cr = add_f(cr, 1.0f);
    // angle n pi/256: j = n mod 512; quadrant j / 128, table index j mod 128
    const int n = __float_as_int(shd) - 0x4b400000;
    const int j = n & 511;
    const int quad = j >> 7, k = j & 127;
    const float4 t = T.cs[k];
    ff ca{t.x, t.y}, sa{t.z, t.w};
    if (quad & 1) {   // + pi/2: (cos, sin) -> (-sin, cos)
        const ff tmp = ca;
        ca = neg(sa);
        sa = tmp;
    }
    if (quad & 2) {   // + pi
        ca = neg(ca);
        sa = neg(sa);
    }
    // sin(a + r) = sa cr + ca sr; cos(a + r) = ca cr - sa sr
    sn = dot2(sa, cr, ca, sr);
    cs = dot2(ca, cr, neg(sa), sr);
}

// Conversion of a float-float value times 2^scale to a double with 32-bit
// integer operations only (no FP64 instruction, no 64-bit integer
// arithmetic): the 53-bit significand is assembled in two 32-bit words,
// hi's 24 bits shifted up by 29 plus lo's bits aligned below them (lo's bits
// beyond the double's 53 are truncated), renormalised by one bit when lo has
// the opposite sign and hi is a power of two.  Error below 1 ulp of the
// double.  No FP64 fallback either (it would sit, predicated, on the hot
// path): zero and denormal hi give 0 (a denormal float pair is 2^-126 below
// the kernels' unit-scaled values), infinite or NaN hi give a NaN, and
// results below or above the double's normal range give 0 or infinity.
__device__ __forceinline__ double to_double(ff a, int scale) {
    const uint32_t h = __float_as_uint(a.hi);
    const uint32_t eh = (h >> 23) & 0xffu;
    if (eh == 0u) return 0.0;                                     // zero (common: K^ of flat pairs) or denormal
    if (eh == 0xffu) return __hiloint2double(0x7ff80000, 0);       // not finite
    if ((int)eh + 896 + scale <= 0) return 0.0;
    if ((int)eh + 896 + scale >= 2047) return __hiloint2double((int)((h & 0x80000000u) | 0x7ff00000u), 0);
    const uint32_t sig = (h & 0x7fffffu) | 0x800000u;   // 24 bits
    // sh = sig << 29 as (shi, slo): bits 32.. and 0..31
    uint32_t shi = sig >> 3, slo = sig << 29;
    const uint32_t l = __float_as_uint(a.lo);
    const uint32_t el = (l >> 23) & 0xffu;
    uint32_t ml = 0u;
    if (el != 0u) {
        // lo's significand in units of 2^(eh - 52): shift left by el - eh + 29 (<= 5)
        const uint32_t sl = (l & 0x7fffffu) | 0x800000u;
        const int sft = (int)el - (int)eh + 29;
        ml = sft >= 0 ? (sl << sft) : (sft > -32 ? (sl >> -sft) : 0u);
    }
    if (((h ^ l) >> 31) == 0u) {
        const uint32_t t = slo + ml;
        shi += (t < slo) ? 1u : 0u;
        slo = t;
    } else {
        const uint32_t t = slo - ml;
        shi -= (t > slo) ? 1u : 0u;
        slo = t;
    }
    int e = (int)eh + 896 + scale;
    if (shi < (1u << 20)) {                    // below 2^52: one bit left
        shi = (shi << 1) | (slo >> 31);
        slo <<= 1;
        e -= 1;
    }
    if (e <= 0) return 0.0;   // renormalised below the normal range
    const uint32_t hw = (h & 0x80000000u) | ((uint32_t)e << 20) | (shi & 0xfffffu);
    return __hiloint2double((int)hw, (int)slo);
}

}  // namespace ffm
}  // namespace pmlbie
