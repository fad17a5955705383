// FP64 elementary functions of the sampling loops and the Taylor-polynomial
// evaluation of the Sec. 4.3 substitution, shared by the FP64 kernels
// (kernels.cu) and the mixed path's kernels (kernels_ff.cu).
#pragma once

#include "device_common.cuh"

namespace pmlbie {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 0.079577471545947667884;

// ---------------------------------------------------------------------------
// Elementary functions for the sampling loops.  The FP64 pipe of the GB300
// retires 2 FMA per SM per clock, so every FP64 instruction in the sampling
// loops counts; these versions do only what the kernels' argument ranges need.
//   exp: Cody-Waite reduction x = n ln2 + r (|r| <= ln2/2, ln2 split into a
//        40-bit head and a tail so n ln2_hi is exact), Taylor series of e^r to
//        r^13 (remainder < 2e-16 relative), 2^n built in the exponent field.
//        Arguments are clamped to [-708, 709]: results below e^-708 are
//        returned as e^-708 (~3e-308), negligible against every kernel value.
//   sin, cos: Cody-Waite reduction by pi/2 (three-part split, 33-bit heads,
//        exact products for |n| < 2^20), Taylor series to r^15 / r^16 on
//        |r| <= pi/4 (remainders < 5e-17), quadrant by integer selects.  The
//        library sincos handles |x| >= 2^19 (never reached by the kernels).
//   1/sqrt: hardware approximation refined by three Newton steps
//        y <- y (3 - x y^2)/2 (quadratic convergence from >= 12 bits).
// ---------------------------------------------------------------------------
constexpr double kRoundShift = 6755399441055744.0;   // 1.5 * 2^52
constexpr double kInvLn2 = 1.4426950408889634;
constexpr double kLn2Hi = 0.6931471805592082;        // 40 significant bits
constexpr double kLn2Lo = 7.371002565167799e-13;
constexpr double kTwoOverPi = 0.6366197723675814;
constexpr double kPio2A = 1.5707963267341256;        // 33 bits
constexpr double kPio2B = 6.077100506303966e-11;     // 33 bits
constexpr double kPio2C = 2.0222662487959506e-21;

__device__ __forceinline__ double fexp(double x) {
    x = fmin(fmax(x, -708.0), 709.0);
    double kd = fma(x, kInvLn2, kRoundShift);
    const int n = __double2loint(kd);
    kd -= kRoundShift;
    double r = fma(-kd, kLn2Hi, x);
    r = fma(-kd, kLn2Lo, r);
    double p = 1.6059043836821613e-10;   // 1/13!
    p = fma(p, r, 2.08767569878681e-09);
    p = fma(p, r, 2.505210838544172e-08);
    p = fma(p, r, 2.755731922398589e-07);
    p = fma(p, r, 2.7557319223985893e-06);
    p = fma(p, r, 2.48015873015873e-05);
    p = fma(p, r, 1.984126984126984e-04);
    p = fma(p, r, 1.388888888888889e-03);
    p = fma(p, r, 8.333333333333333e-03);
    p = fma(p, r, 4.1666666666666664e-02);
    p = fma(p, r, 1.6666666666666666e-01);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    return p * __hiloint2double((n + 1023) << 20, 0);
}

__device__ __forceinline__ void fsincos(double x, double* sp, double* cp) {
    double kd = fma(x, kTwoOverPi, kRoundShift);
    const int n = __double2loint(kd);
    if (n > (1 << 19) || n < -(1 << 19)) {
        sincos(x, sp, cp);
        return;
    }
    kd -= kRoundShift;
    double r = fma(-kd, kPio2A, x);
    r = fma(-kd, kPio2B, r);
    r = fma(-kd, kPio2C, r);
    const double r2 = r * r;
    double ps = -7.647163731819816e-13;   // -1/15!
    ps = fma(ps, r2, 1.6059043836821613e-10);
    ps = fma(ps, r2, -2.505210838544172e-08);
    ps = fma(ps, r2, 2.755731922398589e-06);
    ps = fma(ps, r2, -1.984126984126984e-04);
    ps = fma(ps, r2, 8.333333333333333e-03);
    ps = fma(ps, r2, -1.6666666666666666e-01);
    const double s = fma(ps * r2, r, r);
    double pc = 4.779477332387385e-14;    // 1/16!
    pc = fma(pc, r2, -1.1470745597729725e-11);
    pc = fma(pc, r2, 2.08767569878681e-09);
    pc = fma(pc, r2, -2.755731922398589e-07);
    pc = fma(pc, r2, 2.48015873015873e-05);
    pc = fma(pc, r2, -1.388888888888889e-03);
    pc = fma(pc, r2, 4.1666666666666664e-02);
    pc = fma(pc, r2, -0.5);
    const double c = fma(pc, r2, 1.0);
    // quadrant n mod 4: (s, c), (c, -s), (-s, -c), (-c, s)
    const bool odd = (n & 1) != 0;
    unsigned long long sv = (unsigned long long)__double_as_longlong(odd ? c : s);
    unsigned long long cv = (unsigned long long)__double_as_longlong(odd ? s : c);
    sv ^= (unsigned long long)((n >> 1) & 1) << 63;
    cv ^= (unsigned long long)(((n + 1) >> 1) & 1) << 63;
    *sp = __longlong_as_double((long long)sv);
    *cp = __longlong_as_double((long long)cv);
}

__device__ __forceinline__ double frsqrt(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double hx = 0.5 * x;
#pragma unroll
    for (int it = 0; it < 3; ++it) y = fma(y, fma(-hx * y, y, 0.5), y);
    return y;
}

// e^{i q} with the functions above
__device__ __forceinline__ double2 fcexpi(double2 q) {
    double s, c;
    fsincos(q.x, &s, &c);
    const double m = fexp(-q.y);
    return c2(m * c, m * s);
}

// Principal square root R of z (z not 0) and 1/R = conj(R)/|z|, from two
// reciprocal square roots.  Cancellation-free on both half planes.
__device__ __forceinline__ void fcsqrt_rcp(double2 z, double2& R, double2& iR) {
    const double m2 = fma(z.x, z.x, z.y * z.y);
    const double ir = frsqrt(m2);                  // 1/|z|
    const double r = m2 * ir;                      // |z|
    const double u = 0.5 * (r + fabs(z.x));
    const double it = frsqrt(u);
    const double t = u * it;                       // sqrt((|z| + |Re z|)/2)
    const double s = 0.5 * z.y * it;               // Im z / (2 t)
    R = z.x >= 0.0 ? c2(t, s) : c2(fabs(s), copysign(t, z.y));
    iR = c2(R.x * ir, -R.y * ir);
}

// sum_{k = k0}^{L} c_k q^{k - k0} by Horner, L <= 7 (unrolled: static indices)
__device__ __forceinline__ double2 cpoly_from(const double2 (&c)[8], int k0, int L, double2 q) {
    double2 r = c2(0.0, 0.0);
#pragma unroll
    for (int k = 7; k >= 0; --k)
        if (k >= k0 && k <= L) r = cadd(cmul(r, q), c[k]);
    return r;
}

}  // namespace
}  // namespace pmlbie
