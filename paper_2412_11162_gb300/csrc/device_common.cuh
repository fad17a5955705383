// Device helpers shared by the FP64 kernels (kernels.cu) and the
// float-float kernels of the mixed path (kernels_ff.cu): complex128
// arithmetic and the geometry of a grid node pair.
#pragma once

#include "internal.h"

namespace pmlbie {
namespace {

// ---------------------------------------------------------------------------
// complex helpers (double2 = re, im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 c2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return c2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return c2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return c2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 crcp(double2 a) {
    // 1/a with scaling against overflow
    double s = fmax(fabs(a.x), fabs(a.y));
    double ax = a.x / s, ay = a.y / s;
    double d = ax * ax + ay * ay;
    return c2(ax / (d * s), -ay / (d * s));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return cmul(a, crcp(b)); }
// principal square root (branch cut on the negative real axis)
__device__ __forceinline__ double2 csqrt(double2 z) {
    double r = hypot(z.x, z.y);
    if (r == 0.0) return c2(0.0, 0.0);
    if (z.x >= 0.0) {
        double t = sqrt(0.5 * (r + z.x));
        return c2(t, z.y / (2.0 * t));
    }
    double t = sqrt(0.5 * (r - z.x));
    return c2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}
// e^{i q}
__device__ __forceinline__ double2 cexpi(double2 q) {
    double s, c;
    sincos(q.x, &s, &c);
    double m = exp(-q.y);
    return c2(m * c, m * s);
}
__device__ __forceinline__ double2 clog(double2 z) { return c2(log(hypot(z.x, z.y)), atan2(z.y, z.x)); }

// Geometry of a grid pair (l, m) from node tables: the symmetric sampling
// quantities d~^2 and rho~_l rho~_m, and for both orientations the normal
// factor N_D(psi) = nd0 + nds sin^2(psi/2) of the double layer at the source
// (target l, source m: nu'_r (rho~_m - rho~_l) + nu'_z (z_m - z_l) + 2 nu'_r
// rho~_l sin^2(psi/2) with nu' the conormal at m; target m, source l: the same
// with l and m exchanged).
struct PairGeom {
    double2 d2, rr;
    double2 nd0, nds;   // target l, source m
    double2 nd0t, ndst; // target m, source l
};

__device__ __forceinline__ PairGeom grid_pair(const DeviceTables& T, int l, int m) {
    PairGeom g;
    // separations from breakpoint offsets when both nodes share the nearest
    // breakpoint (graded clusters), else from the absolute positions
    double dr, dz;
    if (T.bk[l] == T.bk[m]) {
        dr = T.off[l].x - T.off[m].x;
        dz = T.off[l].y - T.off[m].y;
    } else {
        dr = T.rho[l] - T.rho[m];
        dz = T.z[l] - T.z[m];
    }
    double dI = T.I[l] - T.I[m];
    double2 drt = c2(dr, dI);
    g.d2 = cadd(cmul(drt, drt), c2(dz * dz, 0.0));
    g.rr = cmul(T.rho_t[l], T.rho_t[m]);
    // nu'_r (rho~' - rho~ cos psi) + nu'_z (z' - z)
    //   = [nu'_r (rho~' - rho~) + nu'_z (z' - z)] + 2 nu'_r rho~ sin^2(psi/2)
    g.nd0 = cadd(cmul(T.nuc_r[m], c2(-dr, -dI)), cscale(T.nuc_z[m], -dz));
    g.nds = cscale(cmul(T.nuc_r[m], T.rho_t[l]), 2.0);
    g.nd0t = cadd(cmul(T.nuc_r[l], drt), cscale(T.nuc_z[l], dz));
    g.ndst = cscale(cmul(T.nuc_r[l], T.rho_t[m]), 2.0);
    return g;
}

}  // namespace
}  // namespace pmlbie
