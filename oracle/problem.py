"""Oracle: problem data, generating curve, graded grid and PML tables (FP64).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow restatement of the
method of Wang & Lu, "An FFT-accelerated PML-BIE solver for 3D acoustic wave
scattering in layered media" (arXiv 2412.11162).  Only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
library never does.

Sections followed here:
  * Sec. 2 (problem statement): wavenumbers omega_1 (above) and omega_2 (below),
    interface Gamma = flat plane z = 0 plus an axisymmetric perturbation, unit
    normal nu pointing toward Omega_2.
  * Sec. 3.1, Eqs. (rhot), (zt), (sgm1): complex stretching
    rho~ = rho + i int_0^rho sigma_1, with the smooth profile sigma_1.
  * Sec. 3.1, Eq. (g1t) and the line after it: conormal nu_c = A^T nu.
  * Sec. 4 intro, Eq. (sxi): graded parametrisation of each smooth segment.

Readings taken where the paper is silent or garbled:
  * Eq. (sxi) maps t^0 to s^1 as printed; the orientation is flipped so that
    t^0 -> s^0.  Each segment uses its own regular parameter s in [0, 1]
    (the paper says arclength; any regular parameter gives the same graded
    integrand smoothness).
  * One global uniform grid t_i = i h, i = 0..Nt, h = 1/Nt; each segment gets a
    whole number of steps proportional to its length.  Breakpoints (the axis
    point A, corners, the PML end B) have |r'| = 0 and carry no unknown, so
    the N unknowns are the Nt + 1 - (#breakpoints) interior grid nodes.
  * The Gaussian bump of the benchmark workloads is taken as
    z = h (e^{-r^2/w} - e^{-R^2/w}) / (1 - e^{-R^2/w}) for r <= R (continuous,
    peak height h, a corner at r = R).
  * sigma_2 is inert on gamma_AB (all curve points have |z| < a_2), so
    z~ = z and alpha_z = 1 on the curve.
  * A segment that starts on the axis with a change in z (a conical point of
    the surface, Sec. 5 Example 2) is graded with exponent 2 instead of p;
    the paper gives no treatment of such a tip (see kConicalP).
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Params:
    """Problem statement (Sec. 2, Sec. 3.1, Sec. 5)."""
    k1: float                      # omega_1, upper medium Omega_1
    k2: float                      # omega_2, lower medium Omega_2
    N: int = 128                   # unknown nodes on gamma_AB
    M: int = 64                    # azimuthal samples; modes n = 0..M/2-1
    a1: float = 2.5                # PML start radius
    T: float = 1.0                 # PML thickness
    S: float = 3.0                 # PML strength
    p: int = 6                     # PML profile and grading exponent
    curve: str = "gauss"           # "gauss" | "polyline" | "wavy"
    bump_h: float = 0.2
    bump_w: float = 0.5            # exp(-r^2 / bump_w)
    bump_R: float = 1.0
    vertices: Optional[List[Tuple[float, float]]] = None  # polyline (rho, z), from the axis
    wavy_R: float = 1.0            # wavy dent (Sec. 5, Example 2): radius,
    wavy_eps: float = 0.1          # relative amplitude
    wavy_m: int = 3                # and number of half-waves of the perturbation
    polar: float = np.pi / 6.0     # incidence polar angle phi_inc
    azimuth: float = 0.0           # incidence azimuth theta_inc
    taylor_L: int = 5              # order of the cH_1 / cH_3 substitution (Sec. 4.3)
    subst: bool = True             # False: the exact split on PML pairs too (the "without
                                   # cH_1" arm of the Sec. 4.3 experiment)
    split_c: float = 8.0          # near-pair threshold eta_s = split_c * 2 pi / M

    @property
    def L(self):
        return self.a1 + self.T

    @property
    def eta_split(self):
        return self.split_c * TWO_PI / self.M


# ----------------------------------------------------------------------------
# generating curve: list of segments, each r(s), r_s(s) for s in [0, 1]
# ----------------------------------------------------------------------------
class _Segment:
    def __init__(self, kind, data, p=None):
        self.kind = kind
        self.data = data
        self.p = p            # grading exponent of this segment (None: Params.p)

    def eval(self, s):
        s = np.asarray(s, dtype=float)
        if self.kind == "wavy":
            # Sec. 5, Example 2: rho = f sin(pi s / 2), z = -f cos(pi s / 2),
            # f = R (1 - eps sin(m pi s)), from (0, -R) on the axis to (R, 0)
            R, eps, m = self.data
            f = R * (1.0 - eps * np.sin(m * np.pi * s))
            df = -R * eps * m * np.pi * np.cos(m * np.pi * s)
            c, si = np.cos(0.5 * np.pi * s), np.sin(0.5 * np.pi * s)
            return f * si, -f * c, df * si + 0.5 * np.pi * f * c, -df * c + 0.5 * np.pi * f * si
        if self.kind == "gauss":
            h, w, R = self.data
            rho = R * s
            e0 = np.exp(-R * R / w)
            g = np.exp(-rho * rho / w)
            z = h * (g - e0) / (1.0 - e0)
            dz = h * (-2.0 * rho / w) * g / (1.0 - e0)   # dz/drho
            return rho, z, R * np.ones_like(s), R * dz
        (r0, z0), (r1, z1) = self.data
        return r0 + s * (r1 - r0), z0 + s * (z1 - z0), (r1 - r0) * np.ones_like(s), (z1 - z0) * np.ones_like(s)

    def offset(self, s, sc, end):
        """r(s) - r(0) (end = 0) or r(s) - r(1) (end = 1), free of cancellation;
        sc = 1 - s computed separately."""
        if self.kind == "wavy":
            # 1 - cos(x) = 2 sin^2(x/2); near s = 1, sin(m pi s) = (-1)^(m+1) sin(m pi sc)
            # (m integer) and sin(pi s / 2) = cos(pi sc / 2)
            R, eps, m = self.data
            if end == 0:
                rho, _, _, _ = self.eval(s)
                return rho, 2.0 * R * np.sin(0.25 * np.pi * s) ** 2 + R * eps * np.sin(m * np.pi * s) * np.cos(
                    0.5 * np.pi * s)
            sm = (-1.0) ** (m + 1) * np.sin(m * np.pi * sc)
            f = R * (1.0 - eps * sm)
            return (-2.0 * R * np.sin(0.25 * np.pi * sc) ** 2 - R * eps * sm * np.cos(0.5 * np.pi * sc),
                    -f * np.sin(0.5 * np.pi * sc))
        if self.kind == "gauss":
            h, w, R = self.data
            c = h / (1.0 - np.exp(-R * R / w))
            if end == 0:
                return R * s, c * np.expm1(-(R * s) ** 2 / w)
            return -R * sc, c * np.exp(-R * R / w) * np.expm1(R * R * sc * (1.0 + s) / w)
        (r0, z0), (r1, z1) = self.data
        if end == 0:
            return s * (r1 - r0), s * (z1 - z0)
        return -sc * (r1 - r0), -sc * (z1 - z0)

    def length(self):
        x, wq = np.polynomial.legendre.leggauss(64)
        s = 0.5 * (x + 1.0)
        _, _, dr, dz = self.eval(s)
        return 0.5 * np.sum(wq * np.hypot(dr, dz))


# Grading exponent of a segment that leaves the axis at an angle (the surface
# has a conical point there).  With the Sec. 5 exponent 6 the graded nodes
# next to the tip sit at rho ~ 1e-8 .. 1e-6, where the double-layer kernel
# of the targets scales like 1/rho^2 over neighbours spaced geometrically in
# rho, and the Alpert-corrected rule does not resolve it; exponent 2 keeps
# the tip nodes at rho ~ h^2.
kConicalP = 2


def build_segments(P: Params):
    L = P.L
    segs = []
    if P.curve == "gauss":
        segs.append(_Segment("gauss", (P.bump_h, P.bump_w, P.bump_R)))
        segs.append(_Segment("line", ((P.bump_R, 0.0), (L, 0.0))))
    elif P.curve == "wavy":
        # leaves the axis at an angle (a conical point): grading exponent 2
        segs.append(_Segment("wavy", (P.wavy_R, P.wavy_eps, int(P.wavy_m)), p=kConicalP))
        segs.append(_Segment("line", ((P.wavy_R, 0.0), (L, 0.0))))
    elif P.curve == "polyline":
        V = list(P.vertices)
        for i, (a, b) in enumerate(zip(V[:-1], V[1:])):
            # a first segment that leaves the axis at an angle: grading exponent 2
            conical = i == 0 and abs(b[1] - a[1]) > 0.0
            segs.append(_Segment("line", (tuple(a), tuple(b)), p=kConicalP if conical else None))
        if abs(V[-1][0] - L) > 1e-14 or abs(V[-1][1]) > 1e-14:
            segs.append(_Segment("line", (tuple(V[-1]), (L, 0.0))))
    else:
        raise ValueError("unknown curve kind")
    return segs


def segment_steps(lengths, Nt, min_steps):
    """Whole number of grid steps per segment, proportional to length."""
    tot = sum(lengths)
    steps = [max(min_steps, int(round(Nt * l / tot))) for l in lengths]
    # fix the total by adjusting the longest segment
    steps[int(np.argmax(lengths))] += Nt - sum(steps)
    if min(steps) < min_steps:
        raise ValueError("too few nodes for the number of segments")
    return steps


# ----------------------------------------------------------------------------
# graded map, Eq. (sxi) with t^0 -> s^0
# ----------------------------------------------------------------------------
def graded(u, p):
    """s(u) and ds/du for the local coordinate u in [0, 1] of one segment.

    xi = 2u - 1; xi_1 = (1/2 - 1/p) xi^3 + xi/p + 1/2, xi_2 = 1 - xi_1;
    s = xi_1^p / (xi_1^p + xi_2^p).  xi_1 and xi_2 are evaluated in the
    factored forms (xi+1)(A xi^2 - A xi + 1/2) and (1-xi)(A xi^2 + A xi + 1/2),
    A = 1/2 - 1/p, which are exact rewrites of the cubic.
    """
    u = np.asarray(u, dtype=float)
    xi = 2.0 * u - 1.0
    A = 0.5 - 1.0 / p
    x1 = (2.0 * u) * (A * xi * xi - A * xi + 0.5)
    x2 = (2.0 * (1.0 - u)) * (A * xi * xi + A * xi + 0.5)
    x1p, x2p = x1 ** p, x2 ** p
    den = x1p + x2p
    s = x1p / den
    dx1 = 3.0 * A * xi * xi + 1.0 / p                  # d xi_1 / d xi
    ds = p * x1 ** (p - 1) * x2 ** (p - 1) / (den * den) * dx1 * 2.0
    return s, ds


def graded_complement(u, p):
    """1 - s(u) = xi_2^p / (xi_1^p + xi_2^p), without cancellation near u = 1."""
    u = np.asarray(u, dtype=float)
    xi = 2.0 * u - 1.0
    A = 0.5 - 1.0 / p
    x1 = (2.0 * u) * (A * xi * xi - A * xi + 0.5)
    x2 = (2.0 * (1.0 - u)) * (A * xi * xi + A * xi + 0.5)
    return x2 ** p / (x1 ** p + x2 ** p)


class Geometry:
    """Nodes, weights and PML tables of gamma_AB for one Params."""

    def __init__(self, P: Params, alpert_a: int = 10):
        self.P = P
        self.segs = build_segments(P)
        lens = [s.length() for s in self.segs]
        nseg = len(self.segs)
        # unknowns N = (Nt + 1) - (nseg + 1)  =>  Nt = N + nseg
        self.Nt = P.N + nseg
        self.h = 1.0 / self.Nt
        self.steps = segment_steps(lens, self.Nt, 2 * alpert_a + 4)
        self.brk = np.concatenate([[0], np.cumsum(self.steps)]).astype(int)   # breakpoint grid indices
        grid = np.arange(self.Nt + 1)
        is_brk = np.zeros(self.Nt + 1, bool)
        is_brk[self.brk] = True
        self.unk_grid = grid[~is_brk]           # grid index of each unknown
        assert len(self.unk_grid) == P.N
        self.unk_of_grid = -np.ones(self.Nt + 1, int)
        self.unk_of_grid[self.unk_grid] = np.arange(P.N)
        self.nodes = self.at(self.unk_grid * self.h)

    # ---- curve evaluation at arbitrary t in [0, 1] ----
    def at(self, t):
        """Dict of per-point quantities at parameter values t (array)."""
        P = self.P
        t = np.atleast_1d(np.asarray(t, dtype=float))
        seg = np.clip(np.searchsorted(self.brk * self.h, t, side="right") - 1, 0, len(self.segs) - 1)
        rho = np.empty_like(t)
        z = np.empty_like(t)
        drho = np.empty_like(t)
        dz = np.empty_like(t)
        bk = np.empty(t.shape, int)      # nearest breakpoint (global index)
        ox = np.empty_like(t)            # r - r(breakpoint), accurate
        oz = np.empty_like(t)
        for k, sg in enumerate(self.segs):
            m = seg == k
            if not np.any(m):
                continue
            t0 = self.brk[k] * self.h
            t1 = self.brk[k + 1] * self.h
            u = (t[m] - t0) / (t1 - t0)
            pk = sg.p or P.p
            s, ds = graded(u, pk)
            sc = graded_complement(u, pk)
            r_, z_, dr_, dz_ = sg.eval(s)
            rho[m] = r_
            z[m] = z_
            scale = ds / (t1 - t0)
            drho[m] = dr_ * scale
            dz[m] = dz_ * scale
            end = (u > 0.5).astype(int)
            o0 = sg.offset(s, sc, 0)
            o1 = sg.offset(s, sc, 1)
            ox[m] = np.where(end == 1, o1[0], o0[0])
            oz[m] = np.where(end == 1, o1[1], o0[1])
            bk[m] = k + end
        speed = np.hypot(drho, dz)                       # |r'(t)|
        with np.errstate(invalid="ignore", divide="ignore"):
            nu_r = np.where(speed > 0, dz / speed, 0.0)    # tangent rotated by -90 deg:
            nu_z = np.where(speed > 0, -drho / speed, -1.0)  # points toward Omega_2
        I = pml_integral(rho, P)
        sig = pml_sigma(rho, P)
        alpha = 1.0 + 1j * sig
        rho_t = rho + 1j * I
        with np.errstate(invalid="ignore", divide="ignore"):
            ratio = np.where(rho > 0, rho_t / np.where(rho > 0, rho, 1.0), 1.0 + 0j)
        nuc_r = nu_r * ratio / alpha              # nu_rho rho~ alpha_z / (rho alpha_rho), alpha_z = 1
        nuc_z = nu_z * ratio * alpha              # nu_z rho~ alpha_rho / (rho alpha_z)
        return dict(t=t, rho=rho, z=z, speed=speed, nu_r=nu_r, nu_z=nu_z,
                    I=I, rho_t=rho_t, z_t=z.astype(complex), nuc_r=nuc_r, nuc_z=nuc_z,
                    W=2.0 * rho * speed, bk=bk, ox=ox, oz=oz)


def separation(tgt, src):
    """(rho_t - rho_s, z_t - z_s); from the breakpoint offsets when both points
    are nearest to the same breakpoint (close pairs at graded clusters, whose
    separation is below the spacing of FP64 absolute positions)."""
    same = tgt["bk"] == src["bk"]
    dr = np.where(same, tgt["ox"] - src["ox"], tgt["rho"] - src["rho"])
    dz = np.where(same, tgt["oz"] - src["oz"], tgt["z"] - src["z"])
    return dr, dz


# ----------------------------------------------------------------------------
# PML, Eq. (sgm1): sigma_1 = 2 S f1^p / (f1^p + f2^p) on [a1, a1 + T]
# ----------------------------------------------------------------------------
def pml_sigma(rho, P: Params):
    rho = np.asarray(rho, dtype=float)
    rb = (rho - P.L) / P.T
    f1 = (0.5 - 1.0 / P.p) * rb ** 3 + rb / P.p + 0.5
    f2 = 1.0 - f1
    inside = (rho > P.a1)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        val = 2.0 * P.S * f1 ** P.p / (f1 ** P.p + f2 ** P.p)
    val = np.where(rho >= P.L, P.S, val)
    return np.where(inside, val, 0.0)


_GL16 = np.polynomial.legendre.leggauss(16)


def _sigma_integral(lo, hi, P: Params, panels=64):
    """int_lo^hi sigma_1 by composite 16-point Gauss-Legendre (lo, hi arrays)."""
    x, w = _GL16
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    tot = np.zeros(np.broadcast(lo, hi).shape)
    for k in range(panels):
        a = lo + (hi - lo) * k / panels
        b = lo + (hi - lo) * (k + 1) / panels
        mid = 0.5 * (a + b)
        half = 0.5 * (b - a)
        pts = mid[..., None] + half[..., None] * x
        tot = tot + half * np.sum(w * pml_sigma(pts, P), axis=-1)
    return tot


def pml_integral(rho, P: Params):
    """I(rho) = int_0^rho sigma_1(t) dt (zero for rho <= a1)."""
    rho = np.asarray(rho, dtype=float)
    lo = np.full_like(rho, P.a1)
    hi = np.maximum(rho, P.a1)
    return _sigma_integral(lo, hi, P)


def delta_I(rho2, drho, P: Params):
    """I(rho2 + drho) - I(rho2) = int_{rho2}^{rho2 + drho} sigma_1, integrated
    directly.  sigma_1 vanishes below a1 and is only C^(p-1) there, so the
    interval is clipped at a1; when both ends lie in the PML the integral runs
    over [rho2, rho2 + drho] with drho given accurately (no cancellation)."""
    rho2 = np.asarray(rho2, float)
    drho = np.asarray(drho, float)
    rho2, drho = np.broadcast_arrays(rho2, drho)
    lo = np.minimum(rho2, rho2 + drho)
    hi = np.maximum(rho2, rho2 + drho)
    inside = lo >= P.a1
    start = np.where(inside, rho2, P.a1)
    length = np.where(inside, drho, np.maximum(hi - P.a1, 0.0) * np.sign(drho))
    x, w = _GL16
    tot = np.zeros(rho2.shape)
    panels = 8
    for k in range(panels):
        xs = (k + 0.5 * (x + 1.0)) / panels
        pts = np.where(inside[..., None], start[..., None] + length[..., None] * xs,
                       start[..., None] + np.abs(length)[..., None] * xs)
        tot = tot + np.sum((0.5 / panels) * w * pml_sigma(pts, P), axis=-1)
    return length * tot
