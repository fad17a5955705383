"""Oracle: Alpert quadrature, per-mode matrices, diagonal D, right-hand sides.

TEST INFRASTRUCTURE ONLY (see oracle/problem.py).

Follows:
  * Sec. 4.1, Eqs. (snab), (snab1), (snt1): hybrid Gauss-trapezoid rule of
    Alpert (order 10, Sec. 5) around the log singularity at t_l, with the
    off-grid density values from Lagrange interpolation on the grid.
  * Sec. 3.3, Eq. (6) and Sec. 4.1 (matrix D): diagonal
    D_l = K0_AB 1 (r_l) + K0_+ 1 (r_l); Sec. 3.2, Lemmas 3.1-3.3: K0 1 is the
    solid-angle term, K0_+ 1 the solid angle of the PML/top surface, which
    through the rim circle equals that of the disc rho <= a1 + T, z = 0.
  * Sec. 2 (reference field u^{tot,0}, Fresnel R, k*) and Sec. 4.2 (b^1, b^2).

Readings (where the paper is silent):
  * the unknown densities are u_n and phi_n = |r'| dnu_c u_n (the paper's phi,
    Sec. 4.1-4.2); the source weight is W_u = 2 rho |r'| for u and
    W_phi = 2 rho for phi (factor 2 and rho' of Eqs. (snpml)-(k0pml)), and
    the weighted density W * density is what the 10-point Lagrange stencil
    interpolates (it vanishes at breakpoints, so stencils may cross them).
  * correction nodes t_l +- x_k h outside [0, 1] are dropped (the graded
    integrand is extended by zero) instead of the paper's rescaling rule.
  * K0 1 is computed with the same normal as K, i.e. the outward normal of
    each region (the printed sign of Lemma 3.1 corresponds to the inward
    normal); K0_AB 1 uses the unstretched Laplace kernel and physical normal.
  * region b (Omega_2 side) uses omega_2 and the normal nu_b = -nu.
"""
import numpy as np
import os

from .problem import Params, Geometry, separation
from . import kernels as KR

_TABLE = os.path.join(os.path.dirname(__file__), "alpert_log_j10_a10.txt")
STENCIL = 10


def alpert_table():
    rows = [l.split() for l in open(_TABLE) if not l.startswith("#")]
    x = np.array([float(r[0]) for r in rows])
    w = np.array([float(r[1]) for r in rows])
    return x, w, 10          # nodes, weights, skip a


def lagrange_weights(tau, Nt, h):
    """First grid index and the 10 Lagrange basis values at tau (uniform grid)."""
    i0 = int(np.floor(tau / h)) - (STENCIL // 2 - 1)
    i0 = min(max(i0, 0), Nt + 1 - STENCIL)
    idx = i0 + np.arange(STENCIL)
    tj = idx * h
    L = np.ones(STENCIL)
    for a in range(STENCIL):
        for b in range(STENCIL):
            if a != b:
                L[a] *= (tau - tj[b]) / (tj[a] - tj[b])
    return idx, L


class Quadrature:
    """The Alpert rule for every target node: grid part and correction part."""

    def __init__(self, G: Geometry):
        self.G = G
        x, w, a = alpert_table()
        self.x, self.w, self.a = x, w, a
        N, h, Nt = G.P.N, G.h, G.Nt
        gi = G.unk_grid
        # grid part: coefficient h W_m where |i_m - i_l| >= a
        self.grid_mask = np.abs(gi[:, None] - gi[None, :]) >= a
        # correction points
        tl, tau, coef_rows = [], [], []
        for l in range(N):
            for sgn in (-1.0, 1.0):
                for k in range(len(x)):
                    t = gi[l] * h + sgn * x[k] * h
                    if t <= 0.0 or t >= 1.0:
                        continue
                    idx, Lw = lagrange_weights(t, Nt, h)
                    c = np.zeros(N)
                    for i, lv in zip(idx, Lw):
                        m = G.unk_of_grid[i]
                        if m >= 0:
                            c[m] += w[k] * h * lv
                    tl.append(l)
                    tau.append(t)
                    coef_rows.append(c)
        self.corr_target = np.array(tl, int)
        self.corr_tau = np.array(tau)
        self.corr_coef = np.array(coef_rows)           # (ncorr, N): w_k h L_m(tau)
        self.corr_pts = G.at(self.corr_tau)
        self.W_u = G.nodes["W"]                        # 2 rho |r'|
        self.W_phi = 2.0 * G.nodes["rho"]              # 2 rho

    def assemble(self, Fgrid, Fcorr, weight):
        """Matrix from grid-pair values Fgrid (N, N), correction values (ncorr,)
        and the source weight vector (W_u or W_phi)."""
        G = self.G
        A = np.where(self.grid_mask, Fgrid, 0.0) * G.h
        np.add.at(A, self.corr_target, Fcorr[:, None] * self.corr_coef)
        return A * weight[None, :]


def _take(d, idx):
    return {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in d.items()}


def _region_nodes(d, sign):
    out = dict(d)
    out["nuc_r"] = sign * d["nuc_r"]
    out["nuc_z"] = sign * d["nuc_z"]
    out["nu_r"] = sign * d["nu_r"]
    out["nu_z"] = sign * d["nu_z"]
    return out


class ModalSystem:
    """All modal kernels on the grid and correction pairs, both regions."""

    def __init__(self, P: Params, G: Geometry = None, Q: Quadrature = None):
        self.P = P
        self.G = G or Geometry(P)
        self.Q = Q or Quadrature(self.G)
        G, Q = self.G, self.Q
        N = P.N
        li, mi = np.nonzero(Q.grid_mask)
        self.grid_pairs = (li, mi)
        tg = _take(G.nodes, li)
        sg = _take(G.nodes, mi)
        tc = _take(G.nodes, Q.corr_target)
        sc = Q.corr_pts
        # stacked pair list: grid pairs then correction pairs
        tgt = {k: np.concatenate([tg[k], tc[k]]) for k in ("rho", "z", "z_t", "rho_t", "bk", "ox", "oz")}
        src = {k: np.concatenate([sg[k], sc[k]]) for k in ("rho", "z", "z_t", "rho_t", "nuc_r", "nuc_z", "bk", "ox", "oz")}
        self.pg = KR.pair_geometry(tgt, src, P)
        self.near = KR.near_mask(self.pg, P)
        self.ngrid = len(li)
        nsub = {k: v[self.near] for k, v in self.pg.items()}
        Zm, Dm = KR.laplace_modes(nsub, P.M - 2)
        self.lap_near = (Zm, Dm)
        self.kern = {}
        for reg, omega, sign in (("a", P.k1, 1.0), ("b", P.k2, -1.0)):
            pg = dict(self.pg)
            pg["nuc_r"] = sign * self.pg["nuc_r"]
            pg["nuc_z"] = sign * self.pg["nuc_z"]
            lap = (np.zeros((len(self.near), P.M - 1), complex), np.zeros((len(self.near), P.M - 1), complex))
            lap[0][self.near] = Zm
            lap[1][self.near] = sign * Dm
            S, K = KR.modal_kernels(pg, omega, P, lap=lap, near=self.near)
            self.kern[reg] = (S, K)

    def grid_kernel(self, reg, which, n):
        """Modal kernel values F^_n(r_l, r_m) on all grid pairs (0 where skipped)."""
        N = self.P.N
        S, K = self.kern[reg]
        F = (S if which == "S" else K)[: self.ngrid, n]
        out = np.zeros((N, N), complex)
        out[self.grid_pairs] = F
        return out

    def matrices(self, reg, n):
        S, K = self.kern[reg]
        Sg = self.grid_kernel(reg, "S", n)
        Kg = self.grid_kernel(reg, "K", n)
        Sm = self.Q.assemble(Sg, S[self.ngrid:, n], self.Q.W_phi)
        Km = self.Q.assemble(Kg, K[self.ngrid:, n], self.Q.W_u)
        return Sm, Km


# ----------------------------------------------------------------------------
# diagonal term D (Sec. 3.2, Lemmas 3.1-3.3; Sec. 4.1)
# ----------------------------------------------------------------------------
def laplace_dl_mode0(tgt, src):
    """int_{-pi}^{pi} dG0/dnu' dpsi for the unstretched Laplace kernel (quadrature)."""
    pts, wts = KR.psi_rule(8)
    dr, dzz = separation(tgt, src)
    drho = dr[:, None]
    dz = dzz[:, None]
    s = np.sin(0.5 * pts)[None, :]
    R2 = drho * drho + dz * dz + 4.0 * tgt["rho"][:, None] * src["rho"][:, None] * s * s
    num = src["nu_r"][:, None] * (-drho + 2.0 * tgt["rho"][:, None] * s * s) \
        + src["nu_z"][:, None] * (-dz)
    F = -num / (4.0 * np.pi * R2 ** 1.5)
    return 2.0 * (F * wts[None, :]).sum(axis=1)


def disc_solid_angle(rho, z, Lr):
    """Solid angle of the disc {rho' <= Lr, z' = 0} seen from (rho, 0, z), rho < Lr.

    Omega = int_0^{2pi} [1 - |z| / sqrt(z^2 + s(th)^2)] dth, s(th) the distance
    in the plane from the foot point to the rim along direction th.  The
    integrand is smooth and 2 pi-periodic for rho < Lr, so the periodic
    trapezoid rule converges geometrically; it is applied to the second term
    alone (Omega = 2 pi - int |z| / sqrt(z^2 + s^2)), doubling the number of
    points until two successive sums agree to 1e-15 x 2 pi.
    """
    out = np.empty(len(rho))
    for i, (r, h) in enumerate(zip(rho, z)):
        if h == 0.0:
            out[i] = 2.0 * np.pi
            continue
        n, prev = 64, None
        while True:
            th = 2.0 * np.pi * np.arange(n) / n
            s = -r * np.cos(th) + np.sqrt(Lr * Lr - (r * np.sin(th)) ** 2)
            val = (2.0 * np.pi / n) * np.sum(abs(h) / np.sqrt(h * h + s * s))
            if prev is not None and abs(val - prev) <= 1e-15 * 2.0 * np.pi:
                break
            if n >= 1 << 22:
                raise RuntimeError("disc solid angle: trapezoid sums did not settle")
            prev, n = val, 2 * n
        out[i] = 2.0 * np.pi - val
    return out


def diagonal(G: Geometry, Q: Quadrature):
    """D^a, D^b at the unknown nodes (region a: outward normal nu, region b: -nu)."""
    N = G.P.N
    li, mi = np.nonzero(Q.grid_mask)
    vals = laplace_dl_mode0(_take(G.nodes, li), _take(G.nodes, mi))
    Fg = np.zeros((N, N))
    Fg[li, mi] = vals
    Fc = laplace_dl_mode0(_take(G.nodes, Q.corr_target), Q.corr_pts)
    K0 = Q.assemble(Fg, Fc, Q.W_u).real
    K0AB = K0.sum(axis=1)
    rho, z = G.nodes["rho"], G.nodes["z"]
    Od = disc_solid_angle(rho, z, G.P.L)
    Om_plus = np.where(z > 0, 4.0 * np.pi - Od, np.where(z < 0, Od, 2.0 * np.pi))
    Da = K0AB - Om_plus / (2.0 * np.pi)
    Db = -K0AB - (4.0 * np.pi - Om_plus) / (2.0 * np.pi)
    return Da, Db


# ----------------------------------------------------------------------------
# reference field and right-hand side (Sec. 2; Sec. 4.2)
# ----------------------------------------------------------------------------
def fresnel(P: Params):
    w1, w2, ph = P.k1, P.k2, P.polar
    kx = w1 * np.sin(ph)
    if w2 > abs(kx):
        ks = np.sqrt(w2 * w2 - kx * kx) + 0j
    else:
        ks = 1j * np.sqrt(kx * kx - w2 * w2)
    R = 2.0 / (1.0 + ks / (w1 * np.cos(ph))) - 1.0
    return R, ks


def reference_field(P: Params, x, y, z):
    """(u1, grad u1, u2, grad u2): the Omega_1 and Omega_2 formulas at (x, y, z)."""
    R, ks = fresnel(P)
    w1, ph, th = P.k1, P.polar, P.azimuth
    ax, ay = -w1 * np.sin(ph) * np.cos(th), -w1 * np.sin(ph) * np.sin(th)
    az = w1 * np.cos(ph)
    lat = np.exp(1j * (ax * x + ay * y))
    ui = lat * np.exp(-1j * az * z)
    ur = R * lat * np.exp(1j * az * z)
    u1 = ui + ur
    g1 = (1j * ax * u1, 1j * ay * u1, -1j * az * ui + 1j * az * ur)
    u2 = (R + 1.0) * lat * np.exp(-1j * ks * z)
    g2 = (1j * ax * u2, 1j * ay * u2, -1j * ks * u2)
    return u1, g1, u2, g2


def rhs_modes(G: Geometry):
    """b^1_n = -[u^{tot,0}]_n, b^2_n = -|r'| [d_nu u^{tot,0}]_n at the nodes (M-point DFT)."""
    P = G.P
    M = P.M
    th = 2.0 * np.pi * np.arange(M) / M
    rho, z = G.nodes["rho"][:, None], G.nodes["z"][:, None]
    nr, nz = G.nodes["nu_r"][:, None], G.nodes["nu_z"][:, None]
    x, y = rho * np.cos(th)[None, :], rho * np.sin(th)[None, :]
    zz = z * np.ones_like(x)
    u1, g1, u2, g2 = reference_field(P, x, y, zz)
    c, s = np.cos(th)[None, :], np.sin(th)[None, :]
    dn1 = nr * (g1[0] * c + g1[1] * s) + nz * g1[2]
    dn2 = nr * (g2[0] * c + g2[1] * s) + nz * g2[2]
    E = KR.dft_matrix(M)
    b1 = -((u1 - u2) @ E)
    b2 = -((dn1 - dn2) @ E) * G.nodes["speed"][:, None]
    return b1, b2            # (N, M/2) each


# ----------------------------------------------------------------------------
# solve (Sec. 4.2): the NtD route of the paper
# ----------------------------------------------------------------------------
def solve_ntd(Sa, Ka, Da, Sb, Kb, Db, b1, b2):
    """phi1 = (N1 - N2)^{-1} (b1 - N2 b2), u1 = N1 phi1; N1 = (Ka-Da)^{-1} Sa,
    N2 = -(Kb-Db)^{-1} Sb (the minus sign from nu_b = -nu)."""
    N1 = np.linalg.solve(Ka - np.diag(Da), Sa)
    N2 = -np.linalg.solve(Kb - np.diag(Db), Sb)
    phi1 = np.linalg.solve(N1 - N2, b1 - N2 @ b2)
    u1 = N1 @ phi1
    return u1, phi1, u1 - b1, phi1 - b2


def block_system(Sa, Ka, Da, Sb, Kb, Db, b1, b2):
    """A x = B with x = (u1, phi1): rows [Ka-Da, -Sa; Kb-Db, Sb]."""
    N = Sa.shape[0]
    A = np.zeros((2 * N, 2 * N), complex)
    A[:N, :N] = Ka - np.diag(Da)
    A[:N, N:] = -Sa
    A[N:, :N] = Kb - np.diag(Db)
    A[N:, N:] = Sb
    B = np.concatenate([np.zeros_like(b1), A[N:, :N] @ b1 + A[N:, N:] @ b2])
    return A, B


class Solution:
    """Full oracle run: every modal matrix and the densities for modes 0..M/2-1."""

    def __init__(self, P: Params, keep_matrices=False, modes=None):
        self.P = P
        self.sys = ModalSystem(P)
        G, Q = self.sys.G, self.sys.Q
        self.Da, self.Db = diagonal(G, Q)
        b1, b2 = rhs_modes(G)
        self.b1, self.b2 = b1, b2
        nh = P.M // 2
        modes = range(nh) if modes is None else modes
        N = P.N
        self.modes = list(modes)
        self.u1 = np.zeros((nh, N), complex)
        self.phi1 = np.zeros_like(self.u1)
        self.u2 = np.zeros_like(self.u1)
        self.phi2 = np.zeros_like(self.u1)
        self.A = {} if keep_matrices else None
        for n in self.modes:
            Sa, Ka = self.sys.matrices("a", n)
            Sb, Kb = self.sys.matrices("b", n)
            r = solve_ntd(Sa, Ka, self.Da, Sb, Kb, self.Db, b1[:, n], b2[:, n])
            self.u1[n], self.phi1[n], self.u2[n], self.phi2[n] = r
            if keep_matrices:
                self.A[n] = block_system(Sa, Ka, self.Da, Sb, Kb, self.Db, b1[:, n], b2[:, n])
