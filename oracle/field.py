"""Oracle (test infrastructure only): scattered field at observation points off
the interface, Sec. 4.2 Eq. (fujs) -- the representation formula evaluated
with the modal kernels and the solved densities.

Green's representation with the outward normal of each region, in the kernel
normalisation of the boundary equations (S and K carry the factor 2 of the
weights W_u = 2 rho |r'|, W_phi = 2 rho):

  upper medium (region a, omega_1, outward normal nu):
    u^{s,1}_n(x) =  1/2 sum_m h [W_phi(m) S^a_n(x, r_m) phi1_m - W_u(m) K^a_n(x, r_m) u1_m]
  lower medium (region b, omega_2, outward normal -nu; phi keeps the curve's nu):
    u^{s,2}_n(x) = -1/2 sum_m h [W_phi(m) S^b_n(x, r_m) phi2_m + W_u(m) K^b_n(x, r_m) u2_m]

K^b is the double-layer kernel for -nu.  At a smooth boundary point these
reduce to the block rows (K - D) u -/+ S phi = 0 with D = -1.  Points lie in
the physical region (rho < a1) and many node spacings off the curve, so the
trapezoid rule on the graded grid needs no corrections and the M-point rule
in psi is resolved as for far pairs.  Mode sums are left to the caller.
"""
import numpy as np

from . import kernels as KR
from .assemble import Quadrature, _region_nodes
from .problem import Geometry, Params


def point_dict(rho, z):
    """Observation points as target records (physical: rho~ = rho, no breakpoint)."""
    rho = np.asarray(rho, float)
    z = np.asarray(z, float)
    return dict(rho=rho, z=z, z_t=z + 0j, rho_t=rho + 0j, bk=np.full(rho.shape, -2), ox=np.zeros_like(rho),
                oz=np.zeros_like(rho))


def field_kernels(P: Params, G: Geometry, rho, z, region):
    """Modal kernels S^_n(x_p, r_m), K^_n(x_p, r_m), n = 0..M/2-1, of the medium
    of each point (region 0: upper, 1: lower) -> arrays (npts, N, M/2)."""
    npts, N = len(rho), P.N
    tg = point_dict(np.repeat(rho, N), np.repeat(z, N))
    S = np.zeros((npts, N, P.M // 2), complex)
    K = np.zeros_like(S)
    for reg, omega, sign in ((0, P.k1, 1.0), (1, P.k2, -1.0)):
        sel = np.nonzero(np.asarray(region) == reg)[0]
        if len(sel) == 0:
            continue
        nodes = _region_nodes(G.nodes, sign)
        src = {k: np.tile(nodes[k], len(sel)) for k in ("rho", "z", "z_t", "rho_t", "nuc_r", "nuc_z", "bk", "ox", "oz")}
        rows = (sel[:, None] * N + np.arange(N)[None, :]).ravel()
        tgt = {k: v[rows] for k, v in tg.items()}
        pg = KR.pair_geometry(tgt, src, P)
        s, k = KR.far_modes(pg, omega, P.M)
        S[sel] = s.reshape(len(sel), N, -1)
        K[sel] = k.reshape(len(sel), N, -1)
    return S, K


def field_modes(P: Params, rho, z, region, u1, phi1, u2, phi2, G: Geometry = None, Q: Quadrature = None):
    """u^s_n(x_p) for points (rho, z) with region 0 (upper) / 1 (lower), from
    densities (M/2, N) of one plane wave.  Returns (M/2, npts)."""
    G = G or Geometry(P)
    Q = Q or Quadrature(G)
    S, K = field_kernels(P, G, rho, z, region)
    h = G.h
    wu, wp = h * Q.W_u, h * Q.W_phi
    out = np.zeros((P.M // 2, len(rho)), complex)
    for p in range(len(rho)):
        if region[p] == 0:
            out[:, p] = 0.5 * (np.einsum("mn,m,nm->n", S[p], wp, phi1) - np.einsum("mn,m,nm->n", K[p], wu, u1))
        else:
            out[:, p] = -0.5 * (np.einsum("mn,m,nm->n", S[p], wp, phi2) + np.einsum("mn,m,nm->n", K[p], wu, u2))
    return out
