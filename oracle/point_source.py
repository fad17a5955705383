"""Oracle (test infrastructure only): right-hand sides of spherical-wave
incidence, Sec. 2 (the incident field u_inc = G_1(., x_s) of a point source
x_s = (rho_s, 0, z_s) in the upper medium), and the densities they give.

The reference field is u^{tot,0} = u_inc in Omega_1 and 0 in Omega_2, so the
jumps are b^1 = -G~_1(r~_m, x_s) and b^2 = -|r'| d_nu_c G~_1 at every node,
the PML part of the curve included (stretched coordinates of the nodes).
Their modes over the node azimuth are the modal kernels of the pairs (target
x_s, source point r_m with the curve's conormal): S^a_n(x_s, r_m) and
K^a_n(x_s, r_m), by the M-point DFT in psi (the source lies off the curve, so
the M-point rule is resolved as for far pairs).  The solution then holds the
scattered field above (u^{s,1}) and the total field below (u^{s,2}).  A source
at azimuth phi_s multiplies mode n of the data, hence of the solution, by
e^{-i n phi_s}.
"""
import numpy as np

from . import kernels as KR
from .field import point_dict
from .problem import Geometry, Params


def point_source_rhs(P: Params, G: Geometry, rho_s, z_s):
    """(b1, b2), each (N, M/2), for a source at (rho_s, 0, z_s) in the upper medium."""
    N = P.N
    tgt = point_dict(np.full(N, float(rho_s)), np.full(N, float(z_s)))
    src = {k: G.nodes[k] for k in ("rho", "z", "z_t", "rho_t", "nuc_r", "nuc_z", "bk", "ox", "oz")}
    pg = KR.pair_geometry(tgt, src, P)
    S, K = KR.far_modes(pg, P.k1, P.M)
    return -S, -K * G.nodes["speed"][:, None]


def point_source_systems(sol, rho_s, z_s, phi_s=0.0):
    """{n: (A_n, B_n)}: the block systems of a Solution built with keep_matrices
    (Sec. 4.2) with the jumps of a source at (rho_s, phi_s, z_s) in B_n, and
    those jumps (b1, b2), each (N, M/2)."""
    P, G = sol.P, sol.sys.G
    b1, b2 = point_source_rhs(P, G, rho_s, z_s)
    rot = np.exp(-1j * np.arange(P.M // 2) * phi_s)[None, :]
    b1, b2 = b1 * rot, b2 * rot
    N = P.N
    out = {}
    for n in sol.modes:
        A = sol.A[n][0]
        out[n] = (A, np.concatenate([np.zeros(N, complex), A[N:, :N] @ b1[:, n] + A[N:, N:] @ b2[:, n]]))
    return out, (b1, b2)


def point_source_densities(sol, rho_s, z_s, phi_s=0.0):
    """Densities (u1, phi1, u2, phi2), each (M/2, N), of a source at
    (rho_s, phi_s, z_s) (Sec. 4.2 block systems with the point-source jumps)."""
    systems, (b1, b2) = point_source_systems(sol, rho_s, z_s, phi_s)
    nh, N = sol.P.M // 2, sol.P.N
    out = [np.zeros((nh, N), complex) for _ in range(4)]
    for n, (A, B) in systems.items():
        x = np.linalg.solve(A, B)
        out[0][n] = x[:N]
        out[1][n] = x[N:]
        out[2][n] = x[:N] - b1[:, n]
        out[3][n] = x[N:] - b2[:, n]
    return tuple(out)
