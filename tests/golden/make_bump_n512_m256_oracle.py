"""Writes bump_n512_m256_oracle.npz: the FP64 oracle's solution of the
benchmark workload (two-layer Gaussian bump, omega_1 = 4 pi, omega_2 = 6 pi,
N = 512, M = 256, PML a1 = 2.5, T = 1, S = 3, plane wave at polar angle
30 degrees) on a sample of modes, for the GPU parity test at that size and the
bench line's error against the oracle.  Calls only oracle/ (a full oracle run
at this size takes longer than a test should).

Stored per sampled mode n (Sec. 4.2, Eqs. (ntdpsi1), (ntdpsi2)): the densities
u1, phi1, u2, phi2 at the N nodes; the scattered-field modes at 32 fixed
points (Sec. 4.2, Eq. (fujs)): 16 at z = +1 (upper medium) and 16 at z = -1
(lower), rho in [0, 2]; and kappa_n, the 2-norm condition number of the
column-equilibrated block matrix of the mode.

Usage: python tests/golden/make_bump_n512_m256_oracle.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "bump_n512_m256_oracle.npz")
MODES = (0, 1, 63, 127)
RHO = np.tile(np.linspace(0.0, 2.0, 16), 2)
ZZ = np.repeat([1.0, -1.0], 16)
REG = np.repeat([0, 1], 16)


def main():
    from oracle.assemble import Solution
    from oracle.field import field_modes
    from oracle.problem import Params
    t0 = time.time()
    P = Params(k1=4 * np.pi, k2=6 * np.pi, N=512, M=256)
    sol = Solution(P, keep_matrices=True, modes=MODES)
    t1 = time.time()
    sel = list(MODES)
    fld = field_modes(P, RHO, ZZ, REG, sol.u1, sol.phi1, sol.u2, sol.phi2, G=sol.sys.G, Q=sol.sys.Q)
    kappa = []
    for n in sel:
        A, _ = sol.A[n]
        kappa.append(np.linalg.cond(A / np.linalg.norm(A, axis=0)[None, :]))
    np.savez_compressed(OUT, modes=np.array(sel), u1=sol.u1[sel], phi1=sol.phi1[sel], u2=sol.u2[sel],
                        phi2=sol.phi2[sel], field=fld[sel], kappa=np.array(kappa), rho=RHO, z=ZZ, region=REG,
                        k1=P.k1, k2=P.k2, N=P.N, M=P.M, polar=P.polar)
    print("wrote %s (oracle solve %.0f s, total %.0f s)" % (OUT, t1 - t0, time.time() - t0))


if __name__ == "__main__":
    main()
