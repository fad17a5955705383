"""Sensitivity of the FP64 oracle's solution at the benchmark size (N = 512,
M = 256, omega = 4 pi / 6 pi) to rounding-level changes of its close-pair
modal Laplace kernels Z^_m, D^_m (Sec. 4.1 kernel splitting): each value is
multiplied by (1 + 2^-52 (U + i V)), U, V uniform in [-1, 1] (seeded), and
the solution of modes 0, 1, 63, 127 is compared with the stored one
(bump_n512_m256_oracle.npz).  Calls only oracle/; prints the relative
2-norm changes (on all nodes and on the physical nodes rho <= a1).

Measured (x86 host, seed 7): u1 2.5e-10 (physical nodes 6.8e-11), phi1
7.9e-9, u2 1.0e-10 (2.8e-11), phi2 2.6e-9.  The same perturbation of every
final modal-kernel value instead moves u1 by 8e-16 and phi1 by 9e-10: the
amplification comes from the split, whose two terms cancel on the PML
close pairs.

Usage: python tests/golden/oracle_sensitivity_n512_m256.py [seed]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(seed=7):
    import oracle.kernels as KR
    from oracle.assemble import Solution
    from oracle.problem import Params
    rng = np.random.default_rng(seed)
    exact = KR.laplace_modes

    def perturbed(pg, mmax, refine=0, chunk=512):
        Zm, Dm = exact(pg, mmax, refine, chunk)
        f = lambda X: X * (1 + 2.0 ** -52 * (rng.uniform(-1, 1, X.shape) + 1j * rng.uniform(-1, 1, X.shape)))
        return f(Zm), f(Dm)

    KR.laplace_modes = perturbed
    try:
        g = np.load(os.path.join(HERE, "bump_n512_m256_oracle.npz"))
        P = Params(k1=float(g["k1"]), k2=float(g["k2"]), N=int(g["N"]), M=int(g["M"]))
        t0 = time.time()
        modes = [int(n) for n in g["modes"]]
        sol = Solution(P, modes=modes)
    finally:
        KR.laplace_modes = exact
    phys = sol.sys.G.nodes["rho"] <= P.a1
    for k in ("u1", "phi1", "u2", "phi2"):
        a, b = getattr(sol, k)[modes], g[k]
        print("%-4s all %.2e  physical %.2e" % (k, np.linalg.norm(a - b) / np.linalg.norm(b),
                                                np.linalg.norm(a[:, phys] - b[:, phys]) / np.linalg.norm(b[:, phys])))
    print("oracle time %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 7)
