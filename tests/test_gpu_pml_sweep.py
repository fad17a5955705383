"""PML-thickness sweep (Sec. 3.1, Eq. (sgm1)): truncation error of the GPU
solve against a thick-PML reference falls exponentially with the PML
thickness T, for the plain FP64 and the mixed path.

Geometry: the dent of Sec. 4.3 (vertices (0,-1), (1,-1), (1,0), (2,0), PML
from a1 = 2) with the same number of grid steps per unit length on every
segment, so that every T shares the physical nodes exactly and the
difference of the solutions there is the truncation error alone.  Modes
0-7 of u1 on the physical nodes are compared with T = 3."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

V = [(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (2.0, 0.0)]


def _sweep(k1, S, steps_per_unit, M, precision, Ts=(0.5, 1.0, 1.5, 2.0, 3.0)):
    from paper_2412_11162_gb300 import Problem
    runs = {}
    for T in Ts:
        Nt = int(round(steps_per_unit * (3 + T)))
        P = Problem(k1, 1.5 * k1, Nt - 4, M, a1=2.0, T=T, S=S, curve="polyline", vertices=V)
        out, rep = P.solve([np.pi / 6], precision=precision, modes=(0, 8))
        nd = P.nodes()
        phys = nd["rho"] < 2.0
        runs[T] = (nd["rho"][phys], out["u1"][:, phys, 0].cpu().numpy())
        P.close()
    r_ref, u_ref = runs[Ts[-1]]
    errs = []
    for T in Ts[:-1]:
        r, u = runs[T]
        assert np.abs(r - r_ref).max() < 1e-12            # the same physical nodes
        errs.append(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
    return errs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_truncation_error_decays_k4pi(precision):
    """k1 = 4 pi, S = 1, 64 steps per unit, M = 256 (measured 3.3e-5, 1.7e-7,
    1.2e-8, 1.2e-8: exponential down to the quadrature floor).  At the floor
    the last two agree to rounding of the close-pair split, so the last one
    only has to stay within 10 % of the one before."""
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    errs = _sweep(4 * np.pi, 1.0, 64, 256, PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED)
    print(precision, ["%.2e" % e for e in errs])
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 50 and errs[2] < errs[1] / 4 and errs[3] <= 1.1 * errs[2], errs


def test_truncation_error_decays_k12pi():
    """k1 = 12 pi (the high-frequency sweep's lowest wavenumber), weak PML
    S = 0.1 so that the decay shows above the quadrature floor of 192 steps
    per unit and M = 512 (~4e-6), mixed path (measured 2.8e-4, 1.3e-5,
    3.4e-6, 4.0e-6)."""
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    errs = _sweep(12 * np.pi, 0.1, 192, 512, PMLBIE_MIXED)
    print("k12pi", ["%.2e" % e for e in errs])
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 10 and max(errs[2:]) < 1e-5, errs
