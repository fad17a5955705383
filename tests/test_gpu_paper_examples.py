"""The worked examples of Sec. 5 on the GPU, with the section's parameters:
omega_1 = 2 pi, omega_2 = 2.4 pi, a1 = 2, T = S = 2, p = 6, Alpert order 10,
plane-wave incidence from polar angle pi/3 and spherical incidence from the
source (0.3, 0, 0.5).  Example 1: rectangular dent of depth and radius 1;
Example 2: the wavy curve; Example 3: the seven-vertex polygon.

* modal kernels of all three against the oracle;
* full solves of all three (FP64 and mixed, both incidences) against the
  oracle's block systems;
* convergence in N of the scattered field at fixed points against N = 1600,
  the paper's reference size (the paper reports the errors only as a figure:
  the check is that they fall).

Example 2's curve meets the axis at an angle (a conical point); the segment
that starts there is graded with exponent 2 instead of p, which keeps its
first nodes at rho ~ h^2 where the double-layer kernel of the targets next to
the tip is still resolved, at the price of a lower order there."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

K1, K2 = 2 * np.pi, 2.4 * np.pi
COMMON = dict(a1=2.0, T=2.0, S=2.0)
EX = {
    "ex1": dict(curve="polyline", vertices=[(0.0, -1.0), (1.0, -1.0), (1.0, 0.0)]),
    "ex2": dict(curve="wavy", wavy_R=1.0, wavy_eps=0.1, wavy_m=3),
    "ex3": dict(curve="polyline", vertices=[(0.0, -0.5), (0.5, -0.5), (0.5, -0.7), (0.25, -0.7), (0.25, -1.0),
                                            (1.0, -1.0), (1.0, 0.0)]),
}
# sizes of the parity cases: Example 3's seven segments need >= 24 grid steps each
NP = {"ex1": 160, "ex2": 120, "ex3": 240}
POLAR = np.pi / 3
SOURCE = (0.3, 0.5)
_SOL = {}


def _oracle(ex, N, M):
    from oracle.assemble import Solution
    from oracle.problem import Params
    key = (ex, N, M)
    if key not in _SOL:
        _SOL[key] = Solution(Params(k1=K1, k2=K2, N=N, M=M, polar=POLAR, **COMMON, **EX[ex]), keep_matrices=True)
    return _SOL[key]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("ex", ["ex1", "ex2", "ex3"])
def test_modal_kernels_paper_examples(ex):
    from oracle.assemble import ModalSystem
    from oracle.problem import Params
    from paper_2412_11162_gb300 import Problem
    P = Problem(K1, K2, NP[ex], 48, **COMMON, **EX[ex])
    K = P.modal_kernels(0, 6).cpu().numpy()
    sysm = ModalSystem(Params(k1=K1, k2=K2, N=NP[ex], M=48, **COMMON, **EX[ex]))
    for n in range(6):
        for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
            ref = sysm.grid_kernel(reg, which, n)
            assert _rel(K[n, kern], ref) <= 1e-10, (ex, n, kern, _rel(K[n, kern], ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ex", ["ex1", "ex2", "ex3"])
def test_solve_paper_examples(ex, precision):
    """Plane wave (pi/3) and point source (0.3, 0.5) in one call each, M = 64,
    against the oracle: the plane wave with the plane-wave parity checks, the
    point source with the point-source ones."""
    from test_gpu_parity import check_densities
    from test_gpu_point_source import check_point
    import types
    from oracle.point_source import point_source_densities, point_source_systems
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    prec = PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED
    tol = 1e-10 if precision == "fp64" else 1e-6
    sol = _oracle(ex, NP[ex], 64)
    P = Problem(K1, K2, NP[ex], 64, **COMMON, **EX[ex])
    out, _ = P.solve([POLAR], precision=prec)
    check_densities(out, sol, tol, 1e-11, "%s plane %s" % (ex, precision))
    out, _ = P.solve(sources=[SOURCE], precision=prec)
    systems, _ = point_source_systems(sol, *SOURCE)
    u1, phi1, u2, phi2 = point_source_densities(sol, *SOURCE)
    ref = types.SimpleNamespace(P=sol.P, A=systems, u1=u1, phi1=phi1, u2=u2, phi2=phi2)
    # The residual of the GPU solution in the oracle's systems sits on the PML
    # rows (rho 2.2 .. 2.7, ~1e-9 in modes 0..3 for Examples 1 and 2 alike;
    # the right-hand sides agree to 3e-16): the PML close pairs' split cancels
    # and the two sides' kernels there agree to ~1e-10.  A point source puts
    # most of its low-mode densities into the PML (65% of mode 1's u1 in
    # Example 2), and Example 2's low modes are well conditioned (kappa_1 =
    # 1.7e3), so that difference shows in its forward errors (phi1 mode 1:
    # 3.3e-8 = 1.9e-11 kappa_1); Example 1 hides it under larger norms.  So:
    # the plane wave's backward bound, and a per-mode forward bound of
    # 1e-10 kappa_n for Example 2.
    check_point(out, 0, ref, tol, "%s point %s" % (ex, precision), sol=sol, backward_tol=1e-11,
                kappa_coef=1e-10 if ex == "ex2" else 1e-12)


# measured errors for N = 200, 400, 800 against N = 1600 (plane wave, point
# source) and the bound asserted on the N = 800 one
CONV = {"ex3": (((1.2e-4, 4.5e-6, 2.4e-6), (4.9e-4, 2.5e-5, 1.3e-5)), 1e-3),
        "ex2": (((1.8e-5, 9.9e-6, 8.5e-7), (1.3e-4, 5.0e-5, 6.3e-6)), 1e-4)}


@pytest.mark.parametrize("ex", ["ex2", "ex3"])
def test_convergence_in_n(ex):
    """Mixed path: scattered-field modes at 16 fixed points (rho in [0, 1.8]
    at z = 0.8 above and z = -1.5 below the interface) for N = 200, 400, 800
    against N = 1600, both incidences: the error falls with N (measured
    values in CONV)."""
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    rho = np.tile(np.linspace(0.0, 1.8, 8), 2)
    zz = np.repeat([0.8, -1.5], 8)
    reg = np.repeat([0, 1], 8)
    fields = {}
    for N in (200, 400, 800, 1600):
        P = Problem(K1, K2, N, 64, **COMMON, **EX[ex])
        f = []
        for kw in (dict(polar=[POLAR]), dict(sources=[SOURCE])):
            out, _ = P.solve(precision=PMLBIE_MIXED, **kw)
            f.append(P.field(rho, zz, reg, out)[:, :, 0].cpu().numpy())
        fields[N] = f
        P.close()
    for inc in (0, 1):
        errs = [_rel(fields[N][inc], fields[1600][inc]) for N in (200, 400, 800)]
        print(ex, ("plane", "point")[inc], ["%.2e" % e for e in errs])
        assert errs[1] < errs[0] and errs[2] < errs[1] and errs[2] < CONV[ex][1], errs
