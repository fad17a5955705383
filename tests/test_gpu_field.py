"""Scattered field at observation points (pmlbie_field, Sec. 4.2 Eq. (fujs))
against the oracle's representation formula (oracle/field.py, pinned by the
point-source fields across the interface), on the N = 128, M = 64 workload at
32 fixed points: 16 at z = +1 (upper medium) and 16 at z = -1 (lower),
rho in [0, 2]."""
import numpy as np
import pytest

from test_gpu_parity import CFG1, oracle_solution

pytestmark = pytest.mark.gpu

RHO = np.tile(np.linspace(0.0, 2.0, 16), 2)
ZZ = np.repeat([1.0, -1.0], 16)
REG = np.repeat([0, 1], 16)


def _oracle_field(sol):
    from oracle.field import field_modes
    return field_modes(sol.P, RHO, ZZ, REG, sol.u1, sol.phi1, sol.u2, sol.phi2)   # (M/2, 32)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_field_from_oracle_densities():
    """The field kernels alone: oracle densities in, same quadrature -> 1e-12."""
    import torch
    from paper_2412_11162_gb300 import Problem
    sol = oracle_solution(**CFG1)
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    dens = {k: torch.tensor(getattr(sol, k)[:, :, None], dtype=torch.complex128, device="cuda")
            for k in ("u1", "phi1", "u2", "phi2")}
    got = P.field(RHO, ZZ, REG, dens)[:, :, 0].cpu().numpy()
    ref = _oracle_field(sol)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale, np.abs(got - ref).max() / scale
    # a mode range gives the same values
    sub = {k: v[5:17].contiguous() for k, v in dens.items()}
    part = P.field(RHO, ZZ, REG, sub, modes=(5, 17))[:, :, 0].cpu().numpy()
    assert np.abs(part - ref[5:17]).max() <= 1e-12 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_field_end_to_end(precision):
    """GPU solve, then GPU field, against the oracle's solve and field:
    relative 2-norm <= 1e-10 (FP64) / 1e-6 (mixed)."""
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    sol = oracle_solution(**CFG1)
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    out, _ = P.solve([np.pi / 6], precision=PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED)
    got = P.field(RHO, ZZ, REG, out)[:, :, 0].cpu().numpy()
    ref = _oracle_field(sol)
    e = _rel(got, ref)
    print(precision, "field rel err %.2e" % e)
    assert e <= (1e-10 if precision == "fp64" else 1e-6), e


def test_field_rejects_bad_points():
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PmlbieError
    P = Problem(CFG1["k1"], CFG1["k2"], 64, 32)
    d = {k: torch.zeros((16, 64, 1), dtype=torch.complex128, device="cuda") for k in ("u1", "phi1", "u2", "phi2")}
    with pytest.raises(PmlbieError):
        P.field([3.0], [1.0], [0], d)          # inside the PML
    with pytest.raises(PmlbieError):
        P.field([0.5], [1.0], [2], d)          # no such medium
