"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded/deterministic inputs.

Tolerances (stated by the workload definition): relative error <= 1e-10 for the
plain FP64 GPU path and <= 1e-6 for the mixed path (FP32 LU + FP64 refinement),
measured as relative 2-norms over all (mode, node, rhs) entries per output.
Modal kernels are compared per (kernel, mode) in relative Frobenius norm.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


_ORACLE = {}


def oracle_solution(**kw):
    from oracle.assemble import Solution
    from oracle.problem import Params
    key = tuple(sorted(kw.items()))
    if key not in _ORACLE:
        _ORACLE[key] = Solution(Params(**kw))
    return _ORACLE[key]


CFG1 = dict(k1=TWO_PI, k2=3 * np.pi, N=128, M=64)


def test_modal_kernels_config1(torch):
    from paper_2412_11162_gb300 import Problem
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    K = P.modal_kernels().cpu().numpy()
    sol = oracle_solution(**CFG1)
    worst = 0.0
    for n in range(CFG1["M"] // 2):
        for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
            ref = sol.sys.grid_kernel(reg, which, n)
            worst = max(worst, _rel(K[n, kern], ref))
    assert worst <= 1e-10, worst


def test_solve_fp64_config1(torch):
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    out, rep = P.solve([np.pi / 6], precision=PMLBIE_FP64)
    sol = oracle_solution(**CFG1)
    for name, ref in (("u1", sol.u1), ("phi1", sol.phi1), ("u2", sol.u2), ("phi2", sol.phi2)):
        got = out[name].cpu().numpy()[:, :, 0]
        assert _rel(got, ref) <= 1e-10, (name, _rel(got, ref))


def test_solve_mixed_config1(torch):
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    out, rep = P.solve([np.pi / 6], precision=PMLBIE_MIXED, allow_noconverge=True)
    sol = oracle_solution(**CFG1)
    for name, ref in (("u1", sol.u1), ("phi1", sol.phi1), ("u2", sol.u2), ("phi2", sol.phi2)):
        got = out[name].cpu().numpy()[:, :, 0]
        assert _rel(got, ref) <= 1e-6, (name, _rel(got, ref), rep.refine_iters, rep.residual)


def test_flat_interface_gives_zero_field(torch):
    from paper_2412_11162_gb300 import Problem
    P = Problem(TWO_PI, 3 * np.pi, 96, 32, bump_h=0.0)
    out, rep = P.solve([np.pi / 6, np.pi / 4])
    for v in out.values():
        assert torch.abs(v).max().item() < 1e-12


def test_equal_media_gives_zero_field(torch):
    from paper_2412_11162_gb300 import Problem
    P = Problem(TWO_PI, TWO_PI, 96, 32)
    out, rep = P.solve([np.pi / 6])
    for v in out.values():
        assert torch.abs(v).max().item() < 1e-12


def test_polyline_radix3_modal_kernels(torch):
    """Corner geometry of Sec. 4.3 (polyline) with M = 48 (radix-3 FFT stages)."""
    from oracle.assemble import ModalSystem
    from oracle.problem import Params
    from paper_2412_11162_gb300 import Problem
    V = [(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (4.0, 0.0)]
    kw = dict(a1=2.0, T=2.0, S=2.0, curve="polyline", vertices=V)
    P = Problem(TWO_PI, 2.4 * np.pi, 120, 48, **kw)
    K = P.modal_kernels(0, 6).cpu().numpy()
    sysm = ModalSystem(Params(k1=TWO_PI, k2=2.4 * np.pi, N=120, M=48, **kw))
    for n in range(6):
        for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
            ref = sysm.grid_kernel(reg, which, n)
            assert _rel(K[n, kern], ref) <= 1e-10, (n, kern, _rel(K[n, kern], ref))


def test_host_output_path_matches_device_path(torch):
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    P = Problem(TWO_PI, 3 * np.pi, 64, 32)
    out, _ = P.solve([np.pi / 6, 1.0])
    shp = (16, 64, 2)
    h = [np.zeros(shp, np.complex128) for _ in range(4)]
    B.pmlbie_solve_host(P.handle, B.PMLBIE_FP64, [np.pi / 6, 1.0], *h)
    for got, key in zip(h, ("u1", "phi1", "u2", "phi2")):
        assert np.array_equal(got, out[key].cpu().numpy())
