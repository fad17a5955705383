"""Solve options through the C ABI (pmlbie_solve_ex): mode chunking and mode
ranges (modes are independent, Sec. 3.3), incidence azimuth and several
right-hand sides (mode n of a wave with azimuth theta is e^{-i n theta} times
that of the azimuth-0 wave), checked against the unchunked solve and the FP64
oracle on the N = 128, M = 64 workload."""
import numpy as np
import pytest

from test_gpu_parity import CFG1, check_densities

pytestmark = pytest.mark.gpu


def _rel(a, b):
    import torch
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


@pytest.fixture(scope="module")
def prob():
    from paper_2412_11162_gb300 import Problem
    return Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chunked_and_mode_range_equal_full_solve(prob, precision):
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    prec = PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED
    pol = [np.pi / 6, 0.9]
    full, rf = prob.solve(pol, precision=prec)
    assert rf.chunks == 1
    chunked, rc = prob.solve(pol, precision=prec, max_chunk_modes=5)
    assert rc.chunks == 7 and rc.chunk_modes == 5
    part, rp = prob.solve(pol, precision=prec, modes=(7, 19), max_chunk_modes=4)
    assert rp.chunks == 3 and rp.n_modes == 12
    # Repeated solves differ by rounding: the Alpert corrections are added with
    # atomics (order not fixed), and in the mixed path each chunk's refinement
    # stops on its own (1e-13 relative residual or 1e-16 backward error).  The
    # phi unknowns carry kappa ~1e7 (mode 0, near-null direction at the axis),
    # so they agree to ~kappa x rounding; u to near rounding.
    # (mixed: each refinement stops at its own point below 1e-13 relative
    # residual, and the u components amplify that by up to ~1e2)
    tol = {"u1": 1e-12, "u2": 1e-12, "phi1": 1e-8, "phi2": 1e-8} if precision == "fp64" else \
        {"u1": 1e-10, "u2": 1e-10, "phi1": 1e-7, "phi2": 1e-7}
    for k in ("u1", "phi1", "u2", "phi2"):
        assert _rel(chunked[k], full[k]) <= tol[k], (k, _rel(chunked[k], full[k]))
        assert _rel(part[k], full[k][7:19]) <= tol[k], (k, _rel(part[k], full[k][7:19]))


def test_workspace_limit_forces_chunks(prob):
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, pmlbie_workspace_bytes
    whole = pmlbie_workspace_bytes(prob.handle, PMLBIE_FP64, 1)
    out, rep = prob.solve([np.pi / 6], precision=PMLBIE_FP64, workspace_limit=whole // 3)
    assert rep.chunks >= 3
    ref, _ = prob.solve([np.pi / 6], precision=PMLBIE_FP64)
    assert _rel(out["u1"], ref["u1"]) <= 1e-12


def test_azimuth_rotation_identity(prob):
    """Mode n for azimuth theta equals e^{-i n theta} times mode n at azimuth 0."""
    import torch
    from paper_2412_11162_gb300.binding import PMLBIE_FP64
    pol = [0.4, 0.4, 1.1]
    az = [0.0, 0.7, -2.3]
    out, _ = prob.solve(pol, precision=PMLBIE_FP64, azimuth=az)
    n = torch.arange(prob.n_modes, dtype=torch.float64, device="cuda")
    for r in (1, 2):
        rot = torch.exp(-1j * n * az[r]).to(torch.complex128)[:, None]
        base, _ = prob.solve([pol[r]], precision=PMLBIE_FP64)
        for k in ("u1", "phi1", "u2", "phi2"):
            e = _rel(out[k][:, :, r], rot * base[k][:, :, 0])
            # separate solves: rounding-level matrix differences (atomic Alpert
            # corrections) times kappa for phi
            assert e <= (1e-12 if k[0] == "u" else 1e-8), (r, k, e)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_azimuth_against_oracle(prob, precision):
    """Oblique incidence (polar 0.4, azimuth 0.7) inside a 3-wave solve,
    against the oracle, whose reference field carries the azimuth directly."""
    from oracle.assemble import Solution
    from oracle.problem import Params
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    prec = PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED
    sol = _oracle_oblique()
    out, _ = prob.solve([np.pi / 6, 0.4, 1.0], precision=prec, azimuth=[0.0, 0.7, 2.0])
    one = {k: v[:, :, 1:2].contiguous() for k, v in out.items()}
    tol = 1e-10 if precision == "fp64" else 1e-6
    check_densities(one, sol, tol, 1e-11, precision + "-oblique")


_SOL = {}


def _oracle_oblique():
    from oracle.assemble import Solution
    from oracle.problem import Params
    if "s" not in _SOL:
        _SOL["s"] = Solution(Params(**CFG1, polar=0.4, azimuth=0.7), keep_matrices=True)
    return _SOL["s"]


def test_bad_options_rejected(prob):
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PmlbieError
    with pytest.raises(PmlbieError):
        prob.solve([0.3], precision=PMLBIE_FP64, modes=(5, 3))
    with pytest.raises(PmlbieError):
        prob.solve([0.3], precision=PMLBIE_FP64, modes=(0, prob.n_modes + 1))
    with pytest.raises(PmlbieError):
        prob.solve([0.3], precision=PMLBIE_FP64, azimuth=[float("nan")])


def test_batch_of_uneven_instances_equals_single_solves():
    """Three instances of different sizes, wavenumbers and bump heights with 4
    oblique plane waves, solved by one batch call on two worker streams, equal
    the instance-by-instance solves."""
    from paper_2412_11162_gb300 import Problem, solve_batch
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    specs = [(2 * np.pi, 3 * np.pi, 96, 48, 0.15), (3 * np.pi, 4.5 * np.pi, 128, 64, 0.3),
             (2.5 * np.pi, 3.75 * np.pi, 64, 32, 0.4)]
    probs = [Problem(k1, k2, N, M, bump_h=h) for k1, k2, N, M, h in specs]
    pol = [0.2, 0.6, 1.0, 1.3]
    az = [0.0, 1.0, 2.5, -0.7]
    outs, reps = solve_batch(probs, pol, az, precision=PMLBIE_MIXED, n_streams=2, release_workspace=True)
    for P, o, r in zip(probs, outs, reps):
        ref, _ = P.solve(pol, precision=PMLBIE_MIXED, azimuth=az)
        assert r.n_modes == P.n_modes
        for k in ("u1", "phi1", "u2", "phi2"):
            e = _rel(o[k], ref[k])
            # two mixed solves agree to their refinement tolerance x conditioning
            # (well inside the 1e-6 bar of the mixed path; a mix-up of
            # instances or waves would show as O(1))
            assert e <= (1e-8 if k[0] == "u" else 1e-6), (P.N, k, e)


def test_lu_graph_replay(prob):
    """The batched LU of a workspace is captured once as a CUDA graph and
    replayed by later solves (FP64 and mixed), with the same results."""
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    for prec, tol in ((PMLBIE_MIXED, 1e-10), (PMLBIE_FP64, 1e-12)):
        first, _ = prob.solve([np.pi / 6], precision=prec)
        again, rep = prob.solve([np.pi / 6], precision=prec)
        assert rep.lu_graph_replays >= 1
        assert _rel(again["u1"], first["u1"]) <= tol


def test_bounded_wait_expiry_reports_timeout(prob):
    """Failure detection without a fault: a bounded mbarrier wait that nothing
    completes expires, the host reads ETIMEOUT, and the context keeps working."""
    import torch
    from paper_2412_11162_gb300 import binding as B
    assert B.pmlbie_selftest_wait(1000) == B.PMLBIE_ETIMEOUT
    assert "expired" in B.lib.pmlbie_last_error().decode()
    out, rep = prob.solve([np.pi / 6], precision=B.PMLBIE_MIXED)
    assert bool(torch.isfinite(torch.view_as_real(out["u1"])).all())


def test_finiteness_scan():
    import torch
    from paper_2412_11162_gb300 import binding as B
    t = torch.zeros(1000, dtype=torch.complex128, device="cuda")
    assert B.pmlbie_check_finite(t) == B.PMLBIE_OK
    t[517] = complex(float("nan"), 0.0)
    assert B.pmlbie_check_finite(t) == B.PMLBIE_ENAN
    t[517] = complex(0.0, float("inf"))
    assert B.pmlbie_check_finite(t) == B.PMLBIE_ENAN
    t[517] = 0
    assert B.pmlbie_check_finite(t[:10]) == B.PMLBIE_OK
