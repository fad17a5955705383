"""Parity against the FP64 oracle at the benchmark workload: two-layer
Gaussian bump, omega_1 = 4 pi, omega_2 = 6 pi, N = 512, M = 256, one plane
wave at polar angle 30 degrees (the problem bench.py times).

A whole oracle run at this size takes several minutes of host time, so its
solution on the sampled modes 0, 1, 63, 127 is stored in
tests/golden/bump_n512_m256_oracle.npz, written by
tests/golden/make_bump_n512_m256_oracle.py, which calls only oracle/.

Checked per precision (plain FP64 GPU path: 1e-10; mixed path: 1e-6),
Sec. 4.2 Eqs. (ntdpsi1), (ntdpsi2) and Eq. (fujs):
  * u1, u2: relative 2-norm over the sampled modes on the physical nodes
    (rho <= a1) <= tol; per mode on all nodes <= max(tol, 1e-12 kappa_n);
  * phi1, phi2: per mode <= max(tol, 1e-12 kappa_n) (kappa_n: condition
    number of the column-equilibrated block matrix of mode n, stored with the
    oracle's solution); the measured values are printed;
  * the scattered field at the 32 fixed points: relative 2-norm over the
    sampled modes <= tol.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bump_n512_m256_oracle.npz")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ref():
    g = np.load(GOLDEN)
    return {k: g[k] for k in g.files}


@pytest.fixture(scope="module")
def problem(ref):
    from paper_2412_11162_gb300 import Problem
    return Problem(float(ref["k1"]), float(ref["k2"]), int(ref["N"]), int(ref["M"]))


def check_against_oracle(out, P, ref, tol, label):
    modes = list(ref["modes"])
    kap = ref["kappa"]
    rho = P.nodes()["rho"]
    phys = rho <= P.params.a1
    errs = {}
    for name in ("u1", "u2", "phi1", "phi2"):
        got = out[name].cpu().numpy()[modes, :, 0]
        want = ref[name]
        errs[name] = _rel(got, want)
        if name.startswith("u"):
            e = _rel(got[:, phys], want[:, phys])
            assert e <= tol, (label, name, "physical nodes", e)
        for i, n in enumerate(modes):
            e = np.linalg.norm(got[i] - want[i]) / np.linalg.norm(want)
            assert e <= max(tol, 1e-12 * kap[i]), (label, name, n, e, kap[i])
    fld = P.field(ref["rho"], ref["z"], ref["region"], out)[:, :, 0].cpu().numpy()[modes]
    errs["field"] = _rel(fld, ref["field"])
    assert errs["field"] <= tol, (label, "field", errs["field"])
    print(label, " ".join("%s %.2e" % kv for kv in errs.items()), "kappa", kap)
    return errs


def test_fp64_solve_matches_oracle_at_bench_size(problem, ref):
    from paper_2412_11162_gb300.binding import PMLBIE_FP64
    out, _ = problem.solve([float(ref["polar"])], precision=PMLBIE_FP64)
    check_against_oracle(out, problem, ref, 1e-10, "fp64")


def test_mixed_solve_matches_oracle_at_bench_size(problem, ref):
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    out, rep = problem.solve([float(ref["polar"])], precision=PMLBIE_MIXED)
    assert rep.backward_error <= 1e-13
    check_against_oracle(out, problem, ref, 1e-6, "mixed")
