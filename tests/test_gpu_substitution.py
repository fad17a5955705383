"""The Sec. 4.3 substitution switch (pmlbie_params.subst_off, a diagnostic
mode): on close pairs with a point in the PML the library can use the exact
split (H1 = cos q, H3 = cos q + q sin q at complex q) instead of the cH1 / cH3
Taylor substitution.  The two differ by the substitution's own truncation:
its remainder Z (e^{iq} - cH1) has an |psi|^L kink that the M-point rule
resolves only to ~5e-6 here (M = 128, L = 5), while the exact split's
remainder is smooth but loses about e^{|Im q|} x eps to cancellation.  With
weak and moderate PMLs (S = 0.5, 2) the kernels therefore agree to ~5e-6
(far below the discretisation error) and the diagnostic mode matches the
oracle's exact split; with a strong PML (S = 12) the exact split's growth
destroys the kernels, which is what the substitution prevents (the oracle
pin of the section's NtD experiment shows the same: 2.4e-2 with, O(10)
without)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

V = [(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (4.0, 0.0)]
K1 = 2 * np.pi


def _kernels(S, subst):
    from paper_2412_11162_gb300 import Problem
    P = Problem(K1, K1, 120, 128, a1=2.0, T=2.0, S=S, curve="polyline", vertices=V, subst=subst)
    return P.modal_kernels(0, 4).cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_switch_agrees_for_weak_pmls_and_blows_up_for_a_strong_one():
    d = {S: _rel(_kernels(S, False), _kernels(S, True)) for S in (0.5, 2.0, 12.0)}
    print("exact split vs substitution:", {S: "%.1e" % v for S, v in d.items()})
    assert d[0.5] < 1e-4 and d[2.0] < 1e-4 and d[12.0] > 1.0, d


def test_exact_split_matches_the_oracle():
    from oracle.assemble import ModalSystem
    from oracle.problem import Params
    K = _kernels(0.5, False)
    sysm = ModalSystem(Params(k1=K1, k2=K1, N=120, M=128, a1=2.0, T=2.0, S=0.5, curve="polyline", vertices=V,
                              subst=False))
    for n in range(4):
        for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
            ref = sysm.grid_kernel(reg, which, n)
            assert _rel(K[n, kern], ref) <= 1e-10, (n, kern, _rel(K[n, kern], ref))
