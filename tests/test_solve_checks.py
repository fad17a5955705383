"""Argument checks of pmlbie_solve_ex on the host: every bad request returns
PMLBIE_EINVAL with its message before the library touches a device (so this
runs without a GPU): wave counts, polar angles, azimuths, precision, point
sources outside the physical region or too close to the interface for the
M-point azimuthal rule (the far-pair criterion d / sqrt(rho_s rho_m) >=
eta_s), mode ranges and chunk sizes."""
import numpy as np
import pytest


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# The requests carry null output pointers: they must never reach a device, so
# the module runs only where there is none (a regression in the checks would
# otherwise launch kernels on null buffers).
pytestmark = pytest.mark.skipif(_has_gpu(), reason="host-only checks; null output buffers")


@pytest.fixture(scope="module")
def prob():
    from paper_2412_11162_gb300 import Problem
    P = Problem(4 * np.pi, 6 * np.pi, 96, 32)
    yield P
    P.close()


def _solve(P, **kw):
    from paper_2412_11162_gb300 import binding as B
    args = dict(precision=B.PMLBIE_MIXED, polar=[0.3])
    args.update(kw)
    return B.pmlbie_solve_ex(P.handle, stream=0, **args)


@pytest.mark.parametrize("kw,frag", [
    (dict(polar=[]), "n_rhs must be in [1, 4096]"),
    (dict(polar=[np.pi / 2]), "polar angle must be in [0, pi/2)"),
    (dict(polar=[-0.1]), "polar angle must be in [0, pi/2)"),
    (dict(polar=[0.3], azimuth=[np.nan]), "azimuth must be finite"),
    (dict(precision=7), "bad precision"),
    (dict(polar=None, sources=[(3.0, 0.5)]), "source must have 0 <= rho < a1"),
    (dict(polar=None, sources=[(0.5, np.inf)]), "source must have 0 <= rho < a1"),
    (dict(mode_lo=5, mode_hi=3), "bad mode range"),
    (dict(mode_lo=0, mode_hi=17), "bad mode range"),
    (dict(max_chunk_modes=-1), "max_chunk_modes must be >= 0"),
])
def test_bad_requests(prob, kw, frag):
    from paper_2412_11162_gb300 import binding as B
    with pytest.raises(B.PmlbieError) as e:
        _solve(prob, **kw)
    assert e.value.code == B.PMLBIE_EINVAL and frag in str(e.value), str(e.value)


def test_source_next_to_the_interface(prob):
    """A source 1e-3 above a node of the bump is closer than the far-pair
    criterion allows and is rejected.  (Only rejected requests are made here:
    an accepted one would go on to the device with the null output pointers
    of this test.)"""
    from paper_2412_11162_gb300 import binding as B
    nd = prob.nodes()
    for l in (5, 40, 55):
        with pytest.raises(B.PmlbieError) as e:
            _solve(prob, polar=None, sources=[(nd["rho"][l], nd["z"][l] + 1e-3)])
        assert e.value.code == B.PMLBIE_EINVAL and "too close to the interface" in str(e.value)
