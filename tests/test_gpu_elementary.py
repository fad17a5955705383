"""The library's own elementary functions (used by the Green's-function
sampling loops, Sec. 3.1 / 4.1: e^{iq} = e^{-Im q} (cos Re q + i sin Re q)
and the complex distance's reciprocal square roots) on dense grids over the
argument ranges the kernels use, through pmlbie_selftest_elementary.

Each is compared in units in the last place (ulp = spacing of the reference
value's magnitude) with the CUDA math library's routine at the same points and
with the host's (numpy / glibc, <= 1 ulp) values:
  * exp on [-708, 709] (the sampling loops clamp arguments to this range);
  * sin and cos on |x| <= 2^19 (beyond it the routine hands over to the CUDA
    library) plus a dense grid on [-10, 10];
  * 1/sqrt on [1e-300, 1e300].
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref, floor=1e-300):
    return np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), floor))


def _run(fn, x):
    import torch
    from paper_2412_11162_gb300 import binding as B
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(xd.numel() * (2 if fn % 10 == 1 else 1), dtype=torch.float64, device="cuda")
    B.pmlbie_selftest_elementary(fn, xd, out)
    return out.cpu().numpy()


def _grid(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([np.linspace(lo, hi, n), rng.uniform(lo, hi, n)])


def test_exp_ulp():
    x = np.concatenate([_grid(-708.0, 709.0, 1 << 20, 1), _grid(-40.0, 0.0, 1 << 18, 2)])
    ours, cuda = _run(0, x), _run(10, x)
    e_host = _ulp_err(ours, np.exp(x)).max()
    e_cuda = _ulp_err(ours, cuda).max()
    print("exp: max ulp vs host %.2f, vs CUDA %.2f" % (e_host, e_cuda))
    assert e_host <= 3.0 and e_cuda <= 4.0, (e_host, e_cuda)
    # below the clamp the routine returns e^{-708}
    below = _run(0, np.array([-709.0, -800.0, -1e4]))
    assert np.all(below == _run(0, np.array([-708.0]))[0])


def test_sincos_ulp():
    x = np.concatenate([_grid(-2.0 ** 19, 2.0 ** 19, 1 << 20, 3), _grid(-10.0, 10.0, 1 << 18, 4),
                        np.arange(-2000, 2001) * (np.pi / 2)])
    ours, cuda = _run(1, x), _run(11, x)
    worst = {}
    for k, (ref_host, part) in enumerate(((np.sin(x), "sin"), (np.cos(x), "cos"))):
        got, ref_cuda = ours[k::2], cuda[k::2]
        # ulp of the value, with the absolute floor 2^-53 (values that vanish
        # in exact arithmetic at multiples of pi/2 are rounding-level numbers)
        worst[part] = (_ulp_err(got, ref_host, 2.0 ** -53).max(), _ulp_err(got, ref_cuda, 2.0 ** -53).max())
    print("sin / cos: max ulp vs host, vs CUDA:", worst)
    for part, (eh, ec) in worst.items():
        assert eh <= 3.0 and ec <= 4.0, (part, eh, ec)


def test_rsqrt_ulp():
    x = np.exp(_grid(np.log(1e-300), np.log(1e300), 1 << 20, 5))
    ours, cuda = _run(2, x), _run(12, x)
    e_host = _ulp_err(ours, 1.0 / np.sqrt(x)).max()
    e_cuda = _ulp_err(ours, cuda).max()
    print("1/sqrt: max ulp vs host %.2f, vs CUDA %.2f" % (e_host, e_cuda))
    assert e_host <= 2.0 and e_cuda <= 3.0, (e_host, e_cuda)


def test_selftest_rejects_unknown_selector():
    import torch
    from paper_2412_11162_gb300 import binding as B
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PmlbieError):
        B.pmlbie_selftest_elementary(7, x, torch.zeros(4, dtype=torch.float64, device="cuda"))
