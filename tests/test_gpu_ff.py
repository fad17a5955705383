"""Float-float (FP32-pair) arithmetic of the mixed path.

* Its elementary functions (pmlbie_selftest_elementary selectors 20-22) against
  the host's FP64 values: exp as mantissa x 2^E, sin / cos, 1/sqrt of the
  float pair nearest to each double.  A float pair carries 48 significant
  bits, so the input itself is rounded by up to 2^-48 relative, which moves
  e^x and sin x by |x| 2^-48; the bounds are 2^-45 + |x| 2^-46.
* The modal kernels of the mixed path (pmlbie_modal_kernels_ex with
  PMLBIE_MIXED: far-pair sampling, transforms and scatter, and the close-pair
  split samples, transforms and convolution, in float-float; the exact modal
  Laplace kernels in FP64) against the FP64 oracle (Sec. 4.1): all pairs at
  N = 128, M = 64, sampled pairs at the benchmark size N = 512, M = 256.
"""
import numpy as np
import pytest

from test_gpu_parity import CFG1, oracle_solution

pytestmark = pytest.mark.gpu


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


def test_ff_exp():
    x = np.concatenate([_grid(-700.0, 80.0, 1 << 19, 11), _grid(-2.0, 0.0, 1 << 17, 12)])
    got = _run(20, x)
    rel = np.abs(got - np.exp(x)) / np.exp(x)
    bound = 2.0 ** -45 + np.abs(x) * 2.0 ** -46
    print("ff exp: max rel err %.2e, max err / bound %.2f" % (rel.max(), (rel / bound).max()))
    assert np.all(rel <= bound)


def test_ff_sincos():
    x = np.concatenate([_grid(-780.0, 780.0, 1 << 19, 13), _grid(-4.0, 4.0, 1 << 17, 14)])
    got = _run(21, x)
    bound = 2.0 ** -45 + np.abs(x) * 2.0 ** -46
    for k, ref in ((0, np.sin(x)), (1, np.cos(x))):
        err = np.abs(got[k::2] - ref)
        print("ff %s: max abs err %.2e, max err / bound %.2f" % ("sin" if k == 0 else "cos", err.max(),
                                                               (err / bound).max()))
        assert np.all(err <= bound)


def test_ff_rsqrt():
    x = np.exp(_grid(np.log(1e-30), np.log(1e30), 1 << 19, 15))
    got = _run(22, x)
    ref = 1.0 / np.sqrt(x)
    rel = np.abs(got - ref) / ref
    print("ff 1/sqrt: max rel err %.2e" % rel.max())
    # one Newton step from a float estimate with a float-pair residual: the
    # step's own error (3/2) e0^2 ~ 2^-46 plus the residual's rounding
    assert rel.max() <= 2.0 ** -44


def test_ff_kernels_vs_oracle_config1():
    """Mixed-path modal kernels (far pairs and the close-pair split in
    float-float, exact Laplace modes in FP64) against the oracle, N = 128,
    M = 64, all modes: far and physical close pairs within 6.4e-11 of the
    block's largest entry, PML close pairs (FP64 in both paths) within 1e-12
    of the split's term scale, every block within 1e-9: the bars of
    test_gpu_parity.test_modal_kernels_config1 with 64 times the FP64 factor
    where float pairs compute (48 significant bits against 53 + 1)."""
    from test_gpu_parity import _split_term_scale
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    K = P.modal_kernels(precision=PMLBIE_MIXED).cpu().numpy()
    S = oracle_solution(**CFG1).sys
    li, mi = S.grid_pairs
    near = S.near[: S.ngrid]
    rt = S.G.nodes["rho_t"].imag
    pml = (rt[li] > 0) | (rt[mi] > 0)
    worst = {"tight": 0.0, "pml_split": 0.0}
    for n in range(CFG1["M"] // 2):
        for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
            ref = S.grid_kernel(reg, which, n)
            got = K[n, kern]
            d = np.abs(got - ref)[li, mi]
            mx = np.abs(ref).max()
            tight = ~(near & pml)
            worst["tight"] = max(worst["tight"], d[tight].max() / mx)
            assert d[tight].max() <= 6.4e-11 * mx, (n, kern, d[tight].max() / mx)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-9
            if which == "S":
                sc = _split_term_scale(S, reg, n)
                loose = near & pml
                ratio = (d[loose] / (sc[loose] + 1e-300)).max() if loose.any() else 0.0
                worst["pml_split"] = max(worst["pml_split"], ratio)
                assert ratio <= 1e-12, (n, kern, ratio)
    print("mixed-path kernels vs oracle, N=128 M=64:", {k: "%.2e" % v for k, v in worst.items()})


def test_ff_kernels_sampled_pairs_bench_size():
    """Mixed-path modal kernels at the benchmark size (N = 512, M = 256) on
    sampled pairs against the oracle pair by pair: |diff| <= 1e-11 x the
    pair's rounding scale (the phase q = omega |dr| reaches ~130 here, and a
    float pair rounds it by |q| 2^-48)."""
    from test_gpu_fullsize import CFG2, check_sampled_kernels
    from paper_2412_11162_gb300.binding import PMLBIE_MIXED
    worst = check_sampled_kernels(CFG2, ((0, 6), (60, 64), (122, 128)), precision=PMLBIE_MIXED, factor=1e-11)
    print("mixed-path kernels vs oracle, N=512 M=256, sampled pairs: max |diff| / rounding scale %.2e" % worst)


def _close_pair_values(P, precision):
    import torch
    from paper_2412_11162_gb300 import binding as B
    g, c = P.near_count()
    nm = P.n_modes
    out = torch.empty((g + c) * 4 * nm, dtype=torch.complex128, device="cuda")
    B.pmlbie_close_pair_kernels(P.handle, precision, 0, nm, out)
    return out.view(g + c, 4, nm).cpu().numpy(), g, c


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_correction_pair_kernels_vs_oracle_config1(precision):
    """The split modal kernels of the Alpert correction pairs (the values the
    assembly spreads over the Lagrange stencils, Sec. 4.1 Eqs. (snab1),
    (snt1)) against the oracle's, pair by pair, N = 128, M = 64: every value
    finite; pairs without a PML point within 1e-12 (FP64) / 6.4e-11 (mixed:
    float pairs) of the kernel's largest correction value; PML pairs (Sec.
    4.3 substitution, FP64 in both paths) within 1e-12 of the split's term
    scale."""
    from test_gpu_parity import split_scale
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    P = Problem(CFG1["k1"], CFG1["k2"], CFG1["N"], CFG1["M"])
    vals, g, c = _close_pair_values(P, PMLBIE_FP64 if precision == "fp64" else PMLBIE_MIXED)
    assert np.isfinite(vals).all()
    fac = 1e-12 if precision == "fp64" else 6.4e-11
    S = oracle_solution(**CFG1).sys
    rows = S.ngrid + np.arange(c)                       # correction pairs in the oracle's stacked list
    near_rows = np.nonzero(S.near)[0]
    pg = {k: v[rows] for k, v in S.pg.items()}
    near = S.near[rows]
    pml = (pg["rho_t"].imag > 0) | (pg["rho_t_s"].imag > 0)
    lap_idx = np.searchsorted(near_rows, rows)
    worst = {"tight": 0.0, "pml": 0.0}
    for kern, (reg, which) in enumerate((("a", "S"), ("a", "K"), ("b", "S"), ("b", "K"))):
        Sk, Kk = S.kern[reg]
        ref_all = (Sk if which == "S" else Kk)[rows]
        for n in range(CFG1["M"] // 2):
            got, ref = vals[g:, kern, n], ref_all[:, n]
            d = np.abs(got - ref)
            mx = np.abs(ref).max()
            tight = ~(near & pml)
            worst["tight"] = max(worst["tight"], d[tight].max() / mx)
            assert d[tight].max() <= fac * mx, (kern, n, d[tight].max() / mx)
            if which == "S" and (near & pml).any():
                sel = near & pml
                sub = {k: v[sel] for k, v in pg.items()}
                sc = split_scale(sub, S.lap_near[0][lap_idx[sel]], P.params.k1 if reg == "a" else P.params.k2,
                                 CFG1["M"], 5, n)
                ratio = (d[sel] / sc).max()
                worst["pml"] = max(worst["pml"], ratio)
                assert ratio <= 1e-12, (kern, n, ratio)
    print(precision, "correction-pair kernels vs oracle:", {k: "%.2e" % v for k, v in worst.items()})
