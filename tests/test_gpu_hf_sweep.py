"""High-frequency sweep: omega_1 = 12 pi ... 20 pi in five steps, omega_2 =
1.5 omega_1, N = 1536, 2176, 2816, 3456, 4096 nodes, M = 512 angles, the two-layer bump of
the other workloads.  Per wavenumber:

* the mixed path's modal kernels (float-float far and close pairs, FP64
  Laplace modes and PML split samples) on sampled grid pairs against the FP64
  oracle pair by pair, lowest and highest modes: |diff| <= 1e-11 x the pair's
  rounding scale (the phases reach |q| ~ 650 here; a float pair rounds q by
  |q| 2^-48);
* mixed against FP64 solves.  The dominant modes 0 and 1 (up to N = 2176;
  at N = 4096 they are numerically singular in FP64, |A| |x| / |b| ~ 1e11, and
  the two solutions differ along near-null directions that carry no field):
  u1, u2 and the scattered field at 32 points within 1e-6 relative.  The
  highest mode (255): its difference within 1e-6 of the solution's scale,
  the mixed solution of modes 0 and 1 (densities and field) -- that mode's
  kernels are ~1e-10 of the largest sample of their transforms, and both
  precisions round relative to that sample (a float pair 2^-48, FP64 2^-53),
  so its own relative difference (printed) grows with the frequency.

The full mixed solves of the sweep's two ends (all modes, in mode chunks at
N = 4096) are timed by bench.py (workloads n1536_m512, n4096_m512)."""
import numpy as np
import pytest

from test_gpu_fullsize import check_sampled_kernels

pytestmark = pytest.mark.gpu

SWEEP = [(12, 1536), (14, 2176), (16, 2816), (18, 3456), (20, 4096)]


def _rel(a, b, scale):
    import torch
    return (torch.linalg.vector_norm(a - b) / scale).item()


@pytest.mark.parametrize("k_over_pi,N", SWEEP)
def test_hf_sweep(k_over_pi, N):
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    cfg = dict(k1=k_over_pi * np.pi, k2=1.5 * k_over_pi * np.pi, N=N, M=512)
    P = Problem(cfg["k1"], cfg["k2"], N, 512)
    worst = check_sampled_kernels(cfg, ((0, 2), (254, 256)), n_pairs=60, precision=PMLBIE_MIXED, factor=1e-11,
                                  P=P, light=True)
    fr = np.tile(np.linspace(0.0, 2.0, 16), 2)
    fz = np.repeat([1.0, -1.0], 16)
    fg = np.repeat([0, 1], 16)
    pol = [np.pi / 6]
    # dominant modes: the solution's scale, and their own comparison up to N = 2176
    lo32, r32 = P.solve(pol, precision=PMLBIE_MIXED, modes=(0, 2))
    assert r32.backward_error <= 1e-13
    flo = P.field(fr, fz, fg, lo32, modes=(0, 2))
    scale = {k: torch.linalg.vector_norm(lo32[k]) for k in ("u1", "u2")}
    fscale = torch.linalg.vector_norm(flo)
    errs = {}
    if N <= 2176:
        lo64, _ = P.solve(pol, precision=PMLBIE_FP64, modes=(0, 2))
        for k in ("u1", "u2"):
            errs[k + "_modes01"] = _rel(lo32[k], lo64[k], torch.linalg.vector_norm(lo64[k]))
        f64 = P.field(fr, fz, fg, lo64, modes=(0, 2))
        errs["field_modes01"] = _rel(flo, f64, torch.linalg.vector_norm(f64))
    # the highest mode against FP64 (one mode: a 2N = 8192 FP64 LU takes seconds)
    hi32, r32 = P.solve(pol, precision=PMLBIE_MIXED, modes=(255, 256))
    hi64, _ = P.solve(pol, precision=PMLBIE_FP64, modes=(255, 256))
    assert r32.backward_error <= 1e-13
    own = {}
    for k in ("u1", "u2"):
        errs[k + "_mode255_of_scale"] = _rel(hi32[k], hi64[k], scale[k])
        own[k] = _rel(hi32[k], hi64[k], torch.linalg.vector_norm(hi64[k]))
    fh32 = P.field(fr, fz, fg, hi32, modes=(255, 256))
    fh64 = P.field(fr, fz, fg, hi64, modes=(255, 256))
    errs["field_mode255_of_scale"] = _rel(fh32, fh64, fscale)
    own["field"] = _rel(fh32, fh64, torch.linalg.vector_norm(fh64))
    print("k1 = %d pi, N = %d: sampled kernels max |diff| / rounding scale %.2e; mixed vs FP64 %s; mode 255 "
          "relative to itself %s" % (k_over_pi, N, worst, {k: "%.1e" % v for k, v in errs.items()},
                                     {k: "%.1e" % v for k, v in own.items()}))
    for k, v in errs.items():
        assert v <= 1e-6, (k, v)
    P.close()
    torch.cuda.empty_cache()
