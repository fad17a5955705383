"""Parity at full size: the benchmark workload (omega_1 = 4 pi, omega_2 = 6 pi,
N = 512, M = 256, the problem bench.py times), the large single instance
(10 pi / 15 pi, N = 1024, M = 512) and the smallest high-frequency instance
(12 pi / 18 pi, N = 1536, M = 512): modal kernels on a sample of node pairs
that the oracle evaluates one by one, and agreement of the mixed and FP64 GPU
solves (FP64 on sampled mode ranges where a full FP64 solve is long)."""
import numpy as np
import pytest

from test_gpu_parity import rounding_scale

pytestmark = pytest.mark.gpu

CFG2 = dict(k1=4 * np.pi, k2=6 * np.pi, N=512, M=256)
CFG4 = dict(k1=10 * np.pi, k2=15 * np.pi, N=1024, M=512)
CFG5 = dict(k1=12 * np.pi, k2=18 * np.pi, N=1536, M=512)


def _take(d, i):
    return {k: (v[i] if isinstance(v, np.ndarray) else v) for k, v in d.items()}


def _sample_pairs(G, Q, rng, n=240):
    """Grid pairs outside the Alpert skip band: random plus neighbours of the
    skip band (close pairs), plus pairs touching breakpoints' neighbours."""
    N = G.P.N
    pairs = set()
    while len(pairs) < n // 2:
        l, m = rng.integers(0, N, 2)
        if Q.grid_mask[l, m]:
            pairs.add((int(l), int(m)))
    gi = G.unk_grid
    for l in rng.integers(0, N, n // 2):
        for d in (10, 11, 14, 20):
            for sgn in (-1, 1):
                tgt = np.nonzero(gi == gi[l] + sgn * d)[0]
                if len(tgt):
                    pairs.add((int(l), int(tgt[0])))
    return sorted(pairs)


class _GridPairs:
    """The oracle quadrature's grid-pair mask alone (|i_m - i_l| >= a of the
    Alpert rule), for sampling pairs at large N without building the whole
    correction table."""

    def __init__(self, G):
        from oracle.assemble import alpert_table
        gi = G.unk_grid
        self.grid_mask = np.abs(gi[:, None] - gi[None, :]) >= alpert_table()[2]


def check_sampled_kernels(cfg, mode_ranges, n_pairs=240, precision=None, factor=1e-12, P=None, light=False):
    """Sampled grid pairs of the library's modal kernels (pmlbie_modal_kernels,
    or pmlbie_modal_kernels_ex in `precision`) against the oracle pair by pair:
    |diff| <= factor x the pair's rounding scale.  Returns the worst ratio.
    P: an existing Problem of cfg; light: sample with the grid-pair mask only."""
    import torch
    import oracle.kernels as KR
    from oracle.assemble import Quadrature
    from oracle.problem import Geometry, Params
    from paper_2412_11162_gb300 import Problem
    if P is None:
        P = Problem(cfg["k1"], cfg["k2"], cfg["N"], cfg["M"])
    Po = Params(**cfg)
    G = Geometry(Po)
    Q = _GridPairs(G) if light else Quadrature(G)
    rng = np.random.default_rng(2412)
    pairs = _sample_pairs(G, Q, rng, n_pairs)
    li = np.array([p[0] for p in pairs])
    mi = np.array([p[1] for p in pairs])
    pg = KR.pair_geometry(_take(G.nodes, li), _take(G.nodes, mi), Po)
    near = KR.near_mask(pg, Po)
    lap = KR.laplace_modes({k: v[near] for k, v in pg.items()}, Po.M - 2)
    assert near.sum() > 20 and (~near).sum() > 20
    worst = 0.0
    for lo, hi in mode_ranges:
        K = P.modal_kernels(lo, hi, precision=precision).cpu().numpy()
        for reg, omega, sign, ks, kk in (("a", Po.k1, 1.0, 0, 1), ("b", Po.k2, -1.0, 2, 3)):
            pgr = dict(pg)
            pgr["nuc_r"] = sign * pg["nuc_r"]
            pgr["nuc_z"] = sign * pg["nuc_z"]
            full = (np.zeros((len(near), Po.M - 1), complex), np.zeros((len(near), Po.M - 1), complex))
            full[0][near] = lap[0]
            full[1][near] = sign * lap[1]
            S, Kr = KR.modal_kernels(pgr, omega, Po, lap=full, near=near)
            for t, n in enumerate(range(lo, hi)):
                for ref, kern, which in ((S[:, n], ks, "S"), (Kr[:, n], kk, "K")):
                    got = K[t, kern][li, mi]
                    d = np.abs(got - ref)
                    # per pair: rounding of the DFT (far) or of the split (close),
                    # relative to the magnitude of its inputs
                    sc = rounding_scale(pgr, near, full, omega, Po.M, Po.taylor_L, n, which)
                    ok = d <= factor * sc + 1e-300     # K == 0 exactly on flat-to-flat pairs
                    ratio = np.where(sc > 0, d / np.where(sc > 0, sc, 1.0), 0.0).max()
                    worst = max(worst, ratio)
                    assert ok.all(), (reg, n, which, ratio)
    return worst


def test_modal_kernels_sampled_pairs_fullsize():
    check_sampled_kernels(CFG2, ((0, 6), (60, 64), (122, 128)))


def test_modal_kernels_sampled_pairs_n1024_m512():
    check_sampled_kernels(CFG4, ((0, 3), (127, 129), (253, 256)), n_pairs=160)


def check_mixed_vs_fp64(cfg, fp64_ranges):
    """Mixed solve of every mode (mode chunks as the memory needs) against FP64
    solves of the given mode ranges: u within 1e-6, refinement residual 1e-13."""
    import time
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    P = Problem(cfg["k1"], cfg["k2"], cfg["N"], cfg["M"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    o32, r32 = P.solve([np.pi / 6], precision=PMLBIE_MIXED)
    torch.cuda.synchronize()
    print("mixed solve %.3f s, chunks %d, refinement %d, residual %.1e, backward error %.1e, "
          "FGMRES modes %d (%d iterations)" % (time.perf_counter() - t0, r32.chunks, r32.refine_iters,
                                               r32.residual, r32.backward_error, r32.gmres_modes, r32.gmres_iters))
    # every mode met |r| <= 1e-13 |B| or |r| <= 1e-14 (|A| |x| + |B|) (else the call raises)
    assert r32.backward_error <= 1e-13
    for lo, hi in fp64_ranges:
        o64, _ = P.solve([np.pi / 6], precision=PMLBIE_FP64, modes=(lo, hi))
        for k in ("u1", "u2"):
            e = (torch.linalg.vector_norm(o32[k][lo:hi] - o64[k]) / torch.linalg.vector_norm(o64[k])).item()
            assert e <= 1e-6, (k, lo, hi, e)


def test_mixed_matches_fp64_n1024_m512():
    check_mixed_vs_fp64(CFG4, ((0, 8), (124, 132), (248, 256)))


def test_mixed_matches_fp64_n1536_m512():
    check_mixed_vs_fp64(CFG5, ((0, 4), (252, 256)))


def test_mixed_matches_fp64_fullsize():
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300.binding import PMLBIE_FP64, PMLBIE_MIXED
    P = Problem(CFG2["k1"], CFG2["k2"], CFG2["N"], CFG2["M"])
    o64, r64 = P.solve([np.pi / 6], precision=PMLBIE_FP64)
    o32, r32 = P.solve([np.pi / 6], precision=PMLBIE_MIXED)
    assert r32.backward_error <= 1e-13
    for k in ("u1", "u2"):
        e = (torch.linalg.vector_norm(o32[k] - o64[k]) / torch.linalg.vector_norm(o64[k])).item()
        assert e <= 1e-6, (k, e)
