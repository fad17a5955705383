"""Exact identities the GPU kernels rely on, checked in numpy on CPU (no
library call): they let one computation serve several outputs, so a wrong
identity would show up only as a parity failure on the GPU.

* Far pairs: K~ of target l, source m is g(psi) (N0 + Ns sin^2(psi/2)) with
  g symmetric in the two nodes; on the M-point DFT of an even sequence,
  sin^2(psi/2) maps G_n to G_n / 2 - (G_{n-1} + G_{n+1}) / 4, so the modes of
  both orientations follow from the DFT of g alone (Sec. 4.1 modes by FFT).
* The even-sequence DFT: the DFT of x_0..x_{M-1} with x_k = x_{M-k} is
  determined by x_0..x_{M/2}, and G_{-n} = G_n (used for G_{-1} = G_1)."""
import numpy as np


def _even_samples(rng, M):
    psi = 2 * np.pi * np.arange(M) / M
    # a smooth even complex function of psi, like the sampled kernels
    a = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    g = sum(a[k] * np.cos(k * psi) / (1 + k * k) for k in range(6))
    g = g * np.exp(0.3j * np.cos(psi)) / (1.2 - np.cos(psi))
    return psi, g


def test_sin2_shift_on_even_dft():
    rng = np.random.default_rng(7)
    for M in (32, 96, 256):
        psi, g = _even_samples(rng, M)
        G = np.fft.fft(g)
        nd0, nds = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        direct = np.fft.fft((nd0 + nds * np.sin(psi / 2) ** 2) * g)
        K = M // 2
        for n in range(K):
            gm = G[1] if n == 0 else G[n - 1]
            shifted = G[n] / 2 - (gm + G[n + 1]) / 4
            assert abs(nd0 * G[n] + nds * shifted - direct[n]) <= 1e-12 * np.abs(direct).max()


def test_even_dft_symmetry():
    rng = np.random.default_rng(8)
    psi, g = _even_samples(rng, 64)
    assert np.allclose(g[1:], g[1:][::-1])          # x_k = x_{M-k}
    G = np.fft.fft(g)
    assert np.allclose(G[1:], G[1:][::-1], atol=1e-12 * np.abs(G).max())   # G_{-n} = G_n


def test_far_flop_model_counts():
    """The bench's algorithmic flop model of the far kernel at M = 256: per
    unordered pair 59,785 flops (a node in the PML) or 41,854 (two physical
    nodes), plus 60 per ordered far pair and mode of the launch."""
    import bench
    assert bench.far_flops_per_launch(256, 128, 1, 0, 0) == 129 * 265 + 4 * (5 * 128 * 7 + 15 * 128) == 59785
    assert bench.far_flops_per_launch(256, 128, 1, 1, 0) == 41854
    assert bench.far_flops_per_launch(256, 16, 0, 0, 3) == 3 * 16 * 60


def test_near_flop_model_counts():
    """The bench's flop model of the close-pair modes kernel at M = 256, all
    128 modes in one launch: 137,015 flops per packed pair, 264,309 per PML
    pair, 64,679 per plain correction pair."""
    import bench
    assert bench.near_flops_per_launch(256, 128, 1, 0, 0) == 137015
    assert bench.near_flops_per_launch(256, 128, 0, 1, 0) == 264309
    assert bench.near_flops_per_launch(256, 128, 0, 0, 1) == 64679
    # a PML pair and its mirror in one CTA: one pair's work + the mirror's extra
    assert bench.near_flops_per_launch(256, 128, 0, 2, 0, 1) == 264309 + 64558
