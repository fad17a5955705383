"""Oracle: PML Green's function samples and modal kernels (FP64, plain sums).

TEST INFRASTRUCTURE ONLY (see oracle/problem.py).

Follows:
  * Sec. 3.1: G~(r, r') = exp(i w |r~ - r~'|) / (4 pi |r~ - r~'|), principal
    square root (branch cut on the negative real axis).
  * Sec. 4.3: stabilised distance |r~ - r~'|^2 = |r~ - r~'|_{rho z}^2
    + 4 rho~ rho~' sin^2(psi / 2).
  * Sec. 4.1, Eqs. (s1), (k1): S~ = Z (H1 + i H2), K~ = D (H3 + i H4) with
    Z = 1/(4 pi |dr|), D = -[nu'_c,rho (rho~' - rho~ cos psi) + nu'_c,z (z~' - z~)]
    / (4 pi |dr|^3), H1 + i H2 = e^{iq}, H3 + i H4 = e^{iq}(1 - iq), q = w |dr|.
  * Sec. 4.1, Eqs. (snspml), (knspml) and the paragraph after them: far pairs by
    the M-point trapezoid (FFT) in psi; close pairs split into a convolution of
    the semi-analytic modal kernels Z_n, D_n with the modes of H1, H3, plus an
    FFT of the smooth remainder.
  * Sec. 4.3, Eq. (ch1): H1 replaced by cH1 = e^{iq} sum_{k<=L} a_k q^k, the
    degree-L Taylor polynomial of H1 e^{-iq}; iH2 replaced by e^{iq} - cH1; the
    same substitution for H3 (cH3) and iH4.

Normalisation: modal kernels are F^_n = int_{-pi}^{pi} e^{-i n psi} F(psi) dpsi
(the paper's (2 pi)^{-1/2} factors cancel out of every equation), so the
convolution of Sec. 3.3, Eq. (con) reads (fg)^_n = (1/2pi) sum_m f^_m g^_{n-m}.

Readings (where the paper is silent):
  * "close" = Re sqrt(2 (chi - 1)) < eta_s with chi - 1 = d^2 / (2 rho~ rho~'),
    d^2 = (rho~ - rho~')^2 + (z~ - z~')^2, eta_s = split_c * 2 pi / M.  This is
    the distance of the kernel's complex singularity from the real psi axis.
  * the substitution of Sec. 4.3 is applied to pairs with a point inside the
    PML (where H1, H3 grow exponentially, the paper's motivation); other close
    pairs keep the exact split H1 = cos q, H3 = cos q + q sin q, whose factors
    are entire in |dr|^2.
  * the convolution runs over |k| <= M/2 - 1 (Nyquist mode dropped), so it
    needs Z^_m, D^_m for |m| <= M - 2.
  * Z^_m, D^_m are the exact integrals; here they are computed by composite
    Gauss-Legendre quadrature in psi, graded geometrically toward psi = 0.
"""
import math

import numpy as np

from .problem import Params, delta_I, separation

FOUR_PI = 4.0 * np.pi


# ----------------------------------------------------------------------------
# pair geometry
# ----------------------------------------------------------------------------
def pair_geometry(tgt, src, P: Params):
    """Pair quantities for broadcastable target/source dicts (see Geometry.at).
    Separations of close points near a breakpoint come from accurate offsets
    (Sec. 4.3: the stabilised distance)."""
    dr, dz = separation(tgt, src)
    drho_t = dr + 1j * delta_I(src["rho"], dr, P)       # rho~ - rho~'
    dz_t = dz + 0j
    rr = tgt["rho_t"] * src["rho_t"]
    d2 = drho_t * drho_t + dz_t * dz_t
    return dict(d2=d2, rr=rr, rho_t=tgt["rho_t"], rho_t_s=src["rho_t"], dz_t=dz_t, drt=-drho_t,
                nuc_r=src["nuc_r"], nuc_z=src["nuc_z"])


def near_mask(pg, P: Params):
    """Close-pair test: Re sqrt(d^2 / (rho~ rho~')) < eta_s."""
    x = pg["d2"] / pg["rr"]
    re_sqrt = np.sqrt(np.maximum((np.abs(x) + x.real) * 0.5, 0.0))
    return re_sqrt < P.eta_split


def _delta2(pg, psi):
    s = np.sin(0.5 * psi)
    return pg["d2"][..., None] + 4.0 * pg["rr"][..., None] * s * s


def _numer_D(pg, psi):
    """nu'_c,rho (rho~' - rho~ cos psi) + nu'_c,z (z~' - z~), evaluated as
    nu'_c,rho [(rho~' - rho~) + 2 rho~ sin^2(psi/2)] + nu'_c,z (z~' - z~) so
    that nothing cancels for close pairs (Sec. 4.3, the stabilised D)."""
    s = np.sin(0.5 * psi)
    return (pg["nuc_r"][..., None] * (pg["drt"][..., None] + 2.0 * pg["rho_t"][..., None] * s * s)
            + pg["nuc_z"][..., None] * (-pg["dz_t"][..., None]))


def kernel_samples(pg, omega, psi):
    """S~(psi), K~(psi) for every pair (rows) and angle (columns)."""
    R = np.sqrt(_delta2(pg, psi))
    q = omega * R
    e = np.exp(1j * q)
    S = e / (FOUR_PI * R)
    D = -_numer_D(pg, psi) / (FOUR_PI * R ** 3)
    K = D * e * (1.0 - 1j * q)
    return S, K


def dft_matrix(M):
    """(2 pi / M) e^{-i n psi_k}, k = 0..M-1 (rows), n = 0..M/2-1 (columns)."""
    k = np.arange(M)[:, None]
    n = np.arange(M // 2)[None, :]
    return (2.0 * np.pi / M) * np.exp(-2j * np.pi * k * n / M)


def far_modes(pg, omega, M):
    """Trapezoid (M-point DFT) modal kernels, n = 0..M/2-1."""
    psi = 2.0 * np.pi * np.arange(M) / M
    S, K = kernel_samples(pg, omega, psi)
    E = dft_matrix(M)
    return S @ E, K @ E


# ----------------------------------------------------------------------------
# Taylor substitution, Sec. 4.3
# ----------------------------------------------------------------------------
def taylor_coeffs(L):
    """Coefficients of P1 = Taylor_L[H1 e^{-iq}], P3 = Taylor_L[H3 e^{-iq}].

    H1 e^{-iq} = (1 + e^{-2iq}) / 2,
    H3 e^{-iq} = (1 + e^{-2iq}) / 2 - i q (1 - e^{-2iq}) / 2.
    """
    e = np.array([(-2j) ** k / math.factorial(k) for k in range(L + 1)])
    a = np.array([((1.0 if k == 0 else 0.0) + e[k]) / 2.0 for k in range(L + 1)])
    b = a.copy()
    for k in range(1, L + 1):
        b[k] += -1j * ((1.0 if k == 1 else 0.0) - e[k - 1]) / 2.0
    return a, b


def _poly(c, q):
    out = np.zeros_like(q)
    for ck in c[::-1]:
        out = out * q + ck
    return out


def _sinc(q):
    """sin(q)/q, with the Taylor series near q = 0."""
    small = np.abs(q) < 1e-3
    qs = np.where(small, 1.0, q)
    ser = 1.0 - q * q / 6.0 + q ** 4 / 120.0
    return np.where(small, ser, np.sin(qs) / qs)


def _h4q3(q):
    """(sin q - q cos q) / q^3, with the Taylor series near q = 0."""
    small = np.abs(q) < 1e-2
    qs = np.where(small, 1.0, q)
    q2 = q * q
    ser = 1.0 / 3.0 - q2 / 30.0 + q2 * q2 / 840.0 - q2 ** 3 / 45360.0
    return np.where(small, ser, (np.sin(qs) - qs * np.cos(qs)) / qs ** 3)


def uses_substitution(pg):
    """cH1/cH3 (Sec. 4.3) for pairs with a point inside the PML (Im rho~ > 0)."""
    return (pg["rho_t"].imag > 0) | (pg["rho_t_s"].imag > 0)


def split_samples(pg, omega, psi, L, subst=True):
    """Smooth factors f1, f3 and remainders r1, r3 of the kernel split.

    S~ = Z f1 + r1 and K~ = D f3 + r3 at every angle, with
      PML pairs (Sec. 4.3):  f1 = cH1 = e^{iq} P1(q),  r1 = Z (e^{iq} - cH1)
                             f3 = cH3 = e^{iq} P3(q),  r3 = D (e^{iq}(1-iq) - cH3)
      other pairs (Sec. 4.1): f1 = H1 = cos q,           r1 = i Z H2
                             f3 = H3 = cos q + q sin q, r3 = i D H4.
    The remainders are written without the removable singularity:
      Z (e^{iq} - cH1) = (w / 4pi) e^{iq} (1 - P1(q)) / q,
      D (e^{iq}(1-iq) - cH3) = -(w^3 / 4pi) N_D e^{iq} ((1 - iq) - P3(q)) / q^3,
      i Z H2 = (i w / 4pi) sin(q)/q,
      i D H4 = -(i w^3 / 4pi) N_D (sin q - q cos q) / q^3,
    (the first three coefficients of (1 - iq) - P3 vanish).  subst=False uses
    the exact split on PML pairs too (complex q).
    """
    a, b = taylor_coeffs(L)
    u1 = -a[1:]                               # (1 - P1)/q
    c3 = -b.copy()
    c3[0] += 1.0
    c3[1] += -1j
    assert np.allclose(c3[:3], 0.0)
    v3 = c3[3:]                               # ((1 - iq) - P3)/q^3
    R = np.sqrt(_delta2(pg, psi))
    q = omega * R
    e = np.exp(1j * q)
    ND = _numer_D(pg, psi)
    sub = (uses_substitution(pg) & bool(subst))[..., None]
    f1 = np.where(sub, e * _poly(a, q), np.cos(q))
    r1 = np.where(sub, (omega / FOUR_PI) * e * _poly(u1, q), (1j * omega / FOUR_PI) * _sinc(q))
    f3 = np.where(sub, e * _poly(b, q), np.cos(q) + q * np.sin(q))
    r3 = np.where(sub, -(omega ** 3 / FOUR_PI) * ND * e * _poly(v3, q),
                  -(1j * omega ** 3 / FOUR_PI) * ND * _h4q3(q))
    return f1, r1, f3, r3


# ----------------------------------------------------------------------------
# exact modal Laplace kernels Z^_m, D^_m (quadrature)
# ----------------------------------------------------------------------------
_GL32 = np.polynomial.legendre.leggauss(32)


def psi_panels(mmax, finest=2.0 ** -52):
    """Panel edges on [0, pi]: geometric toward 0, widths <= 16/(mmax+1)."""
    cap = min(0.25, 16.0 / (mmax + 1))
    edges = [0.0, finest]
    x = finest
    while 2 * x < 1.0:
        x *= 2
        edges.append(x)
    edges.append(np.pi)
    out = [edges[0]]
    for a, b in zip(edges[:-1], edges[1:]):
        k = max(1, int(np.ceil((b - a) / cap)))
        out.extend(list(a + (b - a) * np.arange(1, k + 1) / k))
    return np.array(out)


def psi_rule(mmax, refine=0):
    edges = psi_panels(mmax)
    for _ in range(refine):
        mid = 0.5 * (edges[:-1] + edges[1:])
        edges = np.sort(np.concatenate([edges, mid]))
    x, w = _GL32
    a, b = edges[:-1, None], edges[1:, None]
    pts = (0.5 * (a + b) + 0.5 * (b - a) * x).ravel()
    wts = (0.5 * (b - a) * w).ravel()
    return pts, wts


def laplace_modes(pg, mmax, refine=0, chunk=512):
    """Z^_m and D^_m, m = 0..mmax, by quadrature of 2 int_0^pi cos(m psi) F dpsi."""
    pts, wts = psi_rule(mmax, refine)
    C = 2.0 * wts[:, None] * np.cos(pts[:, None] * np.arange(mmax + 1)[None, :])
    npair = pg["d2"].shape[0]
    Zm = np.empty((npair, mmax + 1), complex)
    Dm = np.empty((npair, mmax + 1), complex)
    for s in range(0, npair, chunk):
        sub = {k: v[s:s + chunk] for k, v in pg.items()}
        R = np.sqrt(_delta2(sub, pts))
        Z = 1.0 / (FOUR_PI * R)
        D = -_numer_D(sub, pts) / (FOUR_PI * R ** 3)
        Zm[s:s + chunk] = Z @ C
        Dm[s:s + chunk] = D @ C
    return Zm, Dm


def near_modes(pg, omega, M, L, lap=None, subst=True):
    """Split modal kernels (S^_n, K^_n), n = 0..M/2-1, for close pairs."""
    if lap is None:
        lap = laplace_modes(pg, M - 2)
    Zm, Dm = lap
    psi = 2.0 * np.pi * np.arange(M) / M
    cH1, rem1, cH3, rem3 = split_samples(pg, omega, psi, L, subst)
    k = np.arange(M)[:, None]
    kk = np.arange(-(M // 2 - 1), M // 2)[None, :]
    Ek = (2.0 * np.pi / M) * np.exp(-2j * np.pi * k * kk / M)     # C_k for k in (-M/2, M/2)
    C1 = cH1 @ Ek
    C3 = cH3 @ Ek
    E = dft_matrix(M)
    R1 = rem1 @ E
    R3 = rem3 @ E
    nh = M // 2
    S = np.empty((pg["d2"].shape[0], nh), complex)
    K = np.empty_like(S)
    kv = np.arange(-(nh - 1), nh)
    for n in range(nh):
        idx = np.abs(n - kv)
        S[:, n] = (Zm[:, idx] * C1).sum(axis=1) / (2.0 * np.pi) + R1[:, n]
        K[:, n] = (Dm[:, idx] * C3).sum(axis=1) / (2.0 * np.pi) + R3[:, n]
    return S, K


def modal_kernels(pg, omega, P: Params, lap=None, near=None):
    """Modal S^_n, K^_n for arbitrary pairs: close pairs split, the rest by FFT."""
    if near is None:
        near = near_mask(pg, P)
    M = P.M
    S = np.empty((pg["d2"].shape[0], M // 2), complex)
    K = np.empty_like(S)
    far = ~near
    if np.any(far):
        sub = {k: v[far] for k, v in pg.items()}
        S[far], K[far] = far_modes(sub, omega, M)
    if np.any(near):
        sub = {k: v[near] for k, v in pg.items()}
        l2 = None if lap is None else (lap[0][near], lap[1][near])
        S[near], K[near] = near_modes(sub, omega, M, P.taylor_L, l2, P.subst)
    return S, K
