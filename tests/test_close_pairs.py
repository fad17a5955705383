"""Close-pair classification of the library's host tables against the oracle
(Sec. 4.1 kernel splitting: a pair is split when Re sqrt(d~^2 / (rho~
rho~')) is below the threshold; every Alpert correction pair is listed, the
far ones marked for the plain FFT).  Index work, so the comparison is exact:
the same grid pairs, the same correction pairs with the same flags, the
Taylor-substitution flag of Sec. 4.3 on the pairs with a point in the PML,
and mirror indices that pair (l, m) with (m, l).  No GPU: the list is a host
table."""
import numpy as np
import pytest

from oracle import kernels as KR
from oracle.assemble import Quadrature, _take
from oracle.problem import Geometry, Params

K1, K2 = 2 * np.pi, 2.4 * np.pi
DENT = [(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (4.0, 0.0)]
EX3 = [(0.0, -0.5), (0.5, -0.5), (0.5, -0.7), (0.25, -0.7), (0.25, -1.0), (1.0, -1.0), (1.0, 0.0)]
CASES = {
    "bump": dict(k1=4 * np.pi, k2=6 * np.pi, N=128, M=64),
    "bump_pml": dict(k1=4 * np.pi, k2=6 * np.pi, N=160, M=128, a1=2.5, T=1.0, S=3.0),
    "dent": dict(k1=K1, k2=K1, N=120, M=128, a1=2.0, T=2.0, S=2.0, curve="polyline", vertices=DENT),
    "ex2": dict(k1=K1, k2=K2, N=120, M=48, a1=2.0, T=2.0, S=2.0, curve="wavy"),
    "ex3": dict(k1=K1, k2=K2, N=240, M=48, a1=2.0, T=2.0, S=2.0, curve="polyline", vertices=EX3),
}


def _oracle_lists(P):
    G = Geometry(P)
    Q = Quadrature(G)
    li, mi = np.nonzero(Q.grid_mask)
    tg, sg = _take(G.nodes, li), _take(G.nodes, mi)
    tc = _take(G.nodes, Q.corr_target)
    sc = Q.corr_pts
    tgt = {k: np.concatenate([tg[k], tc[k]]) for k in ("rho", "z", "z_t", "rho_t", "bk", "ox", "oz")}
    src = {k: np.concatenate([sg[k], sc[k]]) for k in ("rho", "z", "z_t", "rho_t", "nuc_r", "nuc_z", "bk", "ox", "oz")}
    pg = KR.pair_geometry(tgt, src, P)
    near = KR.near_mask(pg, P)
    subst = KR.uses_substitution(pg)
    ng = len(li)
    return li, mi, Q.corr_target, near[:ng], near[ng:], subst[:ng], subst[ng:]


@pytest.mark.parametrize("case", sorted(CASES))
def test_close_pairs_match_oracle(case):
    from paper_2412_11162_gb300 import Problem
    kw = dict(CASES[case])
    k1, k2, N, M = kw.pop("k1"), kw.pop("k2"), kw.pop("N"), kw.pop("M")
    P = Problem(k1, k2, N, M, **kw)
    tgt, src, flags, mirror = P.near_pairs()
    ngl, ncl = P.near_count()
    P.close()
    li, mi, ct, gnear, cnear, gsub, csub = _oracle_lists(Params(k1=k1, k2=k2, N=N, M=M, **kw))

    # grid pairs: the same set, in the library's (target, source) order
    want = sorted(zip(li[gnear].tolist(), mi[gnear].tolist()))
    got = list(zip(tgt[:ngl].tolist(), src[:ngl].tolist()))
    assert got == want, (case, len(got), len(want))
    gs = dict(zip(zip(li.tolist(), mi.tolist()), gsub.tolist()))
    assert all(bool(f & 4) == gs[p] for p, f in zip(got, flags[:ngl].tolist()))
    assert not np.any(flags[:ngl] & 3)

    # correction pairs: one per correction point, in the oracle's order
    assert ncl == len(ct)
    assert np.array_equal(tgt[ngl:], ct) and np.array_equal(src[ngl:], np.arange(ncl))
    assert np.all(flags[ngl:] & 1)
    assert np.array_equal((flags[ngl:] & 2) != 0, ~cnear)
    assert np.array_equal((flags[ngl:] & 4) != 0, csub)

    # mirrors: (l, m) <-> (m, l), an involution on the grid pairs
    idx = {p: i for i, p in enumerate(got)}
    for i, (l, m) in enumerate(got):
        j = mirror[i]
        assert j == idx.get((m, l), -1)
        if j >= 0:
            assert mirror[j] == i
    assert np.all(mirror[ngl:] == -1)


@pytest.mark.parametrize("case", ["bump_pml", "ex3"])
def test_alpert_corrections_match_oracle(case):
    """The Alpert correction table (Sec. 4.1): the same targets exactly, the
    same curve parameters, and the same stencil coefficient rows w_k h L(tau)
    per unknown (the two sides' Alpert nodes and weights come from
    independent generators that agree to ~1e-15)."""
    from paper_2412_11162_gb300 import Problem
    kw = dict(CASES[case])
    k1, k2, N, M = kw.pop("k1"), kw.pop("k2"), kw.pop("N"), kw.pop("M")
    P = Problem(k1, k2, N, M, **kw)
    target, tau, m, coef = P.corrections()
    P.close()
    Q = Quadrature(Geometry(Params(k1=k1, k2=k2, N=N, M=M, **kw)))
    assert np.array_equal(target, Q.corr_target)
    assert np.abs(tau - Q.corr_tau).max() < 1e-14
    rows = np.zeros((len(target), N))
    for c in range(len(target)):
        for a in range(m.shape[1]):
            if m[c, a] >= 0:
                rows[c, m[c, a]] += coef[c, a]
            else:
                assert coef[c, a] == 0.0
    scale = np.abs(Q.corr_coef).max()
    assert np.abs(rows - Q.corr_coef).max() < 1e-13 * scale
    # a stencil covers 10 consecutive grid nodes around tau
    assert np.all((m[:, 1:] == -1) | (m[:, :-1] == -1) | (m[:, 1:] == m[:, :-1] + 1))
