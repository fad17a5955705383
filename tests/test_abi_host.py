"""C-ABI library: loads, exports every declared symbol, and its host-side setup
(geometry, Alpert table, diagonal term, parameter checks) agrees with the oracle.
No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2412_11162_gb300 import build as bld
    if not os.path.exists(bld.OUT):
        bld.build()
    from paper_2412_11162_gb300 import binding
    return binding


def test_exports_every_declared_symbol(B):
    hdr = open(os.path.join(ROOT, "include", "pmlbie.h")).read()
    declared = set(re.findall(r"\b(pmlbie_[a-z_]+)\s*\(", hdr))
    assert declared == set(B.EXPORTS)
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_alpert_rule_matches_oracle_table(B):
    from oracle.assemble import alpert_table
    x, w = B.pmlbie_alpert_rule(10, 10)
    xo, wo, a = alpert_table()
    assert np.allclose(x, xo, rtol=2e-15, atol=0) and np.allclose(w, wo, rtol=2e-15, atol=0)


def test_host_tables_match_oracle(B):
    from paper_2412_11162_gb300 import Problem
    from oracle.assemble import Quadrature, diagonal
    from oracle.problem import Geometry, Params
    P = Problem(2 * np.pi, 3 * np.pi, 128, 64)
    nd = P.nodes()
    G = Geometry(Params(k1=2 * np.pi, k2=3 * np.pi, N=128, M=64))
    assert np.abs(G.nodes["rho"] - nd["rho"]).max() < 1e-15
    assert np.abs(G.nodes["z"] - nd["z"]).max() < 1e-15
    assert np.abs(G.nodes["speed"] - nd["speed"]).max() < 1e-14 * np.abs(nd["speed"]).max()
    Da, Db = P.diagonal()
    Dao, Dbo = diagonal(G, Quadrature(G))
    # separations of close points at graded clusters come from breakpoint
    # offsets on both sides, so D agrees even at the nodes next to the corner
    assert np.median(np.abs(Da - Dao)) < 1e-14
    assert np.abs(Da - Dao).max() < 1e-12 and np.abs(Db - Dbo).max() < 1e-12
    assert np.abs(Da + Db + 2).max() < 1e-13


def test_polyline_host_tables(B):
    from paper_2412_11162_gb300 import Problem
    from oracle.problem import Geometry, Params
    V = [(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (4.0, 0.0)]
    P = Problem(2 * np.pi, 2 * np.pi, 120, 48, a1=2.0, T=2.0, S=2.0, curve="polyline", vertices=V)
    G = Geometry(Params(k1=2 * np.pi, k2=2 * np.pi, N=120, M=48, a1=2.0, T=2.0, S=2.0, curve="polyline",
                        vertices=V))
    nd = P.nodes()
    assert np.abs(G.nodes["rho"] - nd["rho"]).max() < 1e-15
    assert np.abs(G.nodes["z"] - nd["z"]).max() < 1e-15


def test_wavy_dent_host_tables(B):
    """Sec. 5 Example 2 curve (kind 2): nodes, speeds and the diagonal term of
    the library's host tables equal the oracle's.  The curve meets the axis at
    an angle; its first segment is graded with exponent 2 (the conical point),
    which both sides apply.  D agrees to ~3e-13 at the tip node (the oracle's
    adaptive disc solid angle), 1e-15 elsewhere."""
    from paper_2412_11162_gb300 import Problem
    from oracle.assemble import Quadrature, diagonal
    from oracle.problem import Geometry, Params
    kw = dict(a1=2.0, T=2.0, S=2.0, curve="wavy", wavy_R=1.0, wavy_eps=0.1, wavy_m=3)
    P = Problem(2 * np.pi, 2.4 * np.pi, 120, 48, **kw)
    G = Geometry(Params(k1=2 * np.pi, k2=2.4 * np.pi, N=120, M=48, **kw))
    nd = P.nodes()
    assert np.abs(G.nodes["rho"] - nd["rho"]).max() < 1e-15
    assert np.abs(G.nodes["z"] - nd["z"]).max() < 1e-15
    assert np.abs(G.nodes["speed"] - nd["speed"]).max() < 1e-13 * np.abs(nd["speed"]).max()
    Da, Db = diagonal(G, Quadrature(G))
    da, db = P.diagonal()
    for ref, got in ((Da, da), (Db, db)):
        assert np.all(np.abs(ref - got) <= 1e-12 * np.maximum(1.0, np.abs(ref)))


@pytest.mark.parametrize("kw,frag", [
    (dict(M=50), "M must be"), (dict(N=8), "N must be"), (dict(k1=-1.0), "wavenumbers"),
    (dict(T=0.0), "PML"), (dict(taylor_L=9), "taylor_L"), (dict(bump_R=3.0), "bump"),
    (dict(curve="wavy", wavy_R=3.0), "wavy"), (dict(curve="wavy", wavy_eps=1.0), "wavy"),
    (dict(curve="wavy", wavy_m=0), "wavy"),
])
def test_parameter_checks(B, kw, frag):
    base = dict(k1=2 * np.pi, k2=3 * np.pi, N=128, M=64)
    base.update(kw)
    k1, k2, N, M = base.pop("k1"), base.pop("k2"), base.pop("N"), base.pop("M")
    params, keep = B.make_params(k1, k2, N, M, **base)
    with pytest.raises(B.PmlbieError) as e:
        B.pmlbie_create(params)
    assert e.value.code == B.PMLBIE_EINVAL and frag in str(e.value)


def test_polyline_must_start_on_axis(B):
    params, keep = B.make_params(1.0, 1.0, 64, 32, curve="polyline", vertices=[(0.5, -1.0), (3.5, 0.0)])
    with pytest.raises(B.PmlbieError):
        B.pmlbie_create(params)


@pytest.mark.parametrize("kw", [
    dict(a1=2.5, T=1.0, S=3.0),
    dict(a1=2.0, T=2.0, S=2.0, curve="wavy", wavy_R=1.0, wavy_eps=0.1, wavy_m=3),
    dict(a1=2.0, T=2.0, S=2.0, curve="polyline", vertices=[(0.0, -1.0), (1.0, -1.0), (1.0, 0.0), (4.0, 0.0)]),
])
def test_node_tables_match_oracle(B, kw):
    """Per-node PML and weight tables: I = int sigma (Sec. 3.1 Eq. (rhot)),
    the conormal of region a (complex inside the PML), and the column weights
    2 rho |r'| and 2 rho equal the oracle's to rounding."""
    from paper_2412_11162_gb300 import Problem
    from oracle.problem import Geometry, Params
    P = Problem(2 * np.pi, 3 * np.pi, 160, 64, **kw)
    t = P.node_tables()
    P.close()
    G = Geometry(Params(k1=2 * np.pi, k2=3 * np.pi, N=160, M=64, **kw))
    pairs = (("I", G.nodes["I"]), ("nuc_r", G.nodes["nuc_r"]), ("nuc_z", G.nodes["nuc_z"]),
             ("Wu", G.nodes["W"]), ("Wphi", 2.0 * G.nodes["rho"]))
    for k, ref in pairs:
        assert np.abs(t[k] - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), k
    assert np.any(np.abs(t["nuc_z"].imag) > 0) and np.all(t["I"] >= 0)   # the PML is reached


def test_workspace_sizing(B):
    """Device workspace reported for a solve of all modes (host arithmetic, no
    device): at least the per-mode complex128 block matrices (M/2 of order 2N)
    in FP64, plus their complex64 copy in mixed precision; growing with the
    number of right-hand sides and with N and M."""
    from paper_2412_11162_gb300 import Problem
    prev = 0
    for N, M in ((96, 32), (128, 64), (192, 96)):
        P = Problem(4 * np.pi, 6 * np.pi, N, M)
        nm, n = M // 2, 2 * N
        w64 = B.pmlbie_workspace_bytes(P.handle, B.PMLBIE_FP64, 1)
        wmx = B.pmlbie_workspace_bytes(P.handle, B.PMLBIE_MIXED, 1)
        wmx8 = B.pmlbie_workspace_bytes(P.handle, B.PMLBIE_MIXED, 8)
        P.close()
        assert w64 >= nm * n * n * 16
        assert wmx >= w64 + nm * n * n * 8
        assert wmx8 > wmx and w64 > prev
        prev = w64
