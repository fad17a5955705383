"""ctypes binding of libpmlbie.so (include/pmlbie.h): argument marshalling only.

Every function keeps the C name.  Device buffers are torch tensors (their
data_ptr is passed); streams are torch.cuda streams.  The library must be
built (paper_2412_11162_gb300.build); importing this module fails loudly if it
is missing, and there is no fallback path.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmlbie.so")

PMLBIE_OK = 0
PMLBIE_EINVAL = -1
PMLBIE_ENOMEM = -2
PMLBIE_ECUDA = -3
PMLBIE_ESINGULAR = -4
PMLBIE_ENOCONVERGE = -5
PMLBIE_ENAN = -6
PMLBIE_ENODEV = -7
PMLBIE_ETIMEOUT = -8
PMLBIE_CURVE_GAUSS_BUMP = 0
PMLBIE_CURVE_POLYLINE = 1
PMLBIE_CURVE_WAVY_DENT = 2
PMLBIE_FP64 = 0
PMLBIE_MIXED = 1


class pmlbie_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
                ("a1", ctypes.c_double), ("T", ctypes.c_double), ("S", ctypes.c_double),
                ("p", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int),
                ("curve_kind", ctypes.c_int), ("bump_h", ctypes.c_double), ("bump_w", ctypes.c_double),
                ("bump_R", ctypes.c_double), ("n_vertices", ctypes.c_int),
                ("vertices", ctypes.POINTER(ctypes.c_double)), ("taylor_L", ctypes.c_int),
                ("split_c", ctypes.c_double), ("wavy_R", ctypes.c_double), ("wavy_eps", ctypes.c_double),
                ("wavy_m", ctypes.c_int), ("subst_off", ctypes.c_int)]


class pmlbie_report(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("n_modes", ctypes.c_int), ("near_pairs", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("residual", ctypes.c_double),
                ("ms_kernels", ctypes.c_double), ("ms_lu", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("ms_far", ctypes.c_double), ("ms_near", ctypes.c_double), ("ms_assemble", ctypes.c_double),
                ("launches", ctypes.c_int), ("far_pairs", ctypes.c_int), ("ms_near_laplace", ctypes.c_double),
                ("chunks", ctypes.c_int), ("chunk_modes", ctypes.c_int), ("gmres_modes", ctypes.c_int),
                ("gmres_iters", ctypes.c_int), ("backward_error", ctypes.c_double),
                ("far_pairs_physical", ctypes.c_int), ("lu_graph_replays", ctypes.c_int),
                ("far_pairs_per_cta", ctypes.c_int), ("far_pairs_sampled", ctypes.c_int),
                ("far_pairs_sampled_physical", ctypes.c_int), ("ms_near_ff", ctypes.c_double),
                ("ms_lu_update", ctypes.c_double), ("lu_update_launches", ctypes.c_int),
                ("ms_far_alone", ctypes.c_double)]


class pmlbie_solve_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("precision", ctypes.c_int), ("n_rhs", ctypes.c_int),
                ("polar", ctypes.POINTER(ctypes.c_double)), ("azimuth", ctypes.POINTER(ctypes.c_double)),
                ("mode_lo", ctypes.c_int), ("mode_hi", ctypes.c_int), ("max_chunk_modes", ctypes.c_int),
                ("workspace_limit", ctypes.c_size_t), ("source_rho", ctypes.POINTER(ctypes.c_double)),
                ("source_z", ctypes.POINTER(ctypes.c_double))]


EXPORTS = ["pmlbie_create", "pmlbie_destroy", "pmlbie_last_error", "pmlbie_nodes", "pmlbie_diagonal",
           "pmlbie_dims", "pmlbie_near_count", "pmlbie_near_pairs", "pmlbie_corrections", "pmlbie_node_tables",
           "pmlbie_alpert_rule", "pmlbie_workspace_bytes",
           "pmlbie_modal_kernels", "pmlbie_modal_kernels_ex", "pmlbie_close_pair_kernels",
           "pmlbie_modal_kernels_noalloc",
           "pmlbie_solve", "pmlbie_solve_ex", "pmlbie_solve_batch", "pmlbie_field", "pmlbie_solve_host",
           "pmlbie_check_finite", "pmlbie_selftest_wait", "pmlbie_selftest_elementary", "pmlbie_selftest_peak"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpmlbie.so is not built (run paper_2412_11162_gb300.build.build()); "
                          "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.pmlbie_create.argtypes = [ctypes.POINTER(pmlbie_params), ctypes.POINTER(vp)]
    lib.pmlbie_create.restype = ctypes.c_int
    lib.pmlbie_destroy.argtypes = [vp]
    lib.pmlbie_destroy.restype = None
    lib.pmlbie_last_error.argtypes = []
    lib.pmlbie_last_error.restype = ctypes.c_char_p
    lib.pmlbie_nodes.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    lib.pmlbie_diagonal.argtypes = [vp, dp, dp, ctypes.c_int]
    lib.pmlbie_near_count.argtypes = [vp, ip, ip]
    lib.pmlbie_dims.argtypes = [vp, ip, ip]
    lib.pmlbie_near_pairs.argtypes = [vp, ip, ip, ip, ip, ctypes.c_int]
    lib.pmlbie_corrections.argtypes = [vp, ip, dp, ip, dp, ctypes.c_int]
    lib.pmlbie_node_tables.argtypes = [vp, dp, dp, dp, dp, dp, ctypes.c_int]
    lib.pmlbie_alpert_rule.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
    lib.pmlbie_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.pmlbie_workspace_bytes.restype = ctypes.c_size_t
    lib.pmlbie_modal_kernels.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.pmlbie_modal_kernels_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.pmlbie_modal_kernels_ex.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.pmlbie_close_pair_kernels.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.pmlbie_solve.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, vp, vp, vp, vp, vp,
                                 ctypes.POINTER(pmlbie_report)]
    lib.pmlbie_solve_host.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, vp,
                                      ctypes.POINTER(pmlbie_report)]
    lib.pmlbie_solve_ex.argtypes = [vp, ctypes.POINTER(pmlbie_solve_opts), vp, vp, vp, vp, vp,
                                    ctypes.POINTER(pmlbie_report)]
    lib.pmlbie_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(pmlbie_solve_opts),
                                       ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp,
                                       ctypes.POINTER(pmlbie_report)]
    lib.pmlbie_field.argtypes = [vp, ctypes.c_int, dp, dp, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                 vp, vp, vp]
    lib.pmlbie_check_finite.argtypes = [vp, ctypes.c_size_t, vp]
    lib.pmlbie_selftest_wait.argtypes = [ctypes.c_longlong, vp]
    lib.pmlbie_selftest_elementary.argtypes = [ctypes.c_int, vp, vp, ctypes.c_size_t, vp]
    lib.pmlbie_selftest_peak.argtypes = [ctypes.c_int, dp, vp]
    for f in ("pmlbie_check_finite", "pmlbie_selftest_wait", "pmlbie_selftest_elementary", "pmlbie_selftest_peak", "pmlbie_nodes", "pmlbie_diagonal",
              "pmlbie_dims", "pmlbie_near_count", "pmlbie_near_pairs", "pmlbie_corrections", "pmlbie_node_tables",
              "pmlbie_alpert_rule",
              "pmlbie_modal_kernels", "pmlbie_modal_kernels_noalloc", "pmlbie_modal_kernels_ex",
              "pmlbie_close_pair_kernels", "pmlbie_solve", "pmlbie_solve_ex",
              "pmlbie_solve_batch", "pmlbie_field", "pmlbie_solve_host"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


lib = _load()


class PmlbieError(RuntimeError):
    def __init__(self, code, where, message=None):
        self.code = code
        text = message if message is not None else lib.pmlbie_last_error().decode()
        super().__init__("%s failed (%d): %s" % (where, code, text))


def check(code, where):
    if code != PMLBIE_OK:
        raise PmlbieError(code, where)
    return code


def _dptr(a):
    """double* of a contiguous float64 numpy array."""
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check_dev(t, numel, where, name):
    """A device buffer handed to the library: None, or a contiguous complex128
    CUDA tensor on the current device with exactly `numel` elements.  The
    library writes or reads numel elements through the raw pointer, so a
    smaller tensor, another dtype or a strided view would be overrun;
    PmlbieError(EINVAL) before any device work instead."""
    if t is None:
        return
    import torch
    bad = None
    if not isinstance(t, torch.Tensor):
        bad = "is not a torch tensor"
    elif not t.is_cuda:
        bad = "is not a CUDA tensor"
    elif t.dtype != torch.complex128:
        bad = "has dtype %s, not complex128" % t.dtype
    elif not t.is_contiguous():
        bad = "is not contiguous"
    elif t.numel() != numel:
        bad = "has %d elements, the call needs %d" % (t.numel(), numel)
    elif t.device.index != torch.cuda.current_device():
        bad = "is on cuda:%d, the current device is cuda:%d" % (t.device.index, torch.cuda.current_device())
    if bad:
        raise PmlbieError(PMLBIE_EINVAL, where, "%s %s" % (name, bad))


def _mode_count(h, mode_lo, mode_hi):
    """Modes of a call's mode range (mode_lo = mode_hi = 0: all M/2)."""
    _, M = pmlbie_dims(h)
    if mode_lo == 0 and mode_hi == 0:
        return M // 2
    return max(mode_hi - mode_lo, 0)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_params(k1, k2, N, M, a1=2.5, T=1.0, S=3.0, p=6, curve="gauss", bump_h=0.2, bump_w=0.5,
                bump_R=1.0, vertices=None, taylor_L=5, split_c=8.0, wavy_R=1.0, wavy_eps=0.1, wavy_m=3,
                subst=True):
    import numpy as np
    P = pmlbie_params()
    P.struct_size = ctypes.sizeof(pmlbie_params)
    P.k1, P.k2, P.a1, P.T, P.S, P.p, P.N, P.M = k1, k2, a1, T, S, p, N, M
    P.bump_h, P.bump_w, P.bump_R = bump_h, bump_w, bump_R
    P.taylor_L, P.split_c = taylor_L, split_c
    keep = None
    P.wavy_R, P.wavy_eps, P.wavy_m = wavy_R, wavy_eps, wavy_m
    P.subst_off = 0 if subst else 1
    if curve == "gauss":
        P.curve_kind = PMLBIE_CURVE_GAUSS_BUMP
    elif curve == "wavy":
        P.curve_kind = PMLBIE_CURVE_WAVY_DENT
    else:
        P.curve_kind = PMLBIE_CURVE_POLYLINE
        keep = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64).reshape(-1))
        P.n_vertices = len(keep) // 2
        P.vertices = _dptr(keep)
    return P, keep


def pmlbie_create(params):
    h = ctypes.c_void_p()
    check(lib.pmlbie_create(ctypes.byref(params), ctypes.byref(h)), "pmlbie_create")
    return h


def pmlbie_destroy(h):
    lib.pmlbie_destroy(h)


def pmlbie_nodes(h, N):
    import numpy as np
    out = [np.empty(N) for _ in range(4)]
    check(lib.pmlbie_nodes(h, *[_dptr(a) for a in out], N), "pmlbie_nodes")
    return dict(rho=out[0], z=out[1], speed=out[2], t=out[3])


def pmlbie_diagonal(h, N):
    import numpy as np
    Da, Db = np.empty(N), np.empty(N)
    check(lib.pmlbie_diagonal(h, _dptr(Da), _dptr(Db), N), "pmlbie_diagonal")
    return Da, Db


def pmlbie_dims(h):
    """(N, M) of a problem."""
    n, m = ctypes.c_int(), ctypes.c_int()
    check(lib.pmlbie_dims(h, ctypes.byref(n), ctypes.byref(m)), "pmlbie_dims")
    return n.value, m.value


def pmlbie_near_count(h):
    a, b = ctypes.c_int(), ctypes.c_int()
    check(lib.pmlbie_near_count(h, ctypes.byref(a), ctypes.byref(b)), "pmlbie_near_count")
    return a.value, b.value


def pmlbie_near_pairs(h):
    """(tgt, src, flags, mirror) int32 arrays of the close-pair list."""
    import numpy as np
    g, c = pmlbie_near_count(h)
    n = g + c
    out = [np.zeros(n, dtype=np.int32) for _ in range(4)]
    ptr = [o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for o in out]
    check(lib.pmlbie_near_pairs(h, *ptr, n), "pmlbie_near_pairs")
    return tuple(out)


PMLBIE_STENCIL = 10


def pmlbie_node_tables(h, N):
    """dict of the per-node PML and weight tables: I, nuc_r, nuc_z (complex),
    Wu, Wphi."""
    import numpy as np
    I, Wu, Wphi = np.zeros(N), np.zeros(N), np.zeros(N)
    nr, nz = np.zeros(2 * N), np.zeros(2 * N)
    check(lib.pmlbie_node_tables(h, _dptr(I), _dptr(nr), _dptr(nz), _dptr(Wu), _dptr(Wphi), N),
          "pmlbie_node_tables")
    return {"I": I, "nuc_r": nr[0::2] + 1j * nr[1::2], "nuc_z": nz[0::2] + 1j * nz[1::2], "Wu": Wu, "Wphi": Wphi}


def pmlbie_corrections(h):
    """(target, tau, m, coef) of the Alpert correction table; m and coef are
    (n_corr, PMLBIE_STENCIL)."""
    import numpy as np
    _, n = pmlbie_near_count(h)
    t = np.zeros(n, dtype=np.int32)
    tau = np.zeros(n)
    m = np.zeros((n, PMLBIE_STENCIL), dtype=np.int32)
    coef = np.zeros((n, PMLBIE_STENCIL))
    ip = ctypes.POINTER(ctypes.c_int)
    check(lib.pmlbie_corrections(h, t.ctypes.data_as(ip), _dptr(tau), m.ctypes.data_as(ip), _dptr(coef), n),
          "pmlbie_corrections")
    return t, tau, m, coef


def pmlbie_alpert_rule(j, a):
    import numpy as np
    x, w = np.empty(j), np.empty(j)
    check(lib.pmlbie_alpert_rule(j, a, _dptr(x), _dptr(w)), "pmlbie_alpert_rule")
    return x, w


def pmlbie_workspace_bytes(h, precision, n_rhs):
    return lib.pmlbie_workspace_bytes(h, precision, n_rhs)


def pmlbie_modal_kernels(h, mode_lo, mode_hi, out, stream=None):
    """out: complex128 CUDA tensor of (mode_hi-mode_lo)*4*N*N elements."""
    N, _ = pmlbie_dims(h)
    _check_dev(out, max(mode_hi - mode_lo, 0) * 4 * N * N, "pmlbie_modal_kernels", "out")
    check(lib.pmlbie_modal_kernels(h, mode_lo, mode_hi, _tptr(out), _stream(stream)), "pmlbie_modal_kernels")
    return out


def pmlbie_modal_kernels_ex(h, precision, mode_lo, mode_hi, out, stream=None):
    """Modal kernels in the arithmetic of `precision` (same layout as
    pmlbie_modal_kernels)."""
    N, _ = pmlbie_dims(h)
    _check_dev(out, max(mode_hi - mode_lo, 0) * 4 * N * N, "pmlbie_modal_kernels_ex", "out")
    check(lib.pmlbie_modal_kernels_ex(h, precision, mode_lo, mode_hi, _tptr(out), _stream(stream)),
          "pmlbie_modal_kernels_ex")
    return out


def pmlbie_close_pair_kernels(h, precision, mode_lo, mode_hi, out, stream=None):
    """Split modal kernels of every close pair, [pair][kernel][mode]."""
    g, c = pmlbie_near_count(h)
    _check_dev(out, (g + c) * 4 * max(mode_hi - mode_lo, 0), "pmlbie_close_pair_kernels", "out")
    check(lib.pmlbie_close_pair_kernels(h, precision, mode_lo, mode_hi, _tptr(out), _stream(stream)),
          "pmlbie_close_pair_kernels")
    return out


def pmlbie_modal_kernels_noalloc(h, mode_lo, mode_hi, out, stream=None):
    """Allocation-free modal kernels into out (same layout as pmlbie_modal_kernels)."""
    N, _ = pmlbie_dims(h)
    _check_dev(out, max(mode_hi - mode_lo, 0) * 4 * N * N, "pmlbie_modal_kernels_noalloc", "out")
    check(lib.pmlbie_modal_kernels_noalloc(h, mode_lo, mode_hi, _tptr(out), _stream(stream)),
          "pmlbie_modal_kernels_noalloc")
    return out


def pmlbie_solve(h, precision, polar, u1=None, phi1=None, u2=None, phi2=None, stream=None,
                 allow_noconverge=False):
    import numpy as np
    pol = np.ascontiguousarray(np.asarray(polar, dtype=np.float64).reshape(-1))
    N, M = pmlbie_dims(h)
    for name, t in (("u1", u1), ("phi1", phi1), ("u2", u2), ("phi2", phi2)):
        _check_dev(t, (M // 2) * N * len(pol), "pmlbie_solve", name)
    rep = pmlbie_report()
    rep.struct_size = ctypes.sizeof(pmlbie_report)
    rc = lib.pmlbie_solve(h, precision, len(pol), _dptr(pol), _tptr(u1), _tptr(phi1), _tptr(u2), _tptr(phi2),
                          _stream(stream), ctypes.byref(rep))
    if not (allow_noconverge and rc == PMLBIE_ENOCONVERGE):
        check(rc, "pmlbie_solve")
    return rep


def pmlbie_solve_ex(h, precision, polar, azimuth=None, mode_lo=0, mode_hi=0, max_chunk_modes=0,
                    workspace_limit=0, u1=None, phi1=None, u2=None, phi2=None, stream=None,
                    allow_noconverge=False, sources=None):
    o, keep = make_opts(precision, polar, azimuth, mode_lo, mode_hi, max_chunk_modes, workspace_limit, sources)
    N, _ = pmlbie_dims(h)
    for name, t in (("u1", u1), ("phi1", phi1), ("u2", u2), ("phi2", phi2)):
        _check_dev(t, _mode_count(h, mode_lo, mode_hi) * N * o.n_rhs, "pmlbie_solve_ex", name)
    rep = pmlbie_report()
    rep.struct_size = ctypes.sizeof(pmlbie_report)
    rc = lib.pmlbie_solve_ex(h, ctypes.byref(o), _tptr(u1), _tptr(phi1), _tptr(u2), _tptr(phi2), _stream(stream),
                             ctypes.byref(rep))
    del keep
    if not (allow_noconverge and rc == PMLBIE_ENOCONVERGE):
        check(rc, "pmlbie_solve_ex")
    return rep


def make_opts(precision, polar, azimuth=None, mode_lo=0, mode_hi=0, max_chunk_modes=0, workspace_limit=0,
              sources=None):
    """pmlbie_solve_opts and the arrays it points to (keep both alive).  polar:
    plane-wave polar angles; or polar None and sources: (n, 2) point sources
    (rho_s, z_s) in the upper medium."""
    import numpy as np
    o = pmlbie_solve_opts()
    o.struct_size = ctypes.sizeof(pmlbie_solve_opts)
    if sources is not None:
        if polar is not None:
            raise ValueError("give either polar angles or point sources")
        src = np.asarray(sources, dtype=np.float64).reshape(-1, 2)
        rs, zs = np.ascontiguousarray(src[:, 0]), np.ascontiguousarray(src[:, 1])
        o.source_rho, o.source_z, o.polar = _dptr(rs), _dptr(zs), None
        n, keep = len(rs), [rs, zs]
    else:
        pol = np.ascontiguousarray(np.asarray(polar, dtype=np.float64).reshape(-1))
        o.polar = _dptr(pol)
        n, keep = len(pol), [pol]
    az = None if azimuth is None else np.ascontiguousarray(np.asarray(azimuth, dtype=np.float64).reshape(-1))
    if az is not None and len(az) != n:
        raise ValueError("one azimuth per wave or source")
    o.precision, o.n_rhs = precision, n
    o.azimuth = _dptr(az) if az is not None else None
    o.mode_lo, o.mode_hi, o.max_chunk_modes, o.workspace_limit = mode_lo, mode_hi, max_chunk_modes, workspace_limit
    return o, (keep, az)


def pmlbie_solve_batch(handles, opts, u1=None, phi1=None, u2=None, phi2=None, n_streams=2,
                       release_workspace=False, stream=None):
    """handles: problem handles; opts: list of pmlbie_solve_opts; u1..phi2: lists
    of device tensors (or None).  Returns the list of reports."""
    n = len(handles)
    for i, (hh, o) in enumerate(zip(handles, opts)):
        N, _ = pmlbie_dims(hh)
        need = _mode_count(hh, o.mode_lo, o.mode_hi) * N * o.n_rhs
        for name, ts in (("u1", u1), ("phi1", phi1), ("u2", u2), ("phi2", phi2)):
            if ts is not None:
                _check_dev(ts[i], need, "pmlbie_solve_batch", "%s[%d]" % (name, i))
    H = (ctypes.c_void_p * n)(*handles)
    O = (pmlbie_solve_opts * n)(*opts)

    def arr(ts):
        return None if ts is None else (ctypes.c_void_p * n)(*[_tptr(t) for t in ts])

    reps = (pmlbie_report * n)()
    for r in reps:
        r.struct_size = ctypes.sizeof(pmlbie_report)
    check(lib.pmlbie_solve_batch(H, n, O, arr(u1), arr(phi1), arr(u2), arr(phi2), n_streams,
                                 1 if release_workspace else 0, _stream(stream), reps), "pmlbie_solve_batch")
    return list(reps)


def pmlbie_field(h, rho, z, region, n_rhs, u1, phi1, u2, phi2, out, mode_lo=0, mode_hi=0, stream=None):
    import numpy as np
    r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(-1))
    g = np.ascontiguousarray(np.asarray(region, dtype=np.int32).reshape(-1))
    if not (len(r) == len(zz) == len(g)):
        raise ValueError("rho, z and region differ in length")
    N, _ = pmlbie_dims(h)
    nm = _mode_count(h, mode_lo, mode_hi)
    for name, t in (("u1", u1), ("phi1", phi1), ("u2", u2), ("phi2", phi2)):
        _check_dev(t, nm * N * n_rhs, "pmlbie_field", name)
    _check_dev(out, nm * len(r) * n_rhs, "pmlbie_field", "out")
    check(lib.pmlbie_field(h, len(r), _dptr(r), _dptr(zz), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), mode_lo,
                           mode_hi, n_rhs, _tptr(u1), _tptr(phi1), _tptr(u2), _tptr(phi2), _tptr(out),
                           _stream(stream)), "pmlbie_field")


def pmlbie_solve_host(h, precision, polar, u1, phi1, u2, phi2, stream=None):
    """Host outputs: complex128 numpy arrays (any may be None)."""
    import numpy as np
    pol = np.ascontiguousarray(np.asarray(polar, dtype=np.float64).reshape(-1))
    N, M = pmlbie_dims(h)
    for name, a in (("u1", u1), ("phi1", phi1), ("u2", u2), ("phi2", phi2)):
        if a is None:
            continue
        if not (isinstance(a, np.ndarray) and a.dtype == np.complex128 and a.flags.c_contiguous
                and a.size == (M // 2) * N * len(pol)):
            raise PmlbieError(PMLBIE_EINVAL, "pmlbie_solve_host",
                              "%s must be a C-contiguous complex128 array of %d elements" %
                              (name, (M // 2) * N * len(pol)))
    rep = pmlbie_report()
    rep.struct_size = ctypes.sizeof(pmlbie_report)

    def hp(a):
        return ctypes.POINTER(ctypes.c_double)() if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib.pmlbie_solve_host(h, precision, len(pol), _dptr(pol), hp(u1), hp(phi1), hp(u2), hp(phi2),
                                _stream(stream), ctypes.byref(rep)), "pmlbie_solve_host")
    return rep


def pmlbie_check_finite(t, stream=None):
    """Status of the NaN / Inf scan of a complex128 device tensor (no raise
    for the scan's result; a tensor that is not a contiguous complex128 CUDA
    tensor raises PmlbieError(EINVAL))."""
    if t is not None:
        _check_dev(t, t.numel(), "pmlbie_check_finite", "t")
    return lib.pmlbie_check_finite(_tptr(t), t.numel(), _stream(stream))


def pmlbie_selftest_wait(iterations, stream=None):
    """Status of the bounded-wait self-test (ETIMEOUT expected; no raise)."""
    return lib.pmlbie_selftest_wait(int(iterations), _stream(stream))


def pmlbie_selftest_elementary(fn, x, out, stream=None):
    """Evaluate elementary-function selector fn (include/pmlbie.h) at the
    float64 CUDA tensor x into the float64 CUDA tensor out (len(x) values, or
    2 len(x) for the sin / cos selectors)."""
    import torch
    for name, t, want in (("x", x, x.numel()), ("out", out, x.numel() * (2 if fn % 10 == 1 else 1))):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == want):
            raise PmlbieError(PMLBIE_EINVAL, "pmlbie_selftest_elementary",
                              "%s must be a contiguous float64 CUDA tensor of %d elements" % (name, want))
    check(lib.pmlbie_selftest_elementary(fn, _tptr(x), _tptr(out), x.numel(), _stream(stream)),
          "pmlbie_selftest_elementary")
    return out


def pmlbie_selftest_peak(kind, stream=None):
    """Measured TFLOP/s of the FP64 FMA (0), FP32 FMA (1) or TF32 tensor-core
    (2) pipe."""
    v = ctypes.c_double(0.0)
    check(lib.pmlbie_selftest_peak(int(kind), ctypes.byref(v), _stream(stream)), "pmlbie_selftest_peak")
    return v.value
