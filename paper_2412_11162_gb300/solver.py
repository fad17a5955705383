"""Convenience wrapper over the C ABI (device buffers from torch)."""
import numpy as np

from . import binding as B


class Problem:
    """One problem instance: host tables built at construction, device upload on
    first use.  Parameters follow pmlbie_params (include/pmlbie.h)."""

    def __init__(self, k1, k2, N, M, **kw):
        self.params, self._keep = B.make_params(k1, k2, N, M, **kw)
        self.N, self.M = N, M
        self.handle = B.pmlbie_create(self.params)

    def close(self):
        if self.handle:
            B.pmlbie_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_modes(self):
        return self.M // 2

    def nodes(self):
        return B.pmlbie_nodes(self.handle, self.N)

    def diagonal(self):
        return B.pmlbie_diagonal(self.handle, self.N)

    def near_count(self):
        return B.pmlbie_near_count(self.handle)

    def near_pairs(self):
        return B.pmlbie_near_pairs(self.handle)

    def corrections(self):
        return B.pmlbie_corrections(self.handle)

    def node_tables(self):
        return B.pmlbie_node_tables(self.handle, self.N)

    def modal_kernels(self, mode_lo=0, mode_hi=None, stream=None, precision=None):
        """[mode][kernel][l][m] complex128; precision None: pmlbie_modal_kernels
        (FP64), else pmlbie_modal_kernels_ex in that precision's arithmetic."""
        import torch
        mode_hi = self.n_modes if mode_hi is None else mode_hi
        out = torch.empty((mode_hi - mode_lo, 4, self.N, self.N), dtype=torch.complex128, device="cuda")
        if precision is None:
            B.pmlbie_modal_kernels(self.handle, mode_lo, mode_hi, out, stream)
        else:
            B.pmlbie_modal_kernels_ex(self.handle, precision, mode_lo, mode_hi, out, stream)
        return out

    def field(self, rho, z, region, densities, modes=None, stream=None):
        """Scattered-field modes [mode][point][rhs] at points (rho, z) of the
        upper (region 0) or lower (1) medium from solve outputs `densities`
        (dict u1, phi1, u2, phi2 for the same mode range)."""
        import torch
        lo, hi = (0, self.n_modes) if modes is None else modes
        nrhs = densities["u1"].shape[2]
        out = torch.empty((hi - lo, len(np.atleast_1d(rho)), nrhs), dtype=torch.complex128, device="cuda")
        B.pmlbie_field(self.handle, rho, z, region, nrhs, densities["u1"], densities["phi1"], densities["u2"],
                       densities["phi2"], out, lo, hi, stream)
        return out

    def solve(self, polar=None, precision=B.PMLBIE_FP64, stream=None, outputs=None, allow_noconverge=False,
              azimuth=None, modes=None, max_chunk_modes=0, workspace_limit=0, sources=None):
        """Device solve; returns (dict of [mode][node][rhs] complex128 tensors, report).
        polar: plane-wave polar angles; or sources = [(rho_s, z_s), ...] point
        sources in the upper medium (polar None).  modes = (lo, hi) solves modes
        lo..hi-1 only; azimuth: one incidence (or source) azimuth per wave;
        max_chunk_modes / workspace_limit bound the modes factored at once."""
        import torch
        if (polar is None) == (sources is None):
            raise ValueError("give either polar angles or point sources")
        n_rhs = len(np.atleast_1d(np.asarray(polar, dtype=np.float64))) if sources is None else \
            len(np.asarray(sources, dtype=np.float64).reshape(-1, 2))
        lo, hi = (0, self.n_modes) if modes is None else modes
        if outputs is None:
            shape = (max(hi - lo, 0), self.N, n_rhs)   # the library rejects empty or bad ranges
            outputs = {k: torch.empty(shape, dtype=torch.complex128, device="cuda")
                       for k in ("u1", "phi1", "u2", "phi2")}
        if sources is None and azimuth is None and modes is None and max_chunk_modes == 0 and workspace_limit == 0:
            rep = B.pmlbie_solve(self.handle, precision, np.atleast_1d(np.asarray(polar, dtype=np.float64)),
                                 outputs["u1"], outputs["phi1"], outputs["u2"], outputs["phi2"], stream,
                                 allow_noconverge=allow_noconverge)
        else:
            rep = B.pmlbie_solve_ex(self.handle, precision, polar, azimuth, lo, hi, max_chunk_modes,
                                    workspace_limit, outputs["u1"], outputs["phi1"], outputs["u2"],
                                    outputs["phi2"], stream, allow_noconverge=allow_noconverge, sources=sources)
        return outputs, rep


def solve_batch(problems, polar, azimuth=None, precision=B.PMLBIE_MIXED, n_streams=2, release_workspace=False,
                stream=None):
    """Solve several Problem instances for the same plane waves in one batch
    call (pmlbie_solve_batch).  Returns ([outputs dict per problem], [reports])."""
    import torch
    opts, keep, outs = [], [], []
    for P in problems:
        o, k = B.make_opts(precision, polar, azimuth)
        opts.append(o)
        keep.append(k)
        shape = (P.n_modes, P.N, o.n_rhs)
        outs.append({key: torch.empty(shape, dtype=torch.complex128, device="cuda")
                     for key in ("u1", "phi1", "u2", "phi2")})
    reps = B.pmlbie_solve_batch([P.handle for P in problems], opts, [o["u1"] for o in outs],
                                [o["phi1"] for o in outs], [o["u2"] for o in outs], [o["phi2"] for o in outs],
                                n_streams, release_workspace, stream)
    return outs, reps
