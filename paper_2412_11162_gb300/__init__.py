"""GB300 (sm_103a) PML-BIE modal solver for 3D acoustic scattering in a two-layer
medium with an axisymmetric interface perturbation (Wang & Lu, arXiv 2412.11162).

The compute path is libpmlbie.so (hand-written CUDA + host C++); this package is
its thin Python face.  `Problem` (solver.py) is the convenience wrapper and
`binding` holds the raw C-ABI calls.  Importing the package does not load the
library; the first use of `Problem` or `binding` does, and fails loudly if it is
not built.
"""


def __getattr__(name):
    if name in ("Problem", "solve_batch"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
