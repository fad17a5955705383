"""The allocation-free modal-kernel call (pmlbie_modal_kernels_noalloc) against
the allocating one, through the C ABI, on two calls in a row.

The allocation-free call is for callers that must not call cudaMalloc while
they run; its close-pair scratch is a fixed 64 MiB device array inside the
library.  This file is collected last so that a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_call_twice():
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    assert torch.cuda.is_available()
    P = Problem(2 * np.pi, 3 * np.pi, 128, 64)
    ref = P.modal_kernels()            # allocating call; also puts the tables on the device
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full_like(ref, complex(np.nan, np.nan))
        B.pmlbie_modal_kernels_noalloc(P.handle, 0, P.n_modes, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= 1e-12, err


def test_noalloc_mode_subrange_on_side_stream():
    """A mode range that does not start at 0 (modes 3..8), issued on a
    caller-created stream: the call only enqueues work on that stream, so the
    test synchronises it before reading, and compares with the matching modes
    of the allocating call."""
    import torch
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    P = Problem(2 * np.pi, 3 * np.pi, 128, 64)
    ref = P.modal_kernels()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(side):
            out = torch.full((6, 4, 128, 128), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        B.pmlbie_modal_kernels_noalloc(P.handle, 3, 9, out, stream=side)
        side.synchronize()
        assert torch.isfinite(out).all()
        err = (torch.linalg.vector_norm(out - ref[3:9]) / torch.linalg.vector_norm(ref[3:9])).item()
        assert err <= 1e-12, err


def test_noalloc_rejects_scratch_beyond_limit():
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    P = Problem(4 * np.pi, 6 * np.pi, 512, 256)   # ~0.9 GB of close-pair scratch
    import torch
    out = torch.empty((1, 4, 512, 512), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.PmlbieError) as e:
        B.pmlbie_modal_kernels_noalloc(P.handle, 0, 1, out)
    assert e.value.code == B.PMLBIE_EINVAL and "scratch" in str(e.value)
