"""The allocation-free preconditioner entry point (wfft_precond_noalloc).

It exists for callers that cannot allocate device memory themselves (a host
framework that owns every device byte through its own arena, code that must
not change the allocation state while other work runs): its scratch is a
fixed array inside the library.  Its output must equal the handle-based
wfft_precond on the same input, call after call, since every call reuses the
same scratch.  This file is collected last so that a run stopping at its first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _reference_constants(prob):
    """Volume averages of C and rho (the paper's reference medium) and theta."""
    counts = np.bincount(prob.phase.reshape(-1), minlength=prob.C.shape[0]).astype(np.float64)
    cbar = counts @ prob.C / prob.nvox
    rhobar = float(counts @ prob.rho / prob.nvox)
    return cbar, rhobar, prob.beta * prob.dt ** 2


@pytest.mark.parametrize("ndim,n", [(3, (24, 20, 16)), (2, (64, 48, 1))])
def test_noalloc_precond_matches_handle_precond_on_consecutive_calls(ndim, n):
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(77 + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=3, mask_width=1, contrast=4.0)
    s = wfft.Solver.from_problem(prob)
    cbar, rhobar, theta = _reference_constants(prob)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        r = to_dev(torch, rng.standard_normal((ndim, n[2], n[1], n[0])), torch.float64)
        z_ref = torch.zeros_like(r)
        s.precond(r, z_ref, precision=wfft.FP64, masked=False)
        z = torch.full_like(r, float("nan"))
        wfft.precond_noalloc(ndim, n, prob.h, cbar, rhobar, theta, r, z, stream)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), z_ref.cpu().numpy()) < 1e-12, call


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_c3(nsteps=1, n=16, ngrains=4)
    cbar, rhobar, theta = _reference_constants(prob)
    r = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(wfft.WfftError) as e:
        wfft.precond_noalloc(3, (128, 128, 128), (1e-3,) * 3, cbar, rhobar, theta, r, r)
    assert e.value.code == wfft.EINVAL
