"""The allocation-free preconditioner entry point (wfft_precond_noalloc).

It exists for callers that cannot allocate device memory themselves (a host
framework that owns every device byte through its own arena, code that must
not change the allocation state while other work runs): its scratch is a
fixed array inside the library.  Its output must equal the handle-based
wfft_precond and the oracle's preconditioner (Eq. precond, Eq. acous) on the same
input, call after call, since every call reuses the same scratch.  This file is collected last so that a run stopping at its first
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
    from oracle import newmark
    from tests.gpu_util import oracle_field
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(77 + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=3, mask_width=1, contrast=4.0)
    s = wfft.Solver.from_problem(prob)
    cbar, rhobar, theta = _reference_constants(prob)
    stream = torch.cuda.current_stream().cuda_stream
    nm = newmark.oracle_from_problem(prob)
    for call in range(2):
        r = to_dev(torch, rng.standard_normal((ndim, n[2], n[1], n[0])), torch.float64)
        z_ref = torch.zeros_like(r)
        s.precond(r, z_ref, precision=wfft.FP64, masked=False)
        z = torch.full_like(r, float("nan"))
        wfft.precond_noalloc(ndim, n, prob.h, cbar, rhobar, theta, r, z, stream)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), z_ref.cpu().numpy()) < 1e-12, call
        z_oracle = nm.M(oracle_field(prob, r.cpu().numpy()))
        assert rel(oracle_field(prob, z.cpu().numpy()), z_oracle) < 1e-12, call


def test_noalloc_rejects_grids_beyond_its_scratch():
    """A 128^3 grid does not fit the fixed scratch: the library refuses it before any
    device work.  The tensors handed over have the grid's full size, so no launch could
    touch memory outside them even if the size check failed."""
    torch = torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_c3(nsteps=1, n=16, ngrains=4)
    cbar, rhobar, theta = _reference_constants(prob)
    n = (128, 128, 128)
    r = torch.zeros((3, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(wfft.WfftError) as e:
        wfft.precond_noalloc(3, n, (1e-3,) * 3, cbar, rhobar, theta, r, z)
    assert e.value.code == wfft.EINVAL
    assert "too large" in str(e.value)
    torch.cuda.synchronize()
    assert float(z.abs().max()) == 0.0


def test_noalloc_binding_refuses_undersized_buffers():
    """The binding checks the tensors' size, type and placement before calling the library
    (which cannot see the size of a device buffer): nothing is launched."""
    torch = torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_c3(nsteps=1, n=16, ngrains=4)
    cbar, rhobar, theta = _reference_constants(prob)
    n = (16, 16, 16)
    full = torch.zeros((3, 16, 16, 16), dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(3, dtype=torch.float64, device="cuda"),
                torch.zeros((3, 16, 16, 16), dtype=torch.float32, device="cuda"),
                torch.zeros((3, 16, 16, 32), dtype=torch.float64, device="cuda")[..., ::2],
                np.zeros((3, 16, 16, 16))):
        for r, z in ((bad, full), (full, bad)):
            with pytest.raises(wfft.WfftError) as e:
                wfft.precond_noalloc(3, n, (1e-3,) * 3, cbar, rhobar, theta, r, z)
            assert e.value.code == wfft.EINVAL
