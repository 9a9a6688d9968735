"""The paper's Green's-matrix treatment of the prescribed region (Alg. 2) on the
GPU against the oracle's literal form and against the masked solve of wfft_step:
all three give the same displacements up to the solver tolerance."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ndim,n", [(3, (12, 10, 8)), (2, (20, 16, 1))])
def test_green_steps_match_masked_steps_and_the_literal_reference(ndim, n):
    from oracle import green, newmark
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(41 + ndim), ndim, n, nphase=3, mask_width=1, nsteps=3,
                                 contrast=3.0)
    opt = lambda: wfft.default_options(precision=wfft.FP64, tol=1e-13, maxit=2000)
    g = wfft.Solver.from_problem(prob, options=opt())
    g.green_setup()
    m = wfft.Solver.from_problem(prob, options=opt())
    for k in range(prob.nsteps):
        ig = g.green_step(prob.U[k])
        im = m.step(prob.U[k])
        assert ig["status"] == 0 and im["status"] == 0
        assert np.allclose(ig["reaction"][:ndim], im["reaction"][:ndim], rtol=1e-8,
                           atol=1e-8 * max(1e-300, np.abs(im["reaction"][:ndim]).max()))
    ug, um = g.get_state()[0], m.get_state()[0]
    g.close()
    m.close()
    assert rel(ug, um) < 1e-10
    lit, _ = green.GreenNewmark(newmark.oracle_from_problem(prob, tol=1e-14)).run(prob.U)
    assert rel(oracle_field(prob, ug), lit.u) < 1e-10


def test_green_setup_limits():
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(2), 3, (12, 10, 8), nphase=2, mask_width=1, nsteps=1)
    s = wfft.Solver.from_problem(prob)
    with pytest.raises(wfft.WfftError) as e:
        s.green_setup(max_dofs=10)
    assert e.value.code == wfft.EINVAL
    with pytest.raises(wfft.WfftError) as e:
        s.green_step(prob.U[0])
    assert e.value.code == wfft.EINVAL
    s.close()
    mixed = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=wfft.MIXED))
    with pytest.raises(wfft.WfftError) as e:
        mixed.green_setup()
    assert e.value.code == wfft.EINVAL
    mixed.close()
