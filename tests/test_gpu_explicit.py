"""Explicit central-difference scheme (Sec. 2.3) on the GPU against the FP64
reference of oracle/explicit.py: same arithmetic without a solve, so the states
agree to rounding."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _explicit_solver(wfft, prob):
    return wfft.Solver(prob.ndim, prob.n, prob.h, prob.C, prob.rho, prob.phase, prob.mask, prob.dt,
                       beta=0.0, gamma=0.5)


def _udot(nsteps, dt, amp=1e-2, width=2e-6):
    t = dt * np.arange(1, nsteps + 1)
    U = np.zeros((nsteps, 3))
    U[:, 0] = amp * np.sin(np.pi * np.clip(t / width, 0, 1)) ** 2
    U[:, 1] = -0.3 * U[:, 0]
    return U


@pytest.mark.parametrize("ndim,n", [(3, (20, 16, 12)), (2, (24, 18, 1))])
def test_explicit_steps_match_the_reference(ndim, n):
    from oracle import explicit, medium
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(91 + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=3, mask_width=2, nsteps=1, contrast=3.0)
    dt = 0.8 * wfft.explicit_dt(ndim, prob.h, prob.C, prob.rho)
    prob.dt = dt
    nsteps = 15
    Ud = _udot(nsteps, dt)
    s = _explicit_solver(wfft, prob)
    infos = [s.explicit_step(Ud[k]) for k in range(nsteps)]
    u, v, a, nstep = s.get_state()
    s.close()
    assert nstep == nsteps and all(i["status"] == 0 and i["iters"] == 0 for i in infos)
    nm = explicit.ExplicitOracle(medium.medium_from_problem(prob), medium.mask_to_oracle(prob), dt)
    so, reactions = nm.run(Ud)
    assert rel(oracle_field(prob, u), so.u) < 1e-11
    assert rel(oracle_field(prob, v), so.v) < 1e-11
    assert rel(oracle_field(prob, a), so.a) < 1e-10
    last = np.array(reactions[-1][:ndim])
    assert np.abs(np.array(infos[-1]["reaction"][:ndim]) - last).max() <= 1e-9 * np.abs(last).max()


def test_explicit_and_implicit_entry_points_are_kept_apart():
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(3), 3, (12, 10, 8), nphase=2, mask_width=1, nsteps=1)
    ex = _explicit_solver(wfft, prob)
    with pytest.raises(wfft.WfftError) as e:
        ex.step(prob.U[0])
    assert e.value.code == wfft.EINVAL
    ex.close()
    imp = wfft.Solver.from_problem(prob)
    with pytest.raises(wfft.WfftError) as e:
        imp.explicit_step([0.0, 0.0, 0.0])
    assert e.value.code == wfft.EINVAL
    imp.close()
    with pytest.raises(wfft.WfftError) as e:
        wfft.Solver(prob.ndim, prob.n, prob.h, prob.C, prob.rho, prob.phase, prob.mask, prob.dt, beta=0.0,
                    gamma=0.5, options=wfft.default_options(precision=wfft.MIXED))
    assert e.value.code == wfft.EINVAL
