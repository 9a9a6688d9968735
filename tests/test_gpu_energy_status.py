"""Energy of the committed state in the step record, and the NaN / Inf status.

E_n = 1/2 sum rho |v_n|^2 + 1/2 sum eps_n : C : eps_n is the energy of the Newmark energy
identity (Eq. Newmark with beta = 1/4, gamma = 1/2; the oracle pins the identity).  The
library forms it from the corrector's sums and the reaction; here it must equal the oracle's
spectral energy of the very state the GPU committed.  A state or a prescribed value holding a
NaN must end the step with WFFT_ENUMERIC and leave the state unchanged."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _oracle_energy(nm, prob, u, v, a):
    from oracle import newmark
    return nm.energy(newmark.State(oracle_field(prob, u), oracle_field(prob, v), oracle_field(prob, a)))


@pytest.mark.parametrize("ndim,n,precision,tol,bar", [(3, (16, 12, 10), 0, 1e-13, 1e-10),
                                                      (2, (40, 32, 1), 0, 1e-13, 1e-10),
                                                      (3, (20, 16, 12), 1, 1e-10, 1e-7)])
def test_step_energy_equals_oracle_energy_of_the_committed_state(ndim, n, precision, tol, bar):
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(300 + sum(n))
    prob = inputs.random_problem(rng, ndim, n, nphase=3, mask_width=2, nsteps=6, contrast=3.0, dt=4e-7)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=tol))
    nm = newmark.oracle_from_problem(prob)
    energies = []
    for k in range(prob.nsteps):
        info = s.step(prob.U[k])
        u, v, a, _ = s.get_state()
        e_o = _oracle_energy(nm, prob, u, v, a)
        assert e_o > 0
        assert abs(info["energy"] - e_o) <= bar * e_o, (k, info["energy"], e_o)
        energies.append(info["energy"])
    assert energies[-1] > energies[0]  # the prescribed region does work on the medium


def test_explicit_and_batch_steps_report_the_same_energy():
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(41)
    prob = inputs.random_problem(rng, 3, (16, 12, 8), nphase=3, mask_width=2, nsteps=4, contrast=3.0, dt=4e-7)
    nm = newmark.oracle_from_problem(prob)
    # grouped steps: each instance's energy equals its single-handle step's
    opt = wfft.default_options(tol=1e-12)
    a = wfft.Solver.from_problem(prob, options=opt)
    b = wfft.Solver.from_problem(prob, options=opt)
    for k in range(3):
        ia = a.step(prob.U[k])
        rc, infos = wfft.batch_step([b], prob.U[k:k + 1])
        assert rc == wfft.OK
        ib = infos[0]
        assert abs(ia["energy"] - ib["energy"]) <= 1e-12 * abs(ia["energy"])
    # explicit central differences (beta = 0): strain part from K u_n itself
    dt = 0.5 * wfft.explicit_dt(3, prob.h, prob.C, prob.rho)
    e = wfft.Solver(3, prob.n, prob.h, prob.C, prob.rho, prob.phase, prob.mask, dt, beta=0.0, gamma=0.5)
    rng2 = np.random.default_rng(42)
    u0 = 1e-7 * rng2.standard_normal((3, prob.n[2], prob.n[1], prob.n[0]))
    e.set_state(u0, None, None, 0)
    for k in range(3):
        info = e.explicit_step(np.zeros(3))
        u, v, acc, _ = e.get_state()
        e_o = _oracle_energy(nm, prob, u, v, acc)
        assert abs(info["energy"] - e_o) <= 1e-11 * e_o, (k, info["energy"], e_o)


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_state_or_load_returns_enumeric_and_keeps_the_state(precision):
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(43)
    prob = inputs.random_problem(rng, 3, (12, 10, 8), nphase=3, mask_width=2, nsteps=3, contrast=3.0)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=1e-10))
    s.step(prob.U[0])
    u, v, a, n = s.get_state()
    v_bad = v.copy()
    v_bad.reshape(-1)[v.size // 2 + 7] = np.nan  # a free DOF of the state
    s.set_state(u, v_bad, a, n)
    before = s.get_state()
    info = s.step(prob.U[1], raise_on_error=False)
    assert info["rc"] == wfft.ENUMERIC
    after = s.get_state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y, equal_nan=True)
    assert after[3] == before[3]
    # a finite state with a NaN prescribed value
    s.set_state(u, v, a, n)
    info = s.step(np.array([np.nan, 0.0, 0.0]), raise_on_error=False)
    assert info["rc"] == wfft.ENUMERIC
    for x, y in zip((u, v, a), s.get_state()[:3]):
        assert np.array_equal(x, y)
    # the handle still steps normally afterwards
    info = s.step(prob.U[1])
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
