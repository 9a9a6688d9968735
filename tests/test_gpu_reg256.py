"""GPU parity of the register-stage passes over 256-point axes (two radix-16 stages held
in registers, FP32, 3-D grids) through the C ABI: the column passes (plain y transforms,
fused gradient / divergence / preconditioner z passes) and the x passes (middle pass,
operator epilogue, preconditioner epilogue with the search direction, residual update):
the operator A and the preconditioner M against the FP64 oracle (Eq. Fourier_ND_A,
Eq. precond), mixed Newmark step sequences against the same sequences on the general
kernels, and the refusal of the plan codes where the kernels do not apply.  Every
column-tile width (4, 8, 16 kx columns) is covered, with ragged kx tails (N1/2 + 1 = 11
columns), and x tiles of 4 and 10 lines with a ragged last tile."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

REG = 256  # register-stage column-tile code flag (kColReg)
XREG = 1 << 16  # register-stage x-pass flag of the x tile size (kXReg)
CODES = [REG | 4, REG | 8, REG | 16]
N = (20, 256, 256)


def _solver(prob, precision=1, **kw):
    wfft = solver_lib()
    return wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=1e-10, **kw))


def _use_reg(s, code, precision=1):
    plan = s.get_plan(precision)
    plan["bx"][1][0] = plan["bx"][1][1] = code      # plain y passes
    plan["bx"][2][2] = plan["bx"][2][3] = plan["bx"][2][4] = code  # gradient, divergence, preconditioner (z)
    s.set_plan(precision, plan)
    got = s.get_plan(precision)["bx"]
    assert got[1][:2] == [code, code] and got[2][2:] == [code, code, code]


@pytest.fixture(scope="module")
def case():
    from oracle import medium, spectral
    rng = np.random.default_rng(256)
    prob = inputs.random_problem(rng, 3, N, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    med = medium.medium_from_problem(prob)
    sp = spectral.Spectral(med)
    th = prob.beta * prob.dt ** 2
    p = rng.standard_normal((3, N[2], N[1], N[0]))
    mask = oracle_field(prob, prob.mask).astype(bool)
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    zo = np.where(mask, 0.0, spectral.apply_M(med, sp, oracle_field(prob, p), th))
    return prob, p, qo, zo, mask


@pytest.mark.parametrize("code", CODES)
def test_operator_and_preconditioner_match_oracle(case, code):
    torch = torch_cuda()
    prob, p, qo, zo, mask = case
    s = _solver(prob)
    _use_reg(s, code)
    pd = to_dev(torch, p, torch.float32)
    qd = torch.zeros_like(pd)
    s.apply(pd, qd, precision=1, masked=False)
    zd = torch.zeros_like(pd)
    s.precond(pd, zd, precision=1, masked=True)
    qm = torch.zeros_like(pd)
    s.apply(pd, qm, precision=1, masked=True)
    torch.cuda.synchronize()
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < 3e-6
    assert rel(oracle_field(prob, qm.cpu().numpy().astype(np.float64)), np.where(mask, 0.0, qo)) < 3e-6
    assert rel(oracle_field(prob, zd.cpu().numpy().astype(np.float64)), zo) < 3e-6


def test_mixed_steps_same_as_general_kernels():
    """The preconditioner pass also forms the Parseval sum (r, z) that sets the Krylov
    beta: a wrong sum changes the iteration counts.  Steps on the register-stage kernels
    take the general kernels' iteration counts (within one) and solution (both solves
    within tol 1e-10 of the same discrete equation)."""
    torch_cuda()
    rng = np.random.default_rng(257)
    prob = inputs.random_problem(rng, 3, (16, 256, 256), nphase=4, mask_width=2, nsteps=4, contrast=4.0,
                                 dt=4e-7)
    runs = []
    for code in (None, REG | 8):
        s = _solver(prob)
        if code:
            _use_reg(s, code)
        infos = [s.step(prob.U[n]) for n in range(prob.nsteps)]
        u, _, _, _ = s.get_state()
        runs.append((np.asarray(u), infos))
    (u0, i0), (u1, i1) = runs
    assert rel(u1, u0) < 1e-7
    for a, b in zip(i0, i1):
        assert b["rel_res"] <= 1e-10
        assert abs(a["iters"] - b["iters"]) <= 1


def test_register_codes_refused_where_they_do_not_apply():
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(258)
    # a 128-point axis
    prob = inputs.random_problem(rng, 3, (16, 128, 64), nphase=2, mask_width=1)
    s = _solver(prob)
    plan = s.get_plan(1)
    plan["bx"][2][4] = REG | 8
    with pytest.raises(wfft.WfftError):
        s.set_plan(1, plan)
    # FP64 plans, and widths other than 4, 8, 16
    prob = inputs.random_problem(rng, 3, (16, 256, 256), nphase=2, mask_width=1)
    s = _solver(prob)
    plan = s.get_plan(0)
    plan["bx"][2][4] = REG | 8
    with pytest.raises(wfft.WfftError):
        s.set_plan(0, plan)
    plan = s.get_plan(1)
    plan["bx"][2][4] = REG | 2
    with pytest.raises(wfft.WfftError):
        s.set_plan(1, plan)
    plan["bx"][2][4] = REG | 16
    s.set_plan(1, plan)


XCASES = [((256, 22, 17), 4096), ((256, 22, 17), 2048), ((256, 256, 12), 4096)]


@pytest.mark.parametrize("n,xe", XCASES)
def test_register_x_passes_operator_matches_oracle(n, xe):
    from oracle import medium, spectral
    torch = torch_cuda()
    rng = np.random.default_rng(259 + xe + n[1])
    prob = inputs.random_problem(rng, 3, n, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    med = medium.medium_from_problem(prob)
    sp = spectral.Spectral(med)
    th = prob.beta * prob.dt ** 2
    s = _solver(prob)
    plan = s.get_plan(1)
    plan["xelems"] = XREG | xe
    if n[1] == 256:
        plan["bx"][1][0] = plan["bx"][1][1] = REG | 16
    s.set_plan(1, plan)
    assert s.get_plan(1)["xelems"] == XREG | xe
    p = rng.standard_normal((3, n[2], n[1], n[0]))
    mask = oracle_field(prob, prob.mask).astype(bool)
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    pd = to_dev(torch, p, torch.float32)
    for masked in (False, True):
        qd = torch.zeros_like(pd)
        s.apply(pd, qd, precision=1, masked=masked)
        torch.cuda.synchronize()
        ref = np.where(mask, 0.0, qo) if masked else qo
        assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), ref) < 3e-6


@pytest.mark.parametrize("n,xe", XCASES[:2])
def test_register_x_passes_mixed_steps_same_as_general_kernels(n, xe):
    """Inside the Krylov loop the register x passes form r -= alpha q with ||r||^2, the
    operator product with (p, q), and z = P(t), p = z + beta p with the half spectrum of
    p: a wrong dot or search direction changes the iteration counts."""
    torch_cuda()
    rng = np.random.default_rng(260 + xe)
    prob = inputs.random_problem(rng, 3, n, nphase=4, mask_width=2, nsteps=5, contrast=4.0, dt=4e-7)
    runs = []
    for flag in (0, XREG):
        s = _solver(prob)
        plan = s.get_plan(1)
        plan["xelems"] = flag | xe
        s.set_plan(1, plan)
        infos = [s.step(prob.U[k]) for k in range(prob.nsteps)]
        u, _, _, _ = s.get_state()
        runs.append((np.asarray(u), infos))
    (u0, i0), (u1, i1) = runs
    assert rel(u1, u0) < 1e-7
    for a, b in zip(i0, i1):
        assert b["rel_res"] <= 1e-10
        assert abs(a["iters"] - b["iters"]) <= 1


def test_register_x_flag_refused_where_it_does_not_apply():
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(261)
    prob = inputs.random_problem(rng, 3, (128, 20, 16), nphase=2, mask_width=1)
    s = _solver(prob)
    plan = s.get_plan(1)
    plan["xelems"] = XREG | 4096
    with pytest.raises(wfft.WfftError):
        s.set_plan(1, plan)  # 128-point rows
    prob = inputs.random_problem(rng, 3, (256, 20, 16), nphase=2, mask_width=1)
    s = _solver(prob)
    plan = s.get_plan(0)
    plan["xelems"] = XREG | 4096
    with pytest.raises(wfft.WfftError):
        s.set_plan(0, plan)  # FP64 plan
    prob = inputs.random_problem(rng, 2, (256, 64, 1), nphase=2, mask_width=1)
    s = _solver(prob)
    plan = s.get_plan(1)
    plan["xelems"] = XREG | 4096
    with pytest.raises(wfft.WfftError):
        s.set_plan(1, plan)  # 2-D grid
