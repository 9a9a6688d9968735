"""Axes with a prime factor above 7: the paper's odd grids (Sec. 4.1: 129 = 3 x 43 voxels
per edge for the spherical waves, 1025 = 5^2 x 41 for the circular-wave plates) and
others (11, 13, 127, 176 = 16 x 11), taken by the direct prime-length DFT stage ahead of
the radix stages.  The batched real FFT is checked against the DFT definition (numpy),
and the operator A and the preconditioner M against the FP64 oracle, with the prime
axis in the x passes and in the column passes.  The paper's 129^3 aluminium cube takes
Newmark steps whose displacements must satisfy the oracle's discrete equation (Eq.
Fourier_ND_A, Eq. Fourier_ND_b) and keep the mirror symmetries of the problem."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# (ndim, (N1, N2, N3)): prime factors above 7 on x (x passes) and on y, z (column passes)
PRIME_SHAPES = [(3, (22, 13, 3)), (3, (43, 4, 3)), (3, (6, 41, 4)), (3, (4, 3, 129)), (3, (129, 6, 2)),
                (3, (127, 2, 3)), (3, (176, 3, 2)), (2, (1025, 4, 1)), (2, (6, 1025, 1)), (2, (82, 26, 1))]


def _solver(prob, precision=0):
    wfft = solver_lib()
    return wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=1e-12))


@pytest.mark.parametrize("ndim,n", PRIME_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_prime_axis_rfft3_matches_dft_definition(ndim, n, prec):
    torch = torch_cuda()
    rng = np.random.default_rng(sum(n) + 5 * prec)
    prob = inputs.random_problem(rng, ndim, n, nphase=2, mask_width=0)
    s = _solver(prob, prec)
    pitch = s.spectral_pitch()
    nc = 2 if ndim == 2 else 3
    f = rng.standard_normal((nc, n[2], n[1], n[0]))
    dt = torch.float64 if prec == 0 else torch.float32
    fin = to_dev(torch, f, dt)
    spec = torch.zeros((nc, n[2], n[1], pitch, 2), dtype=dt, device="cuda")
    s.rfft3(fin, spec, precision=prec, direction=-1, ncomp=nc)
    torch.cuda.synchronize()
    got = spec.cpu().numpy().astype(np.float64)
    got = (got[..., 0] + 1j * got[..., 1])[..., : n[0] // 2 + 1]
    ref = np.fft.rfftn(f, axes=(1, 2, 3))
    tol = 1e-13 if prec == 0 else 3e-6
    assert rel(got, ref) < tol
    back = torch.zeros_like(fin)
    s.rfft3(spec, back, precision=prec, direction=+1, ncomp=nc)
    torch.cuda.synchronize()
    assert rel(back.cpu().numpy() / (n[0] * n[1] * n[2]), f) < tol
    s.close()


@pytest.mark.parametrize("ndim,n", PRIME_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_prime_axis_operator_and_preconditioner_match_oracle(ndim, n, prec):
    from oracle import medium, spectral
    torch = torch_cuda()
    rng = np.random.default_rng(13 * sum(n) + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    s = _solver(prob, prec)
    med = medium.medium_from_problem(prob)
    sp = spectral.Spectral(med)
    th = prob.beta * prob.dt ** 2
    dt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 3e-6
    free = ~oracle_field(prob, prob.mask).astype(bool)
    p = rng.standard_normal((ndim, n[2], n[1], n[0]))
    qd = torch.zeros((ndim, n[2], n[1], n[0]), dtype=dt, device="cuda")
    s.apply(to_dev(torch, p, dt), qd, precision=prec, masked=True)
    zd = torch.zeros_like(qd)
    s.precond(to_dev(torch, p, dt), zd, precision=prec, masked=True)
    torch.cuda.synchronize()
    qo = np.where(free, spectral.apply_A(med, sp, oracle_field(prob, p), th), 0.0)
    zo = np.where(free, spectral.apply_M(med, sp, oracle_field(prob, p), th), 0.0)
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < tol
    assert rel(oracle_field(prob, zd.cpu().numpy().astype(np.float64)), zo) < tol
    s.close()


def test_hand_set_radix16_with_prime_stage_matches_oracle():
    """176 = 16 x 11 on x and 208 = 16 x 13 on y with a radix-16 stage set by hand (FP32
    plans): the prime stage runs ahead of it; the operator stays the oracle's."""
    from oracle import medium, spectral
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(176)
    n = (176, 208, 2)
    prob = inputs.random_problem(rng, 3, n, nphase=3, mask_width=2, contrast=3.0, dt=4e-7)
    s = _solver(prob, wfft.MIXED)
    s.set_radix(wfft.MIXED, 0, [0, 0, 0, 0, 0, 0, 1])
    s.set_radix(wfft.MIXED, 1, [0, 0, 0, 0, 0, 0, 1])
    plan = s.get_plan(wfft.MIXED)
    assert plan["radix"][0][6] == 1 and plan["radix"][1][6] == 1
    with pytest.raises(wfft.WfftError) as e:
        s.set_radix(wfft.MIXED, 0, [0, 0, 0, 0, 0, 0, 2])  # 256 != 176 / 11
    assert e.value.code == wfft.EINVAL
    med = medium.medium_from_problem(prob)
    sp = spectral.Spectral(med)
    th = prob.beta * prob.dt ** 2
    free = ~oracle_field(prob, prob.mask).astype(bool)
    p = rng.standard_normal((3, n[2], n[1], n[0]))
    qd = torch.zeros((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    s.apply(to_dev(torch, p, torch.float32), qd, precision=wfft.MIXED, masked=True)
    torch.cuda.synchronize()
    qo = np.where(free, spectral.apply_A(med, sp, oracle_field(prob, p), th), 0.0)
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < 3e-6
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spherical_wave_129_steps_satisfy_the_oracle_equation(precision):
    """The 129^3 aluminium cube of Sec. 4.1 under the central u_1 pulse: every checked
    step's displacement satisfies ||P(b - A u_n)|| <= tol ref with b and A the oracle's,
    and u_1 is even under the mirror x_2 -> -x_2 (the medium is homogeneous and isotropic
    and the prescribed region and pulse are mirror-symmetric about the centre)."""
    from oracle import newmark, spectral
    from oracle.medium import field_to_oracle
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_sphere129(nsteps=4)
    prec = wfft.FP64 if precision == "fp64" else wfft.MIXED
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=prec, tol=1e-10, maxit=400))
    nm = newmark.oracle_from_problem(prob, tol=1e-10)
    worst = 0.0
    for k in range(prob.nsteps):
        check = k in (1, prob.nsteps - 1)
        if check:
            u, v, a, _ = s.get_state()
        info = s.step(prob.U[k])
        assert info["status"] == 0
        if not check:
            continue
        un = s.get_state()[0]
        b = spectral.rhs_b(nm.med, field_to_oracle(prob, u), field_to_oracle(prob, v), field_to_oracle(prob, a),
                           prob.dt, prob.beta)
        r = np.where(nm.mask, 0.0, b - nm.A(field_to_oracle(prob, un)))
        worst = max(worst, np.linalg.norm(r) / info["ref"])
        # prescribed voxels carry U(t_n) on u_1 and zero on u_2, u_3
        m = prob.mask[0].astype(bool)
        assert np.abs(un[0][m] - prob.U[k, 0]).max() <= 1e-12 * abs(prob.U[k, 0])
        assert np.all(un[1][m] == 0) and np.all(un[2][m] == 0)
        # mirror x_2 -> -x_2 about the centre voxel (index 64 of 129): u_1 even
        u1 = un[0]
        assert rel(u1[:, ::-1, :], u1) < 1e-8
        assert np.abs(u1).max() > 0
    s.close()
    assert worst <= 1e-10 * (1 + 1e-2), worst
