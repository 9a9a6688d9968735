"""Long axes: every 7-smooth length up to 1050 points, with the limit set by the tiles
of the passes (each radix stage's per-thread register batch and the shared memory).
The batched real FFT is checked against the DFT definition (numpy), and the operator A
and the preconditioner M against the FP64 oracle, with the long axis in the x passes
and in the column passes.  The paper's polycrystalline bar (Sec. 4.3, 35 x 35 x 567
voxels) takes Newmark steps whose displacements must satisfy the oracle's discrete
equation (Eq. Fourier_ND_A, Eq. Fourier_ND_b).  Axes of 450-500 points with a radix-5
stage are included: their FP64 x tiles once held more butterflies than a stage
transforms."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# (ndim, (N1, N2, N3)): long x axes (x passes), long y and z axes (column passes)
LONG_SHAPES = [(3, (500, 4, 3)), (3, (480, 3, 2)), (3, (567, 5, 4)), (3, (5, 4, 567)), (3, (4, 729, 3)),
               (3, (1024, 3, 2)), (3, (3, 4, 1050)), (2, (1050, 6, 1)), (2, (6, 768, 1)), (2, (625, 4, 1))]


def _solver(prob, precision=0):
    wfft = solver_lib()
    return wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=1e-12))


@pytest.mark.parametrize("ndim,n", LONG_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_long_axis_rfft3_matches_dft_definition(ndim, n, prec):
    torch = torch_cuda()
    rng = np.random.default_rng(sum(n) + 7 * prec)
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


@pytest.mark.parametrize("ndim,n", LONG_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_long_axis_operator_and_preconditioner_match_oracle(ndim, n, prec):
    from oracle import medium, spectral
    torch = torch_cuda()
    rng = np.random.default_rng(11 * sum(n) + ndim)
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


def test_axes_beyond_the_tiles_are_refused():
    wfft = solver_lib()
    rng = np.random.default_rng(1)
    # 1536 on x: three line pairs exceed every stage's register batch; 1080 on y or z: the
    # FP64 six-slot column tile exceeds the shared memory (both 7-smooth)
    for n in [(1536, 2, 2), (4, 3, 1080), (4, 1080, 3)]:
        prob = inputs.random_problem(rng, 3, n, nphase=2, mask_width=1)
        with pytest.raises(wfft.WfftError) as e:
            wfft.Solver.from_problem(prob)
        assert e.value.code == wfft.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polycrystal_bar_steps_satisfy_the_oracle_equation(precision):
    """The 35 x 35 x 567 nickel bar under the long pulse: every checked step's displacement
    satisfies ||P(b - A u_n)|| <= tol ref with b and A the oracle's."""
    from oracle import newmark, spectral
    from oracle.medium import field_to_oracle
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_bar567(nsteps=8)
    prec = wfft.FP64 if precision == "fp64" else wfft.MIXED
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=prec, tol=1e-10, maxit=800))
    nm = newmark.oracle_from_problem(prob, tol=1e-10)
    worst = 0.0
    for k in range(prob.nsteps):
        check = k in (2, prob.nsteps - 1)
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
        # the prescribed plane carries U(t_n) on u_3 and zero on u_1, u_2
        assert np.abs(un[2, 0] - prob.U[k, 2]).max() <= 1e-12 * abs(prob.U[k, 2])
        assert np.all(un[:2, 0] == 0)
    s.close()
    assert worst <= 1e-10 * (1 + 1e-2), worst
