"""GPU parity of the building blocks through the C ABI: the batched real FFT
against the DFT definition (numpy), the operator A and the preconditioner M
against the FP64 oracle, in FP64 and FP32, on sizes that span several tiles
and ragged tails, every radix, 2-D and 3-D, table and per-voxel materials."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import abi_field, oracle_field, rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# (ndim, (N1, N2, N3)) -- radices 2, 3, 4, 5, 7, 8, odd and even lengths, singleton axes
FFT_SHAPES = [(3, (16, 12, 10)), (3, (64, 48, 40)), (3, (30, 20, 14)), (3, (7, 9, 5)), (2, (64, 64, 1)),
              (2, (80, 96, 1)), (3, (8, 1, 6)), (3, (8, 6, 1)), (3, (256, 16, 8)), (3, (6, 256, 4))]


def _solver(prob, precision=0):
    wfft = solver_lib()
    return wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=1e-12))


@pytest.mark.parametrize("ndim,n", FFT_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_rfft3_matches_dft_definition(ndim, n, prec):
    torch = torch_cuda()
    rng = np.random.default_rng(sum(n) + prec)
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
    got = got[..., 0] + 1j * got[..., 1]
    got = got[..., : n[0] // 2 + 1]
    ref = np.fft.rfftn(f, axes=(1, 2, 3))
    tol = 1e-13 if prec == 0 else 2e-6
    assert rel(got, ref) < tol
    # unnormalised inverse back to V f
    back = torch.zeros_like(fin)
    s.rfft3(spec, back, precision=prec, direction=+1, ncomp=nc)
    torch.cuda.synchronize()
    V = n[0] * n[1] * n[2]
    assert rel(back.cpu().numpy() / V, f) < tol


# N1 % 16 == 0 runs the FP32 x passes with staged elementwise inputs (phase ids, per-voxel
# densities, masks, operator input); other N1 read them directly
APPLY_CASES = [(2, (64, 64, 1), False), (2, (30, 28, 1), False), (3, (16, 12, 10), False),
               (3, (24, 20, 18), True), (3, (7, 9, 5), False), (3, (40, 36, 30), False), (3, (8, 1, 6), False),
               (3, (8, 6, 1), True), (3, (32, 20, 14), True), (2, (64, 40, 1), True), (3, (48, 18, 10), False)]


def _oracle_ops(prob):
    from oracle import medium, spectral
    med = medium.medium_from_problem(prob)
    sp = spectral.Spectral(med)
    th = prob.beta * prob.dt ** 2
    return med, sp, th


@pytest.mark.parametrize("ndim,n,dense", APPLY_CASES)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("masked", [False, True])
def test_operator_matches_oracle(ndim, n, dense, prec, masked):
    from oracle import spectral
    torch = torch_cuda()
    rng = np.random.default_rng(3 * sum(n) + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=2, dense=dense, contrast=4.0,
                                 dt=4e-7)
    s = _solver(prob, prec)
    med, sp, th = _oracle_ops(prob)
    p = rng.standard_normal((ndim, n[2], n[1], n[0]))
    dt = torch.float64 if prec == 0 else torch.float32
    pd = to_dev(torch, p, dt)
    qd = torch.zeros_like(pd)
    s.apply(pd, qd, precision=prec, masked=masked)
    torch.cuda.synchronize()
    q = qd.cpu().numpy().astype(np.float64)
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    if masked:
        qo = np.where(oracle_field(prob, prob.mask).astype(bool), 0.0, qo)
    tol = 1e-12 if prec == 0 else 3e-6
    assert rel(oracle_field(prob, q), qo) < tol


@pytest.mark.parametrize("ndim,n,dense", APPLY_CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_preconditioner_matches_oracle(ndim, n, dense, prec):
    from oracle import spectral
    torch = torch_cuda()
    rng = np.random.default_rng(5 * sum(n) + ndim)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=1, dense=dense, contrast=4.0)
    s = _solver(prob, prec)
    med, sp, th = _oracle_ops(prob)
    r = rng.standard_normal((ndim, n[2], n[1], n[0]))
    dt = torch.float64 if prec == 0 else torch.float32
    rd = to_dev(torch, r, dt)
    zd = torch.zeros_like(rd)
    s.precond(rd, zd, precision=prec, masked=True)
    torch.cuda.synchronize()
    zo = spectral.apply_M(med, sp, oracle_field(prob, r), th)
    zo = np.where(oracle_field(prob, prob.mask).astype(bool), 0.0, zo)
    tol = 1e-12 if prec == 0 else 3e-6
    assert rel(oracle_field(prob, zd.cpu().numpy().astype(np.float64)), zo) < tol


def test_preconditioner_inverts_homogeneous_operator_on_gpu():
    """M A = I for a homogeneous medium (Eq. A_oper_inv_homog generalised), FP64."""
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(9)
    n = (24, 20, 16)
    Cv = inputs.voigt21_from_matrix(inputs.rotate_voigt(inputs.cubic_voigt(*inputs.NI_CUBIC),
                                                        inputs.random_rotations(rng, 1)[0]))[None]
    s = wfft.Solver(3, n, (1e-3,) * 3, Cv, np.array([8960.0]), np.zeros((n[2], n[1], n[0]), np.uint16), None,
                    2e-7)
    u = to_dev(torch, rng.standard_normal((3, n[2], n[1], n[0])), torch.float64)
    q = torch.zeros_like(u)
    z = torch.zeros_like(u)
    s.apply(u, q)
    s.precond(q, z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), u.cpu().numpy()) < 1e-13


# hand-set radix schedules (wfft_set_radix): stages of radix 8, 4, 2, 3, 5, 7, 16
RADIX_CASES = [
    (3, (64, 32, 16), 1, [[0, 1, 0, 0, 0, 0, 1], [0, 0, 1, 0, 0, 0, 1], [0, 0, 0, 0, 0, 0, 1]]),
    (3, (64, 32, 16), 0, [[0, 3, 0, 0, 0, 0, 0], [0, 2, 1, 0, 0, 0, 0], [1, 0, 1, 0, 0, 0, 0]]),
    (2, (256, 48, 1), 1, [[0, 0, 0, 0, 0, 0, 2], [0, 0, 0, 1, 0, 0, 1], None]),
    (3, (256, 32, 48), 0, [[0, 0, 0, 0, 0, 0, 2], [0, 0, 1, 0, 0, 0, 1], [0, 0, 0, 1, 0, 0, 1]]),
    (2, (80, 64, 1), 0, [[0, 0, 0, 0, 1, 0, 1], [0, 1, 0, 0, 0, 0, 1], None]),
]


@pytest.mark.parametrize("ndim,n,prec,plans", RADIX_CASES)
def test_hand_set_radix_schedules_match_oracle(ndim, n, prec, plans):
    """Radix-16 stages and other decompositions than the built-in one give the
    same operator and preconditioner as the oracle, at the usual tolerances."""
    from oracle import spectral
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(7 * sum(n) + prec)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    s = _solver(prob, prec)
    for axis, cnt in enumerate(plans):
        if cnt is not None:
            s.set_radix(wfft.MIXED if prec else wfft.FP64, axis, cnt)
    med, sp, th = _oracle_ops(prob)
    dt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 3e-6
    p = rng.standard_normal((ndim, n[2], n[1], n[0]))
    pd = to_dev(torch, p, dt)
    qd = torch.zeros_like(pd)
    s.apply(pd, qd, precision=prec, masked=False)
    zd = torch.zeros_like(pd)
    s.precond(pd, zd, precision=prec, masked=False)
    torch.cuda.synchronize()
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    zo = spectral.apply_M(med, sp, oracle_field(prob, p), th)
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < tol
    assert rel(oracle_field(prob, zd.cpu().numpy().astype(np.float64)), zo) < tol
    with pytest.raises(wfft.WfftError):
        s.set_radix(wfft.FP64, 0, [0, 0, 0, 0, 0, 0, 9])


# x-pass tile sizes other than the default (wfft_plan_choice.xelems): more or fewer lines per block
XTILE_CASES = [(3, (64, 48, 40), 1, 4096), (3, (64, 48, 40), 1, 1024), (3, (30, 20, 14), 0, 1024),
               (3, (30, 20, 14), 1, 8192), (2, (80, 96, 1), 1, 4096), (3, (256, 12, 6), 0, 4096)]


@pytest.mark.parametrize("ndim,n,prec,xelems", XTILE_CASES)
def test_x_tile_sizes_match_oracle(ndim, n, prec, xelems):
    from oracle import spectral
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(11 * sum(n) + prec)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    s = _solver(prob, prec)
    pr = wfft.MIXED if prec else wfft.FP64
    plan = s.get_plan(pr)
    assert plan["xelems"] == 2048
    plan["xelems"] = xelems
    s.set_plan(pr, plan)
    assert s.get_plan(pr)["xelems"] == xelems
    med, sp, th = _oracle_ops(prob)
    dt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 3e-6
    p = rng.standard_normal((ndim, n[2], n[1], n[0]))
    pd = to_dev(torch, p, dt)
    qd, zd = torch.zeros_like(pd), torch.zeros_like(pd)
    s.apply(pd, qd, precision=prec, masked=False)
    s.precond(pd, zd, precision=prec, masked=False)
    torch.cuda.synchronize()
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    zo = spectral.apply_M(med, sp, oracle_field(prob, p), th)
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < tol
    assert rel(oracle_field(prob, zd.cpu().numpy().astype(np.float64)), zo) < tol
    plan["xelems"] = 100
    with pytest.raises(wfft.WfftError):
        s.set_plan(pr, plan)


@pytest.mark.parametrize("prec", [0, 1])
def test_wide_plain_column_tiles_match_oracle(prec):
    """Plain column passes 16 columns wide (FP32 only; FP64 refuses them) give the oracle's operator."""
    from oracle import spectral
    torch = torch_cuda()
    wfft = solver_lib()
    n = (64, 48, 20)
    rng = np.random.default_rng(77 + prec)
    prob = inputs.random_problem(rng, 3, n, nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    s = _solver(prob, prec)
    pr = wfft.MIXED if prec else wfft.FP64
    plan = s.get_plan(pr)
    plan["bx"][1][0] = plan["bx"][1][1] = 16
    if prec == 0:
        with pytest.raises(wfft.WfftError):
            s.set_plan(pr, plan)
        return
    s.set_plan(pr, plan)
    assert s.get_plan(pr)["bx"][1][:2] == [16, 16]
    med, sp, th = _oracle_ops(prob)
    p = rng.standard_normal((3, n[2], n[1], n[0]))
    pd = to_dev(torch, p, torch.float32)
    qd = torch.zeros_like(pd)
    s.apply(pd, qd, precision=prec, masked=False)
    torch.cuda.synchronize()
    qo = spectral.apply_A(med, sp, oracle_field(prob, p), th)
    assert rel(oracle_field(prob, qd.cpu().numpy().astype(np.float64)), qo) < 3e-6
