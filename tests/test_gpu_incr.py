"""Incremental residual of the mixed solve (wfft_options.incr_resid).

The residual after a sweep that started from a full FP64 evaluation may be formed as
b - (A x + xc A d), A d the FP32 product of the correction, when the rounding
estimate kIncrC u32 lam_max ||xc d|| is below a quarter of the target.  These tests pin the
rounding constant (the FP32 operator's error against the FP64 one, relative to
u32 lam_max ||d||, on white noise and smooth fields, 2-D / 3-D, phase and per-voxel
tables, radix-16 plans), check that every step certified this way satisfies the TRUE
FP64 residual bound ||P(b - A u_n)|| <= tol ref, and that the results equal the solve
with full FP64 residuals and the oracle."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KINCR = 8.0         # the library's rounding constant (kIncrC)
U32 = 2.0 ** -24


def _pulse_problem(n, seed, nsteps, width=10.0, ngrains=None):
    """Rotated-cubic nickel polycrystal with a Gaussian pulse on the 4-voxel x-face slab."""
    ids, Cv, rho = inputs.polycrystal(n, ngrains or max(8, n[0] * n[1] * n[2] // 2000), seed)
    dt = 2e-7
    U = inputs._U_series(nsteps, dt, lambda t: inputs.gaussian_pulse(t, 1e-6, width * dt, 3 * width * dt))
    return inputs.Problem(f"pulse{n}_{seed}", 3, n, (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                          inputs.slab_mask(3, n, 4), U, tol=1e-10)


def _case(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "poly":
        return _pulse_problem((48, 40, 36), seed, 1)
    if kind == "poly16":
        return _pulse_problem((64, 32, 32), seed, 1)
    if kind == "random":
        return inputs.random_problem(rng, 3, (30, 28, 20), nphase=4, mask_width=2, contrast=4.0, dt=4e-7)
    if kind == "dense":
        return inputs.random_problem(rng, 3, (24, 20, 18), nphase=4, mask_width=2, dense=True, contrast=4.0,
                                     dt=4e-7)
    return inputs.random_problem(rng, 2, (96, 80, 1), nphase=4, mask_width=2, contrast=4.0, dt=4e-7)


def _field(rng, shape, kind):
    d = rng.standard_normal(shape)
    if kind == "smooth":  # Gaussian low-pass: the spectrum of a displacement correction
        axes = tuple(range(1, len(shape)))
        k2 = sum(np.meshgrid(*[np.fft.fftfreq(shape[a]) ** 2 for a in axes], indexing="ij"))
        d = np.real(np.fft.ifftn(np.fft.fftn(d, axes=axes) * np.exp(-k2 / (2 * 0.05 ** 2)), axes=axes))
    return d.astype(np.float32)


@pytest.mark.parametrize("kind", ["poly", "poly16", "random", "dense", "plane"])
@pytest.mark.parametrize("field", ["white", "smooth"])
def test_fp32_operator_rounding_within_the_incremental_bound(kind, field):
    torch = torch_cuda()
    wfft = solver_lib()
    prob = _case(kind, 41)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=wfft.MIXED))
    if kind == "poly16":
        for axis, cnt in enumerate(([0, 1, 0, 0, 0, 0, 1], [0, 0, 1, 0, 0, 0, 1], [0, 0, 1, 0, 0, 0, 1])):
            s.set_radix(wfft.MIXED, axis, cnt)
    lam = wfft.operator_bound(prob.ndim, prob.n, prob.h, prob.C, prob.rho, prob.beta * prob.dt ** 2)
    rng = np.random.default_rng(7)
    shape = (prob.ndim, prob.n[2], prob.n[1], prob.n[0])
    d = _field(rng, shape, field)
    d32 = to_dev(torch, d, torch.float32)
    d64 = to_dev(torch, d.astype(np.float64), torch.float64)
    q32, q64 = torch.zeros_like(d32), torch.zeros_like(d64)
    s.apply(d32, q32, precision=wfft.MIXED, masked=False)
    s.apply(d64, q64, precision=wfft.FP64, masked=False)
    torch.cuda.synchronize()
    err = np.linalg.norm(q32.cpu().numpy().astype(np.float64) - q64.cpu().numpy())
    ratio = err / (U32 * lam * np.linalg.norm(d.astype(np.float64)))
    print(kind, field, ratio)
    s.close()
    assert ratio <= KINCR / 4, ratio


def _run_checked(wfft, torch, prob, incr, tol=1e-10):
    """Steps prob with the mixed solve; after each step, the true FP64 residual of the
    committed displacement, ||P(b - A u_n)|| with b = rho (u + dt v + dt^2 (1/2 - beta) a)."""
    opts = wfft.default_options(precision=wfft.MIXED, tol=tol, incr_resid=incr)
    s = wfft.Solver.from_problem(prob, options=opts)
    rho = prob.rho_field()[None]
    gamma_dofs = prob.mask.astype(bool)
    infos, true_rel = [], []
    for k in range(prob.nsteps):
        u, v, a, _ = s.get_state()
        b = rho * (u + prob.dt * v + prob.dt ** 2 * (0.5 - prob.beta) * a)
        info = s.step(prob.U[k])
        un = s.get_state()[0]
        q = torch.zeros(un.shape, dtype=torch.float64, device="cuda")
        s.apply(to_dev(torch, un, torch.float64), q, precision=wfft.FP64, masked=False)
        torch.cuda.synchronize()
        r = b - q.cpu().numpy()
        r[gamma_dofs] = 0.0
        infos.append(info)
        true_rel.append(np.linalg.norm(r) / info["ref"])
    u = s.get_state()[0]
    s.close()
    return u, infos, true_rel


def test_incremental_residual_certifies_the_true_fp64_residual():
    from oracle import newmark
    torch = torch_cuda()
    wfft = solver_lib()
    prob = _pulse_problem((40, 40, 40), 12, 14, width=6.0)
    u_i, inf_i, tr_i = _run_checked(wfft, torch, prob, 1)
    u_f, inf_f, tr_f = _run_checked(wfft, torch, prob, 0)
    print([i["incr_resids"] for i in inf_i], [i["outer_applies"] for i in inf_i], max(tr_i))
    assert all(i["status"] == 0 for i in inf_i + inf_f)
    # every committed step meets ||P(b - A u_n)|| <= tol ref in FP64, either way
    assert max(tr_i) <= prob.tol * (1 + 1e-6), max(tr_i)
    assert max(tr_f) <= prob.tol * (1 + 1e-6), max(tr_f)
    # the reported residual is the evaluated one: within the bound of the true one
    for i, t in zip(inf_i, tr_i):
        assert abs(i["rel_res"] - t) <= 0.25 * prob.tol, (i["rel_res"], t)
    # the incremental form engages and saves FP64 applications
    assert sum(i["incr_resids"] for i in inf_i) >= prob.nsteps // 2
    assert sum(i["outer_applies"] for i in inf_i) < sum(i["outer_applies"] for i in inf_f)
    assert all(i["incr_resids"] == 0 for i in inf_f)
    assert rel(u_i, u_f) < 1e-8
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    assert rel(oracle_field(prob, u_i), so.u) < 1e-6


def test_tight_tolerance_still_meets_the_true_residual():
    """At tol 1e-12 the bound rejects the incremental form where the correction is still
    large and accepts it only for the last, small correction: every committed step meets
    the true FP64 residual bound."""
    torch = torch_cuda()
    wfft = solver_lib()
    prob = _pulse_problem((32, 32, 32), 5, 4, width=4.0)
    u, infos, tr = _run_checked(wfft, torch, prob, 1, tol=1e-12)
    print([i["incr_resids"] for i in infos], [i["outer_applies"] for i in infos], max(tr))
    assert all(i["status"] == 0 for i in infos)
    assert max(tr) <= 1e-12 * (1 + 1e-3), max(tr)


@pytest.mark.parametrize("warm", ["taylor", "learned"])
def test_incremental_residual_with_increment_warm_starts(warm):
    """With the Taylor or a learned increment as the first inner solve's initial guess
    (stored A u, FP32 residual of the increment), every step certified with an incremental
    last residual still meets the true FP64 residual bound."""
    torch = torch_cuda()
    wfft = solver_lib()
    prob = _pulse_problem((32, 32, 32), 17, 8, width=5.0)
    opts = wfft.default_options(precision=wfft.MIXED, tol=1e-10,
                                warm_start=wfft.WARM_TAYLOR if warm == "taylor" else wfft.WARM_LEARNED)
    s = wfft.Solver.from_problem(prob, options=opts)
    if warm == "learned":
        rng = np.random.default_rng(3)
        _, params = wfft.blob_params(wfft.model_init(16, 5))
        W4 = 0.3 * rng.standard_normal(params[3][0].shape) / np.sqrt(27 * 16)
        params[3] = (W4.astype(np.float32), params[3][1])
        s.set_model(wfft.params_blob(16, params))
    rho = prob.rho_field()[None]
    gamma_dofs = prob.mask.astype(bool)
    n_incr, worst = 0, 0.0
    for k in range(prob.nsteps):
        u, v, a, _ = s.get_state()
        b = rho * (u + prob.dt * v + prob.dt ** 2 * (0.5 - prob.beta) * a)
        info = s.step(prob.U[k])
        q = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
        s.apply(to_dev(torch, s.get_state()[0], torch.float64), q, precision=wfft.FP64, masked=False)
        torch.cuda.synchronize()
        r = b - q.cpu().numpy()
        r[gamma_dofs] = 0.0
        worst = max(worst, np.linalg.norm(r) / info["ref"])
        n_incr += info["incr_resids"]
    s.close()
    assert n_incr >= prob.nsteps // 2
    assert worst <= prob.tol * (1 + 1e-6), worst


def test_incremental_residual_plane_strain_matches_oracle():
    from oracle import newmark
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(23)
    prob = inputs.random_problem(rng, 2, (96, 64, 1), nphase=4, mask_width=3, nsteps=6, contrast=3.0)
    prob.U[:, 0] = 1e-6 * np.sin(np.linspace(0.3, 1.5, 6))
    u_i, inf_i, tr_i = _run_checked(wfft, torch, prob, 1, tol=1e-10)
    assert all(i["status"] == 0 for i in inf_i)
    assert max(tr_i) <= 1e-10 * (1 + 1e-6)
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    assert rel(oracle_field(prob, u_i), so.u) < 1e-6
