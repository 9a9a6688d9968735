"""3-D grids with a single voxel along x_1 (N1 = 1): the paper's circular waves in a plate,
1 x 1025 x 1025 voxels of 0.001 x 1 x 1 m (Sec. 4.1), homogeneous aluminium and aluminium in
an iron frame, loaded perpendicular to the plate at its centre.

The library runs such a grid on the cyclically relabeled axes (x_2, x_3, x_1) and maps the
displacement components back; every field the caller sees keeps the caller's [c][N3][N2][N1]
layout.  The oracle runs the grid as given (its transforms include the length-1 axis), so
equality with it checks the relabeling of the stiffness, the components, the prescribed
DOFs, the prescribed values and the reactions."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _random_plate(rng, n2, n3, nsteps):
    """1 x n2 x n3 plate of four random anisotropic phases (rotated cubic), prescribed on
    the two voxel rows x_2 < 2 (all components), load on u_1 and u_2."""
    ids = rng.integers(0, 4, size=(n3, n2, 1)).astype(np.uint16)
    Rs = inputs.random_rotations(rng, 4)
    base = inputs.cubic_voigt(168.4e9, 121.4e9, 75.4e9)
    C = np.stack([inputs.voigt21_from_matrix(inputs.rotate_voigt(base, R)) for R in Rs])
    rho = 8960.0 * (1.0 + 0.5 * rng.random(4))
    mask = np.zeros((3, n3, n2, 1), np.uint8)
    mask[:, :, :2, 0] = 1
    U = np.zeros((nsteps, 3))
    U[:, 0] = 1e-6 * np.sin(np.linspace(0.2, 1.0, nsteps))
    U[:, 1] = -4e-7 * np.sin(np.linspace(0.1, 0.7, nsteps))
    return inputs.Problem("plate_random", 3, (1, n2, n3), (1e-3, 1.2e-3, 0.9e-3), 4e-7, 0.25, 0.5, C, rho, ids,
                          mask, U, tol=1e-13)


@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-13, 1e-10), (1, 1e-10, 1e-6)])
def test_random_plate_with_one_voxel_along_x1_matches_the_oracle(precision, tol, bar):
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = _random_plate(np.random.default_rng(71), 40, 36, 4)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=tol))
    assert s.shape == (3, 36, 40, 1)
    nm = newmark.oracle_from_problem(prob, tol=1e-13)
    st = nm.zero_state()
    for k in range(prob.nsteps):
        info = s.step(prob.U[k])
        st, io = nm.step(st, prob.U[k])
        assert np.allclose(info["reaction"], io["reaction"], rtol=1e-6, atol=1e-9 * abs(info["ref"]))
        assert abs(info["energy"] - nm.energy(st)) <= 1e-6 * nm.energy(st)
    u, v, a, n = s.get_state()
    assert rel(oracle_field(prob, u), st.u) < bar
    assert rel(oracle_field(prob, v), st.v) < 100 * bar
    # the caller's prescribed values sit on the caller's components
    m = prob.mask.astype(bool)
    for j in range(3):
        assert np.all(u[j][m[j]] == prob.U[-1, j])
    # device-state round trip keeps the caller's component order
    torch = torch_cuda()
    du = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    dv, da = torch.empty_like(du), torch.empty_like(du)
    s.get_state_dev(du, dv, da)
    assert np.array_equal(du.cpu().numpy(), u)
    s.set_state_dev(du, dv, da, n)
    assert all(np.array_equal(x, y) for x, y in zip(s.get_state()[:3], (u, v, a)))
    with pytest.raises(wfft.WfftError) as e:
        s.apply(du, dv)
    assert e.value.code == wfft.EUNSUPPORTED


@pytest.mark.parametrize("framed", [False, True])
def test_paper_plate_1x1025x1025_steps_match_the_oracle(framed):
    """The paper's plate (1025 = 5^2 x 41 on both in-plane axes: the direct 41-point stage),
    first three steps of the pulse, FP64 to 1e-12 on both sides."""
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.config_plate1025(nsteps=3, framed=framed)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-12, maxit=400))
    nm = newmark.oracle_from_problem(prob, tol=1e-12)
    st = nm.zero_state()
    for k in range(prob.nsteps):
        info = s.step(prob.U[k])
        st, io = nm.step(st, prob.U[k])
        assert abs(info["iters"] - io["iters"]) <= 1
    u = s.get_state()[0]
    assert rel(oracle_field(prob, u), st.u) < 1e-9
    # transverse load, in-plane components stay at rest (isotropic layers decouple u_1)
    assert np.abs(u[1:]).max() <= 1e-12 * np.abs(u[0]).max()
