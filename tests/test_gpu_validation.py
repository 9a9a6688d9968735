"""The paper's validation workloads on the GPU (Sec. 3.1, Tables 2 and 3 and the order of
accuracy in time; Sec. 3.2, Table 4).

A 1-D bar is run as a 2-D plane-strain strip of N x 2 voxels loaded uniformly across
its width: for a y-uniform field the spectral y derivative is exactly zero, so with
nu = 0 (lambda = 0, C11 = E) the strip's discrete operator (Eq. Fourier_ND_A) is the
1-D bar's.  The paper's bar has N = 6561 voxels, longer than one block's transform; the
GPU runs odd N that fit (729 = 3^6 and 1025 = 5^2 x 41, the latter through the direct
prime-length stage) at the paper's own time increments, and its final field must equal
the 1-D oracle's at the same N, with the same d'Alembert error (Eq. normL2, App. C).
The oracle reproduces Table 2's printed errors at N = 6561 (the oracle pins), which ties
the GPU to the paper's numbers through this workload family.  Even N are not used: with
the Nyquist multiplier zero, a point source excites a mode without stiffness (the paper
runs odd N only, Sec. 3.4).  The plane P and S waves of Table 4 are run the same way
(an Al strip with nu = 0.345 at h = 1 mm): the pulse centroid must move at the analytic
c_L = 6395.5 m/s and c_S = 3111.1 m/s, at the speed the oracle gives on the same strip."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import solver_lib, torch_cuda

pytestmark = pytest.mark.gpu

AL_E, AL_RHO = 70.3e9, 2700.0


def _strip(N, L, E, nu, rho, dt, U):
    """N x 2 plane-strain strip of length L, voxel plane x_idx = 0 prescribed (both
    components), U = [nsteps, 3] prescribed displacement."""
    h = L / N
    C = inputs.voigt21_from_matrix(inputs.isotropic_voigt(E, nu))[None, :]
    phase = np.zeros((1, 2, N), np.uint16)
    mask = np.zeros((2, 1, 2, N), np.uint8)
    mask[:, :, :, 0] = 1
    return inputs.Problem(f"strip_{N}", 2, (N, 2, 1), (h, h, h), dt, 0.25, 0.5, C, np.array([rho]), phase, mask,
                          U, tol=1e-12)


def _bar_oracle(N, L, dt, U):
    """The 1-D bar of Table 2 on the FP64 oracle: final u."""
    from oracle import medium, newmark
    med = medium.Medium(1, (N,), (L,), np.full((1, 1, 1, 1, 1), AL_E), np.zeros(N, np.int64), np.full(N, AL_RHO))
    mask = np.zeros((1, N), bool)
    mask[0, 0] = True
    s, _ = newmark.NewmarkOracle(med, mask, dt, tol=1e-12).run(U)
    return s.u[0]


@pytest.mark.parametrize("N", [729, 1025])
@pytest.mark.parametrize("ratio", [5, 10])
def test_1d_aluminium_bar_on_gpu_equals_the_oracle_and_its_analytic_error(N, ratio):
    from oracle import analytic
    torch_cuda()
    wfft = solver_lib()
    L = 2.0
    c0 = np.sqrt(AL_E / AL_RHO)
    omega = 5 * np.pi * c0 / L
    Uf = lambda t: inputs.bell_pulse(t, 1e-3, omega, 4)
    dt = ratio * (L / 6561) / c0  # the paper's increment (Delta t / CFL at N = 6561)
    nsteps = int(round(3.919e-4 / dt))
    U = np.zeros((nsteps, 3))
    U[:, 0] = Uf(dt * np.arange(1, nsteps + 1))
    prob = _strip(N, L, AL_E, 0.0, AL_RHO, dt, U)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-12, maxit=400))
    for k in range(nsteps):
        info = s.step(U[k])
        assert info["status"] == 0
    u = s.get_state()[0]
    s.close()
    ux = u[0, 0]  # [N2][N1]
    assert np.abs(u[1]).max() <= 1e-12 * np.abs(ux).max()  # no transverse motion
    assert np.abs(ux[1] - ux[0]).max() <= 1e-12 * np.abs(ux).max()  # y-uniform
    uo = _bar_oracle(N, L, dt, U)
    assert np.linalg.norm(ux[0] - uo) / np.linalg.norm(uo) < 1e-9
    x = (np.arange(N) + 0.5) * (L / N)
    ua = analytic.dalembert_periodic(x, nsteps * dt, 0.0, c0, L, Uf)
    e_gpu = np.linalg.norm(ux[0] - ua) / np.linalg.norm(ua)
    e_orc = np.linalg.norm(uo - ua) / np.linalg.norm(ua)
    assert abs(e_gpu - e_orc) <= 1e-6 * e_orc
    assert e_gpu < 2e-2  # 1.6e-2 at N = 729: the source voxel is 9x the paper's


def test_order_of_accuracy_in_time_on_gpu():
    """Sec. 3.1, order of accuracy in time: the Table 2 bar as the N x 2 strip at N = 729, run
    to the same final time with Delta t = 4, 2, 1 x h / c0.  Each GPU run equals the oracle's
    bar at the same Delta t, and the differences of successive runs shrink by the factor 4
    of a second-order scheme (Richardson), as the oracle's do."""
    torch_cuda()
    wfft = solver_lib()
    N, L, T = 729, 2.0, 3.919e-4
    c0 = np.sqrt(AL_E / AL_RHO)
    Uf = lambda t: inputs.bell_pulse(t, 1e-3, 5 * np.pi * c0 / L, 4)  # noqa: E731
    runs = {}
    for r in (4.0, 2.0, 1.0):
        nsteps = int(round(T / (r * (L / N) / c0)))
        dt = T / nsteps
        U = np.zeros((nsteps, 3))
        U[:, 0] = Uf(dt * np.arange(1, nsteps + 1))
        s = wfft.Solver.from_problem(_strip(N, L, AL_E, 0.0, AL_RHO, dt, U),
                                     options=wfft.default_options(tol=1e-12, maxit=400))
        for k in range(nsteps):
            assert s.step(U[k])["status"] == 0
        ux = s.get_state()[0][0, 0, 0]
        s.close()
        uo = _bar_oracle(N, L, dt, U)
        assert np.linalg.norm(ux - uo) / np.linalg.norm(uo) < 1e-9, r
        runs[r] = ux
    ratio = np.linalg.norm(runs[4.0] - runs[2.0]) / np.linalg.norm(runs[2.0] - runs[1.0])
    print("Richardson ratio (Delta t = 4, 2, 1 h / c0):", ratio)
    assert 3.3 < ratio < 4.5, ratio


@pytest.mark.parametrize("comp", [0, 1])
def test_plane_wave_speeds_on_gpu_match_the_oracle_and_table_4(comp):
    """P (comp 0) and S (comp 1) plane waves at 10 CFL on a 1029 x 2 strip (h = 1 mm,
    1029 = 3 x 7^3, odd): the GPU's pulse-centroid speed equals the oracle's on the same
    strip, and both are within 2 % of the analytic speed (the 20-step pulse of this
    length has a larger Newmark dispersion than the paper's 2187-voxel run, whose
    speeds the oracle pins reproduce within 1 %)."""
    from oracle import analytic, newmark
    torch_cuda()
    wfft = solver_lib()
    nu = 0.345
    lam, mu = analytic.lame(AL_E, nu)
    cL, cS = analytic.isotropic_speeds(lam, mu, AL_RHO)
    assert abs(cL - 6395.5) < 1.0 and abs(cS - 3111.1) < 1.0
    c = cL if comp == 0 else cS
    N, h = 1029, 1e-3
    dt = 10 * h / c
    omega = 5 * np.pi * c / (N * h)
    Uf = lambda t: inputs.bell_pulse(t, 1e-6, omega, 4)
    # the right-going pulse and its periodic image stay apart in x < L/2 until t = L/(2c)
    nsteps = int(0.4 * N * h / c / dt)
    U = np.zeros((nsteps, 3))
    U[:, comp] = Uf(dt * np.arange(1, nsteps + 1))
    prob = _strip(N, N * h, AL_E, nu, AL_RHO, dt, U)
    x = (np.arange(N) + 0.5) * h
    n1 = int(0.25 * N * h / c / dt)
    centroid = lambda line: np.sum(line ** 2 * (x < 0.5 * N * h) * x) / np.sum(line ** 2 * (x < 0.5 * N * h))
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-12, maxit=400))
    gpu = {}
    for k in range(nsteps):
        info = s.step(U[k])
        assert info["status"] == 0
        if k + 1 in (n1, nsteps):
            gpu[k + 1] = centroid(s.get_state()[0][comp, 0, 1])
    s.close()
    orc = {}

    def cb(n, st, info):
        if n in (n1, nsteps):
            orc[n] = centroid(st.u[comp, 1])  # oracle 2-D fields are [c][N2][N1]

    newmark.oracle_from_problem(prob, tol=1e-12).run(U, callback=cb)
    v_gpu = (gpu[nsteps] - gpu[n1]) / ((nsteps - n1) * dt)
    v_orc = (orc[nsteps] - orc[n1]) / ((nsteps - n1) * dt)
    assert abs(v_gpu - v_orc) <= 1e-6 * c, (v_gpu, v_orc)
    assert abs(v_gpu - c) / c < 2e-2, (comp, v_gpu, c)


def _materials():
    """E (Pa) and rho of the paper's material table (tests/golden/table1_materials.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_materials.txt")
    out = {}
    with open(path) as f:
        for line in f:
            p = line.split()
            if p and not p[0].startswith("#"):
                out[p[0]] = (float(p[1]) * 1e9, float(p[2]))
    return out


@pytest.mark.parametrize("middle", ["Iron", "Uranium"])
@pytest.mark.parametrize("ratio", [5, 10])
def test_layered_bar_on_gpu_equals_the_layered_oracle_and_its_analytic_error(middle, ratio):
    """Sec. 3.1, Table 3: the bar of Table 2 with iron or uranium between 0.6 and 1.2 m (read
    in metres), as an N x 2 nu = 0 strip with a middle layer at N = 729; Delta t / CFL of the
    paper's N = 6561 bar taken on the fastest layer, Table 2's final time.  The GPU's final
    field equals the 1-D layered oracle's at the same N, and its error against the layered
    d'Alembert solution (App. C, interfaces at the voxel faces) is the oracle's."""
    from oracle import analytic, medium, newmark
    torch_cuda()
    wfft = solver_lib()
    mat = _materials()
    E = [mat[m][0] for m in ("Aluminium", middle, "Aluminium")]
    rho = [mat[m][1] for m in ("Aluminium", middle, "Aluminium")]
    c = [np.sqrt(e / r) for e, r in zip(E, rho)]
    Z = [r * ci for r, ci in zip(rho, c)]
    L, N = 2.0, 729
    h = L / N
    xc = (np.arange(N) + 0.5) * h
    ph = ((xc >= 0.6) & (xc < 1.2)).astype(np.int64)
    bounds = [0.0, np.argmax(ph) * h, (N - np.argmax(ph[::-1])) * h, L]
    Uf = lambda t: inputs.bell_pulse(t, 1e-3, 5 * np.pi * c[0] / L, 4)
    dt = ratio * (L / 6561) / max(c)
    nsteps = int(round(3.919e-4 / dt))
    U = np.zeros((nsteps, 3))
    U[:, 0] = Uf(dt * np.arange(1, nsteps + 1))
    # GPU: N x 2 plane-strain strip, nu = 0 in both materials
    Cs = np.stack([inputs.voigt21_from_matrix(inputs.isotropic_voigt(E[k], 0.0)) for k in (0, 1)])
    phase = np.broadcast_to(ph.astype(np.uint16), (1, 2, N)).copy()
    mask = np.zeros((2, 1, 2, N), np.uint8)
    mask[:, :, :, 0] = 1
    prob = inputs.Problem(f"layered_{middle}_{N}", 2, (N, 2, 1), (h, h, h), dt, 0.25, 0.5, Cs,
                          np.array([rho[0], rho[1]]), phase, mask, U, tol=1e-12)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-12, maxit=400))
    for k in range(nsteps):
        info = s.step(U[k])
        assert info["status"] == 0
    u = s.get_state()[0]
    s.close()
    ux = u[0, 0]
    assert np.abs(u[1]).max() <= 1e-12 * np.abs(ux).max()
    assert np.abs(ux[1] - ux[0]).max() <= 1e-12 * np.abs(ux).max()
    # oracle: the 1-D layered bar
    med = medium.Medium(1, (N,), (L,), np.array([E[0], E[1]]).reshape(2, 1, 1, 1, 1), ph,
                        np.where(ph == 1, rho[1], rho[0]))
    m1 = np.zeros((1, N), bool)
    m1[0, 0] = True
    so, _ = newmark.NewmarkOracle(med, m1, dt, tol=1e-12).run(U)
    uo = so.u[0]
    assert np.linalg.norm(ux[0] - uo) / np.linalg.norm(uo) < 1e-9
    ua = analytic.layered_dalembert_periodic(xc, nsteps * dt, bounds, c, Z, Uf)
    e_gpu = np.linalg.norm(ux[0] - ua) / np.linalg.norm(ua)
    e_orc = np.linalg.norm(uo - ua) / np.linalg.norm(ua)
    assert abs(e_gpu - e_orc) <= 1e-6 * e_orc
    assert e_gpu < 5e-2
