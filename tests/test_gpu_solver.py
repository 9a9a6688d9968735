"""GPU parity of whole beta-Newmark steps (Alg. 2 loop body) through the C ABI
against the FP64 oracle: FP64 path <= 1e-10 relative L2 (both sides solved to
1e-13, reading 6 of the Dirichlet/tolerance notes), mixed FP32+FP64-refinement
path <= 1e-6 against the oracle at tol 1e-10; edge cases and failure statuses."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import abi_field, oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _oracle_run(prob, tol, nsteps=None, warm="prev"):
    from oracle import newmark
    nm = newmark.oracle_from_problem(prob, tol=tol, warm=warm)
    s, infos = nm.run(prob.U, nsteps)
    return s, infos


def _gpu_run(prob, precision, tol, nsteps=None, warm=0, **kw):
    torch_cuda()
    wfft = solver_lib()
    opt = wfft.default_options(precision=precision, tol=tol, warm_start=warm, **kw)
    s = wfft.Solver.from_problem(prob, options=opt)
    infos = []
    for n in range(prob.nsteps if nsteps is None else nsteps):
        infos.append(s.step(prob.U[n]))
    u, v, a, nst = s.get_state()
    return (u, v, a), infos, s


STEP_CASES = [(2, (48, 40, 1), 2, False), (2, (30, 28, 1), 3, True), (3, (16, 12, 10), 2, False),
              (3, (20, 18, 14), 1, True), (3, (7, 9, 5), 2, False), (3, (24, 16, 8), 3, False)]


@pytest.mark.parametrize("ndim,n,width,dense", STEP_CASES)
def test_fp64_steps_match_oracle(ndim, n, width, dense):
    rng = np.random.default_rng(100 + sum(n))
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=width, nsteps=4, dense=dense, contrast=4.0,
                                 dt=4e-7)
    so, io = _oracle_run(prob, 1e-13)
    (u, v, a), ig, _ = _gpu_run(prob, 0, 1e-13)
    assert rel(oracle_field(prob, u), so.u) < 1e-10
    assert rel(oracle_field(prob, v), so.v) < 1e-9
    assert rel(oracle_field(prob, a), so.a) < 1e-8
    for g, o in zip(ig, io):
        assert abs(g["iters"] - o["iters"]) <= 1
        assert abs(g["ref"] - o["ref"]) <= 1e-12 * o["ref"]
        assert np.allclose(g["reaction"][:ndim], o["reaction"], rtol=1e-8, atol=1e-12 * max(1.0, abs(o["ref"])))


@pytest.mark.parametrize("ndim,n,width,dense", STEP_CASES[:4])
def test_mixed_steps_match_fp64_oracle(ndim, n, width, dense):
    rng = np.random.default_rng(200 + sum(n))
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=width, nsteps=6, dense=dense, contrast=4.0,
                                 dt=4e-7)
    so, _ = _oracle_run(prob, 1e-10)
    (u, v, a), ig, _ = _gpu_run(prob, 1, 1e-10)
    assert rel(oracle_field(prob, u), so.u) < 1e-6
    for g in ig:
        assert g["rel_res"] <= 1e-10 and g["outer_applies"] >= 1


def test_config_c1_fp64_matches_oracle_all_steps():
    """The 2-D 64x64 strip workload, 50 steps, FP64, tol 1e-10 on both sides."""
    prob = inputs.config_c1()
    so, io = _oracle_run(prob, 1e-13)
    (u, v, a), ig, _ = _gpu_run(prob, 0, 1e-13)
    assert rel(oracle_field(prob, u), so.u) < 1e-10
    (u2, _, _), ig2, _ = _gpu_run(prob, 0, 1e-10)
    so2, _ = _oracle_run(prob, 1e-10)
    # at the paper-style tolerance the gap is set by the two solvers' stopping points
    assert rel(oracle_field(prob, u2), so2.u) < 1e-8


def test_taylor_warm_start_same_solution_fewer_iterations():
    rng = np.random.default_rng(7)
    prob = inputs.random_problem(rng, 3, (16, 16, 12), nphase=3, mask_width=2, nsteps=6, contrast=3.0)
    prob.U[:, 0] = 1e-6 * np.sin(np.linspace(0.1, 0.6, 6))
    (u0, _, _), i0, _ = _gpu_run(prob, 0, 1e-12, warm=0)
    (u1, _, _), i1, _ = _gpu_run(prob, 0, 1e-12, warm=1)
    assert rel(u1, u0) < 1e-9
    assert sum(i["iters"] for i in i1) <= sum(i["iters"] for i in i0)


def test_solve_api_matches_oracle_masked_pcg():
    from oracle import newmark
    from oracle.pcg import masked_pcg
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(11)
    prob = inputs.random_problem(rng, 3, (12, 10, 8), nphase=3, mask_width=2, contrast=3.0)
    nm = newmark.oracle_from_problem(prob, tol=1e-13)
    b = rng.standard_normal((3,) + nm.med.shape)
    x0 = rng.standard_normal((3,) + nm.med.shape) * 0.1
    xg = np.where(nm.mask, x0, 0.0)
    xo, _ = masked_pcg(nm.A, nm.M, b, x0, nm.mask, xg, 1e-13)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-13))
    out = s.solve(abi_field(prob, b), abi_field(prob, x0), tol=1e-13)
    assert rel(oracle_field(prob, out["x"]), xo) < 1e-10
    assert np.array_equal(oracle_field(prob, out["x"])[nm.mask], x0[nm.mask])


def test_edge_cases_rest_homogeneous_and_no_mask():
    torch_cuda()
    wfft = solver_lib()
    # at rest with U = 0: ref = 0, the solution is x_Gamma = 0, no iteration
    prob = inputs.config_c1(nsteps=2)
    prob.U[:] = 0.0
    s = wfft.Solver.from_problem(prob)
    info = s.step(prob.U[0])
    assert info["iters"] == 0 and info["ref"] == 0.0
    u, v, a, n = s.get_state()
    assert not u.any() and not v.any() and not a.any() and n == 1
    # homogeneous medium, strip: the solver converges and the prescribed DOFs hold U
    prob = inputs.config_c1(nsteps=3)
    s = wfft.Solver.from_problem(prob)
    for k in range(3):
        s.step(prob.U[k])
    u, _, _, _ = s.get_state()
    assert np.allclose(u[0][prob.mask[0].astype(bool)], prob.U[2, 0], rtol=0, atol=0)
    # no prescribed region: free vibration from a smooth initial displacement
    rng = np.random.default_rng(3)
    p2 = inputs.random_problem(rng, 2, (32, 24, 1), nphase=2, mask_width=0, nsteps=3)
    s2 = wfft.Solver.from_problem(p2, options=wfft.default_options(tol=1e-13))
    from oracle import newmark
    nm = newmark.oracle_from_problem(p2, tol=1e-13)
    u0 = np.zeros((2, 1, 24, 32))
    yy, xx = np.meshgrid(np.arange(24), np.arange(32), indexing="ij")
    u0[0, 0] = 1e-6 * np.cos(2 * np.pi * xx / 32) * np.sin(2 * np.pi * 2 * yy / 24)
    s2.set_state(u0, None, None, 0)
    st = newmark.State(oracle_field(p2, u0).copy(), np.zeros((2, 24, 32)), np.zeros((2, 24, 32)))
    for k in range(3):
        s2.step(np.zeros(3))
        st, _ = nm.step(st, np.zeros(3))
    u, _, _, _ = s2.get_state()
    assert rel(oracle_field(p2, u), st.u) < 1e-10


def test_failure_statuses_leave_state_unchanged():
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(5)
    prob = inputs.random_problem(rng, 3, (12, 12, 8), nphase=4, mask_width=2, nsteps=3, contrast=6.0)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(tol=1e-12, maxit=2))
    before = s.get_state()
    info = s.step(prob.U[0], raise_on_error=False)
    assert info["rc"] == wfft.ENOTCONV
    after = s.get_state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
    assert after[3] == before[3]
    # the watchdog ends a mixed solve whose inner iterations are capped
    s2 = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=1, tol=1e-12, maxit=1,
                                                                      max_sweeps=3))
    info2 = s2.step(prob.U[0], raise_on_error=False)
    assert info2["rc"] in (wfft.ENOTCONV, wfft.ETIMEOUT)
    # invalid inputs are rejected before any device work
    with pytest.raises(wfft.WfftError) as e:
        wfft.Solver(3, (8, 8, 8), (1e-3,) * 3, prob.C, -np.abs(prob.rho), prob.phase[:8, :8, :8], None, 1e-7)
    assert e.value.code == wfft.EINVAL
    with pytest.raises(wfft.WfftError) as e:
        # 143 = 11 x 13: two prime factors above 7 (one direct prime stage per axis)
        wfft.Solver(3, (143, 8, 8), (1e-3,) * 3, prob.C, prob.rho, np.zeros((8, 8, 143), np.uint16), None, 1e-7)
    assert e.value.code == wfft.EUNSUPPORTED


def test_checkpoint_resume_is_bitwise():
    """Run 2k steps vs k steps + get_state/set_state into a fresh handle + k steps."""
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(8)
    prob = inputs.random_problem(rng, 3, (16, 12, 10), nphase=3, mask_width=2, nsteps=6, contrast=3.0)
    opt = wfft.default_options(tol=1e-11)
    a = wfft.Solver.from_problem(prob, options=opt)
    for k in range(6):
        a.step(prob.U[k])
    b = wfft.Solver.from_problem(prob, options=opt)
    for k in range(3):
        b.step(prob.U[k])
    st = b.get_state()
    c = wfft.Solver.from_problem(prob, options=opt)
    c.set_state(st[0], st[1], st[2], st[3])
    for k in range(3, 6):
        c.step(prob.U[k])
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)


def test_launch_count_is_a_lifetime_counter_across_profiling():
    """wfft_launch_count keeps counting through wfft_profile(1), which resets only
    the per-kind totals; the per-kind launches of a profiled step add up to the
    lifetime counter's increase."""
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(4), 3, (16, 12, 10), nphase=2, mask_width=2, nsteps=3)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=wfft.MIXED))
    s.step(prob.U[0])
    n0 = s.launch_count()
    assert n0 > 0
    s.profile(True)
    s.step(prob.U[1])
    n1 = s.launch_count()
    prof = s.profile_read()
    s.profile(False)
    assert n1 > n0
    assert sum(d["launches"] for d in prof.values()) == n1 - n0
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_cuda_graph_blocks_match_plain_launches_bitwise(precision):
    """use_graphs replays a captured block of check_every PCG iterations; it must
    compute exactly what plain launches compute (same kernels, same arguments),
    with the same iteration and kernel-launch counts, on the legacy default stream
    and on a user stream."""
    torch = torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(12), 3, (20, 16, 12), nphase=3, mask_width=2, nsteps=4)
    side = torch.cuda.Stream()
    for stream in (0, side.cuda_stream):
        runs = []
        for g in (1, 0):
            s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, use_graphs=g),
                                         stream=stream)
            n0 = s.launch_count()
            its = [s.step(prob.U[k])["iters"] for k in range(prob.nsteps)]
            runs.append((s.get_state()[:3], its, s.launch_count() - n0))
            s.close()
        (sa, ia, la), (sb, ib, lb) = runs
        assert all(np.array_equal(x, y) for x, y in zip(sa, sb))
        assert ia == ib and la == lb


@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-12, 1e-10), (1, 1e-10, 1e-6)])
def test_autotuned_plan_keeps_the_results(precision, tol, bar):
    """wfft_autotune may pick other radix decompositions and column-tile widths; the
    steps must still agree with the default plan and the oracle within the solver
    bars, and a second handle of the same grid takes the cached plan."""
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(21), 3, (32, 24, 16), nphase=3, mask_width=2, nsteps=3)
    opt = lambda: wfft.default_options(precision=precision, tol=tol)
    tuned = wfft.Solver.from_problem(prob, options=opt())
    changed = tuned.autotune(2)
    plain = wfft.Solver.from_problem(prob, options=opt())
    again = wfft.Solver.from_problem(prob, options=opt())
    assert again.autotune(2) == changed
    copied = wfft.Solver.from_problem(prob, options=opt())   # the tuned choices set by hand
    for pr in ([wfft.FP64] + ([wfft.MIXED] if precision == 1 else [])):
        copied.set_plan(pr, tuned.get_plan(pr))
        assert copied.get_plan(pr) == tuned.get_plan(pr)
    for k in range(prob.nsteps):
        for s in (tuned, plain, again, copied):
            assert s.step(prob.U[k])["status"] == 0
    ut, up, ua, uc = (s.get_state()[0] for s in (tuned, plain, again, copied))
    assert np.array_equal(ut, ua) and np.array_equal(ut, uc)
    assert rel(ut, up) < bar
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    assert rel(oracle_field(prob, ut), so.u) < bar
    for s in (tuned, plain, again, copied):
        s.close()


def test_inner_floor_keeps_the_accuracy_and_never_adds_iterations():
    """inner_floor lets an FP32 inner solve stop at a fraction of the outer target;
    the FP64 residual still decides convergence, so the steps stay within the mixed
    bar of the oracle, every step meets the tolerance, and no iterations are added."""
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = inputs.random_problem(np.random.default_rng(33), 3, (24, 20, 16), nphase=3, mask_width=2, nsteps=5)
    runs = {}
    for fl in (0.0, 0.5):
        opt = wfft.default_options(precision=wfft.MIXED, tol=1e-10)
        opt.inner_floor = fl
        s = wfft.Solver.from_problem(prob, options=opt)
        infos = [s.step(prob.U[k]) for k in range(prob.nsteps)]
        runs[fl] = (s.get_state()[0], infos)
        s.close()
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    for fl, (u, infos) in runs.items():
        assert rel(oracle_field(prob, u), so.u) < 1e-6
        assert all(i["rel_res"] <= 1e-10 * 1.0001 for i in infos)
    assert sum(i["iters"] for i in runs[0.5][1]) <= sum(i["iters"] for i in runs[0.0][1])


def test_async_download_matches_sync_and_is_ordered_before_state_writes():
    """wfft_download_async copies u_n (and v, a) while the next step runs: the copies equal
    the synchronous wfft_get_state bit for bit, and a state write issued right after the
    download (set_state) does not reach the copy."""
    torch = torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(31)
    prob = inputs.random_problem(rng, 3, (24, 20, 16), nphase=3, mask_width=2, nsteps=5, contrast=3.0)
    prob.U[:, 0] = 1e-6 * np.arange(1, 6)
    opts = wfft.default_options(precision=wfft.MIXED, tol=1e-10)
    ref = wfft.Solver.from_problem(prob, options=opts)
    want = []
    for k in range(prob.nsteps):
        ref.step(prob.U[k])
        want.append(ref.get_state()[0].copy())
    ref.close()
    s = wfft.Solver.from_problem(prob, options=opts)
    bufs = [torch.empty(s.shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(prob.nsteps)]
    for k in range(prob.nsteps):
        s.step(prob.U[k])
        s.download_async(bufs[k])
    s.download_wait()
    for k in range(prob.nsteps):
        assert np.array_equal(bufs[k], want[k]), k
    u, v, a = (torch.empty(s.shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3))
    u0, v0, a0, _ = s.get_state()
    s.download_async(u, v, a)
    s.set_state(np.zeros(s.shape), np.zeros(s.shape), np.zeros(s.shape))
    s.download_wait()
    assert np.array_equal(u, u0) and np.array_equal(v, v0) and np.array_equal(a, a0)
    assert not s.get_state()[0].any()
    with pytest.raises(ValueError):
        s.download_async(np.zeros(5))
    s.close()
