"""Grouped steps of uneven grids (wfft_batch_step): one launch per pass over
all unconverged instances must give the same states as stepping each handle on
its own (and as the FP64 oracle), in FP64 and mixed precision, also with axes that
have a prime factor above 7; an instance that fails does not commit while the
others do."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [(16, 16, 16), (24, 20, 12), (20, 16, 24), (32, 24, 16)]
# axes with a prime factor above 7 (direct prime-length stage), per instance
PRIME_SIZES = [(22, 13, 12), (43, 16, 6), (16, 11, 26)]


def _problems(seed, nsteps=4, sizes=SIZES):
    rng = np.random.default_rng(seed)
    probs = []
    for n in sizes:
        p = inputs.random_problem(rng, 3, n, nphase=3, mask_width=2, nsteps=nsteps, contrast=3.0, dt=4e-7)
        p.U[:, 0] = 1e-6 * np.sin(np.linspace(0.2, 1.0, nsteps)) * (1.0 + rng.random())
        probs.append(p)
    return probs


@pytest.mark.parametrize("sizes", [SIZES, PRIME_SIZES], ids=["smooth", "prime"])
@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-12, 1e-10), (1, 1e-10, 1e-6)])
def test_batched_steps_match_single_steps_and_oracle(precision, tol, bar, sizes):
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    probs = _problems(5, sizes=sizes)
    opt = lambda: wfft.default_options(precision=precision, tol=tol)
    grouped = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    single = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    n_incr = 0
    for k in range(probs[0].nsteps):
        U = np.stack([p.U[k] for p in probs])
        rc, infos = wfft.batch_step(grouped, U)
        assert rc == wfft.OK, infos
        for s, p in zip(single, probs):
            s.step(p.U[k])
        for inf in infos:
            assert inf["status"] == wfft.OK and inf["rel_res"] <= tol * 1.0001
            n_incr += inf["incr_resids"]
    if precision == 0:
        assert n_incr == 0
    for g, s, p in zip(grouped, single, probs):
        ug, vg, ag, ng = g.get_state()
        us, vs, as_, ns = s.get_state()
        assert ng == ns == p.nsteps
        assert rel(ug, us) < (1e-10 if precision == 0 else 1e-6)
        so, _ = newmark.oracle_from_problem(p, tol=1e-13).run(p.U)
        assert rel(oracle_field(p, ug), so.u) < bar


def test_batched_instance_failure_does_not_commit_and_others_do():
    torch_cuda()
    wfft = solver_lib()
    probs = _problems(9, nsteps=1)
    solvers = [wfft.Solver.from_problem(p, options=wfft.default_options(tol=1e-12, maxit=(2 if i == 1 else 500)))
               for i, p in enumerate(probs)]
    before = solvers[1].get_state()
    U = np.stack([p.U[0] for p in probs])
    rc, infos = wfft.batch_step(solvers, U)
    assert rc == wfft.ENOTCONV
    assert infos[1]["status"] == wfft.ENOTCONV
    assert all(infos[i]["status"] == wfft.OK for i in (0, 2, 3))
    after = solvers[1].get_state()
    assert all(np.array_equal(x, y) for x, y in zip(before[:3], after[:3])) and after[3] == 0
    assert all(solvers[i].get_state()[3] == 1 for i in (0, 2, 3))


def test_mixed_structure_falls_back_to_one_by_one():
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(3)
    p2 = inputs.random_problem(rng, 2, (32, 24, 1), nphase=2, mask_width=2, nsteps=1)
    p3 = inputs.random_problem(rng, 3, (16, 12, 8), nphase=2, mask_width=2, nsteps=1)
    s = [wfft.Solver.from_problem(p) for p in (p2, p3)]
    U = np.stack([p2.U[0], p3.U[0]])
    rc, infos = wfft.batch_step(s, U)
    assert rc == wfft.OK and all(i["status"] == wfft.OK for i in infos)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_graph_blocks_match_plain_launches_bitwise(precision):
    """Grouped PCG blocks replayed as CUDA graphs compute exactly what direct launches do."""
    torch_cuda()
    wfft = solver_lib()
    probs = _problems(9, nsteps=3)
    states = {}
    for graphs in (1, 0):
        hs = [wfft.Solver.from_problem(p, options=wfft.default_options(precision=precision, tol=1e-10,
                                                                       use_graphs=graphs)) for p in probs]
        iters = []
        for k in range(probs[0].nsteps):
            rc, infos = wfft.batch_step(hs, np.stack([p.U[k] for p in probs]))
            assert rc == wfft.OK, infos
            iters.append([i["iters"] for i in infos])
        states[graphs] = ([h.get_state()[0] for h in hs], iters)
        for h in hs:
            h.close()
    assert states[1][1] == states[0][1]
    for a, b in zip(states[1][0], states[0][0]):
        assert np.array_equal(a, b)


def test_batched_mixed_steps_take_the_incremental_residual():
    """Polycrystal pulses of uneven sizes: the grouped mixed solve replaces its last FP64
    residual by the incremental one when every instance's rounding estimate allows it,
    and the grouped states equal the single solves' within the solver tolerance."""
    torch_cuda()
    wfft = solver_lib()
    probs = []
    for n, seed in (((24, 24, 24), 31), ((32, 24, 20), 32), ((20, 28, 24), 33)):
        ids, Cv, rho = inputs.polycrystal(n, 12, seed)
        dt = 2e-7
        U = inputs._U_series(6, dt, lambda t: inputs.gaussian_pulse(t, 1e-6, 5 * dt, 15 * dt))
        probs.append(inputs.Problem(f"pulse{n}", 3, n, (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                                    inputs.slab_mask(3, n, 4), U, tol=1e-10))
    opt = lambda: wfft.default_options(precision=wfft.MIXED, tol=1e-10)
    grouped = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    single = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    n_incr, outer = 0, 0
    for k in range(probs[0].nsteps):
        rc, infos = wfft.batch_step(grouped, np.stack([p.U[k] for p in probs]))
        assert rc == wfft.OK, infos
        for s, p in zip(single, probs):
            s.step(p.U[k])
        n_incr += sum(i["incr_resids"] for i in infos)
        outer += sum(i["outer_applies"] for i in infos)
        assert all(i["rel_res"] <= 1e-10 for i in infos)
    print(n_incr, outer)
    assert n_incr > 0
    for g, s in zip(grouped, single):
        assert rel(g.get_state()[0], s.get_state()[0]) < 1e-8


# ten uneven instances, two with a prime factor above 7 on an axis
MANY = [(16, 16, 16), (24, 20, 12), (20, 16, 24), (32, 24, 16), (12, 18, 10), (40, 16, 8), (22, 13, 12),
        (16, 11, 26), (30, 12, 20), (48, 8, 8)]


def _own_schedule(wfft, s, precision, i):
    """Instance i's own plan: column-tile widths cycling through 1, 2, 4 per instance and
    pass, and on the x axis a radix schedule that differs from the built-in one where the
    length allows (16 = 4 x 4 or 2 x 8)."""
    pl = s.get_plan(precision)
    for a in (1, 2):
        for o in range(5):
            trial = [[*r] for r in pl["bx"]]
            trial[a][o] = (1, 2, 4)[(i + a + o) % 3]
            try:
                s.set_plan(precision, {**pl, "bx": trial})
                pl = s.get_plan(precision)
            except wfft.WfftError:
                pass
    if s.n[0] == 16:
        cnt = [0, 2, 0, 0, 0, 0, 0] if i % 2 else [1, 0, 1, 0, 0, 0, 0]
        s.set_radix(precision, 0, cnt)
    return s.get_plan(precision)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10)])
def test_many_instances_with_their_own_schedules_match_single_steps(precision, tol):
    """Ten instances, each with its own radix schedule and column-tile widths (the grouped
    column passes then run one launch per width): grouped steps equal single-handle steps
    with the same plans, and the instances' plans really differ."""
    torch_cuda()
    wfft = solver_lib()
    probs = _problems(21, nsteps=3, sizes=MANY)
    opt = lambda: wfft.default_options(precision=precision, tol=tol)  # noqa: E731
    grouped = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    single = [wfft.Solver.from_problem(p, options=opt()) for p in probs]
    precs = (wfft.FP64,) if precision == 0 else (wfft.FP64, wfft.MIXED)
    widths = set()
    for i, (g, s) in enumerate(zip(grouped, single)):
        for pr in precs:
            pl = _own_schedule(wfft, g, pr, i)
            s.set_plan(pr, pl)
            widths.add(tuple(pl["bx"][1]))
    assert len(widths) > 1
    for k in range(probs[0].nsteps):
        U = np.stack([p.U[k] for p in probs])
        rc, infos = wfft.batch_step(grouped, U)
        assert rc == wfft.OK, infos
        for s, p, inf in zip(single, probs, infos):
            i1 = s.step(p.U[k])
            assert inf["status"] == wfft.OK and inf["rel_res"] <= tol * 1.0001
            assert abs(inf["iters"] - i1["iters"]) <= 1
    for g, s in zip(grouped, single):
        ug = g.get_state()[0]
        us = s.get_state()[0]
        assert rel(ug, us) < (1e-10 if precision == 0 else 1e-7)
